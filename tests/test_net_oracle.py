"""Pins of the learned tile proposer's CPU oracle (oracle/net_oracle.py) against what does not depend on it: scipy's
2-D correlation, scipy's log-sum-exp, torch's bfloat16 rounding, and finite differences of its own loss in float64
(a wrong sign, index or transposed operand anywhere in the backward pass fails the last one)."""
import numpy as np
import pytest

import scenes
from oracle import net_oracle as net

scipy_signal = pytest.importorskip("scipy.signal")
scipy_special = pytest.importorskip("scipy.special")


def test_param_layout_matches_the_shared_initializer():
    assert net.param_count() == scenes.net_param_count() == len(scenes.net_init(0))
    layers, We, be, b0 = net.unpack(scenes.net_init(3))
    assert [w.shape for w, _ in layers] == [(co, 9, ci) for ci, co in net.LAYERS]
    np.testing.assert_array_equal(net.pack(layers, We, be, b0), scenes.net_init(3))
    assert not layers[0][0][:, :, 1:].any()          # first layer reads channel 0 only


def test_conv_is_scipy_correlation_with_zero_padding():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(9, 13, 5)).astype(np.float64)
    Wt = rng.normal(size=(4, 9, 5))
    b = rng.normal(size=4)
    Y = net.conv3x3_same(X, Wt, b)
    for co in range(4):
        exp = b[co] + sum(scipy_signal.correlate2d(X[..., ci], Wt[co, :, ci].reshape(3, 3), mode="same")
                          for ci in range(5))
        np.testing.assert_allclose(Y[..., co], exp, rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]]).astype(np.float32)
    exp = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(net.bf16(x), exp)


def test_tile_logits_are_log_mean_exp():
    D = scenes.make_scene(scenes.spec_array(70, 50), 5)
    views = [(0.0, 1.0), (135.0, float(np.float32(np.sqrt(2.0))))]
    fw = net.forward(scenes.net_init(7), D, views)
    z, s = fw["z"], fw["s"]
    assert s.shape == (2, 3, 2)
    for v in range(2):
        for i, j, ys, xs in net.tiles(70, 50):
            zt = z[v, ys, xs].astype(np.float64).ravel()
            np.testing.assert_allclose(s[v, i, j], scipy_special.logsumexp(zt) - np.log(zt.size), rtol=1e-5,
                                       atol=1e-5)


def test_gradients_match_finite_differences_in_float64():
    rng = np.random.default_rng(2)
    H, W = 20, 37                                    # two tile columns, one partial
    D = scenes.make_scene(scenes.spec_array(H, W), 9).astype(np.float64)
    views = [(0.0, 1.0), (225.0, 1.5)]
    p = scenes.net_init(11).astype(np.float64)
    p += rng.normal(size=p.size) * 0.05              # non-zero biases, first-layer weights on every channel
    labels = np.array([[[1, 0]], [[0, 1]]], dtype=np.float64)
    loss, g = net.loss_and_grads(p, D, views, labels, pos_weight=3.0, dtype=np.float64, rounding=False)
    # Every parameter block: a few entries each (conv weights of each layer, biases, encoding, output bias).
    idx = []
    off = 0
    for ci, co in net.LAYERS:
        idx += list(off + rng.choice(co * 9 * ci, 6, replace=False))
        off += co * 9 * ci
        idx += list(off + rng.choice(co, 2, replace=False))
        off += co
    idx += list(off + rng.choice(net.FEATURES * net.ENC, 4, replace=False)) + [off + 48 + 3, off + 48 + 16]
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp, _ = net.loss_and_grads(pp, D, views, labels, 3.0, np.float64, False)
        lm, _ = net.loss_and_grads(pm, D, views, labels, 3.0, np.float64, False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8, (k, fd, g[k])
