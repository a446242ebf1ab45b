"""The learned tile proposer's tensor-core kernels against the CPU oracle (oracle/net_oracle.py): each convolution
layer (forward, gated input gradient, weight gradient) and the whole loss gradient.

Tolerances.  Stored tensors are bf16 on both sides; a product sum of the GPU (fp32, tensor-core order) and of the
oracle (fp32 or fp64, numpy order) differ by rounding only, so a bf16 output differs by at most one bf16 rounding
(2^-8 relative) where the two sums straddle a rounding boundary.  Gradients accumulate such rare flips through four
layers.  The whole gradient is therefore compared element by element against one bf16 rounding (2^-8) of the sum of
the magnitudes of the terms that make up each element (net_oracle.grad_magnitudes); the oracle with its bf16
roundings switched off misses that bound, so it tells the rounding points apart."""
import numpy as np
import pytest

import paper_2408_14050_gb300 as occ
import scenes
from oracle import net_oracle as net

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAIRS = [(8, 16), (16, 16), (16, 32), (32, 16)]


@pytest.fixture(scope="module", autouse=True)
def need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_bf16(a):
    return torch.from_numpy(net.bf16(a)).cuda().to(torch.bfloat16)


def pack_weights(Wt):
    """[co][9][ci] -> [co][K] with k = tap * ci + c, zero up to K = 9 ci rounded up to 16."""
    co, _, ci = Wt.shape
    K = (9 * ci + 15) // 16 * 16
    out = np.zeros((co, K), np.float32)
    out[:, :9 * ci] = Wt.reshape(co, 9 * ci)
    return out


def conv_ref(X, Wt, b):
    """float64 3x3 'same' convolution of n images."""
    return np.stack([net.conv3x3_same(x.astype(np.float64), Wt.astype(np.float64), b.astype(np.float64)) for x in X])


@pytest.mark.parametrize("ci,co", PAIRS)
@pytest.mark.parametrize("shape", [(1, 5, 7), (2, 13, 37), (3, 32, 64)])
def test_conv_layer_forward_and_gated(ci, co, shape):
    rng = np.random.default_rng(ci * 100 + co + shape[1])
    n, H, W = shape
    X = net.bf16(rng.normal(size=(n, H, W, ci)).astype(np.float32))
    Wt = net.bf16((rng.normal(size=(co, 9, ci)) / np.sqrt(9 * ci)).astype(np.float32))
    b = rng.normal(size=co).astype(np.float32)
    gate = net.bf16(rng.normal(size=(n, H, W, co)).astype(np.float32))
    Wb = to_bf16(pack_weights(Wt))
    Xg = to_bf16(X)
    ref = conv_ref(X, Wt, b)
    Y = occ.occ_net_conv3x3(Xg, Wb, bias=torch.from_numpy(b).cuda(), relu=True).float().cpu().numpy()
    exp = np.maximum(ref, 0)
    assert np.all(np.abs(Y - exp) <= 2.0 ** -8 * np.abs(exp) + 1e-5)
    Yg = occ.occ_net_conv3x3(Xg, Wb, gate=to_bf16(gate)).float().cpu().numpy()
    exp = np.where(gate > 0, ref - b, 0.0)
    assert np.all(np.abs(Yg - exp) <= 2.0 ** -8 * np.abs(exp) + 1e-5)
    assert occ.occ_net_status() == occ.OCC_OK


@pytest.mark.parametrize("ci,co", [pc for pc in PAIRS if pc[0] >= 16])
@pytest.mark.parametrize("shape", [(4, 192, 256), (5, 150, 230)])
def test_conv_persistent_ctas_walk_several_blocks(ci, co, shape):
    """The tensor-memory convolution runs at most four CTAs per multiprocessor, each walking output blocks of 16 x 8
    pixels b, b + grid, b + 2 grid, ... and loading the block after next into the halo buffer it has just freed.
    With more than twice as many blocks as CTAs (1,536 and 1,450 blocks against at most 4 x 152), every CTA takes a
    second block and most a third, so both halo buffers are reused; the second shape leaves ragged blocks on the
    right and bottom edges.  Forward with bias and ReLU, and the gated form of the input gradient."""
    n, H, W = shape
    nblk = n * ((H + 15) // 16) * ((W + 7) // 8)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert nblk > 2 * min(nblk, 4 * sms)
    rng = np.random.default_rng(ci * 1000 + co + H)
    X = net.bf16(rng.normal(size=(n, H, W, ci)).astype(np.float32))
    Wt = net.bf16((rng.normal(size=(co, 9, ci)) / np.sqrt(9 * ci)).astype(np.float32))
    b = rng.normal(size=co).astype(np.float32)
    gate = net.bf16(rng.normal(size=(n, H, W, co)).astype(np.float32))
    Wb = to_bf16(pack_weights(Wt))
    Xg = to_bf16(X)
    ref = conv_ref(X, Wt, b)
    Y = occ.occ_net_conv3x3(Xg, Wb, bias=torch.from_numpy(b).cuda(), relu=True).float().cpu().numpy()
    exp = np.maximum(ref, 0)
    assert np.all(np.abs(Y - exp) <= 2.0 ** -8 * np.abs(exp) + 1e-5)
    Yg = occ.occ_net_conv3x3(Xg, Wb, gate=to_bf16(gate)).float().cpu().numpy()
    exp = np.where(gate > 0, ref - b, 0.0)
    assert np.all(np.abs(Yg - exp) <= 2.0 ** -8 * np.abs(exp) + 1e-5)
    assert occ.occ_net_status() == occ.OCC_OK


@pytest.mark.parametrize("ci,co", PAIRS)
@pytest.mark.parametrize("shape", [(1, 9, 11), (2, 40, 70)])
def test_conv_weight_gradient(ci, co, shape):
    rng = np.random.default_rng(ci + co * 7 + shape[2])
    n, H, W = shape
    X = net.bf16(rng.normal(size=(n, H, W, ci)).astype(np.float32))
    dY = net.bf16(rng.normal(size=(n, H, W, co)).astype(np.float32))
    dWt = occ.occ_net_conv3x3_wgrad(to_bf16(X), to_bf16(dY)).cpu().numpy()
    exp = np.zeros((9 * ci + 1, co))
    mag = np.zeros((9 * ci + 1, co))
    for t, (dy, dx) in enumerate(net.TAPS):
        for k in range(n):
            S = net.shifted(X[k].astype(np.float64), dy, dx)
            exp[t * ci:(t + 1) * ci] += np.einsum("yxi,yxo->io", S, dY[k])
            mag[t * ci:(t + 1) * ci] += np.einsum("yxi,yxo->io", np.abs(S), np.abs(dY[k]))
    exp[9 * ci] = dY.sum(axis=(0, 1, 2))
    mag[9 * ci] = np.abs(dY).sum(axis=(0, 1, 2))
    assert np.all(np.abs(dWt - exp) <= 1e-5 * mag + 1e-6)
    # Accumulates into the given buffer.
    twice = occ.occ_net_conv3x3_wgrad(to_bf16(X), to_bf16(dY), dWt=torch.from_numpy(dWt).cuda()).cpu().numpy()
    assert np.all(np.abs(twice - 2 * exp) <= 2e-5 * mag + 2e-6)   # partial sums arrive in any order


def frames_and_labels(n, H, W, views, seed):
    Ds = [scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(80 + seed, k)) for k in range(n)]
    rng = np.random.default_rng(seed)
    labels = (rng.random((n, len(views), (H + 31) // 32, (W + 31) // 32)) < 0.5).astype(np.uint8)
    return np.stack(Ds), labels


def block_slices():
    off = 0
    for li, (ci, co) in enumerate(net.LAYERS):
        yield f"W{li + 1}", slice(off, off + co * 9 * ci)
        off += co * 9 * ci
        yield f"b{li + 1}", slice(off, off + co)
        off += co
    yield "We", slice(off, off + 48)
    yield "be", slice(off + 48, off + 64)
    yield "b0", slice(off + 64, off + 65)


def assert_gradient_elementwise(got, exp_g, mag, unrounded=None):
    """|got - exp| <= 2^-8 * (sum of the magnitudes of the element's terms) + 1e-9 for every element; and, where the
    oracle's gradient without bf16 roundings is given, that it does not meet the same bound."""
    tol = 2.0 ** -8 * mag + 1e-9
    bad = np.abs(got - exp_g) > tol
    for name, sl in block_slices():
        assert not bad[sl].any(), (name, float((np.abs(got - exp_g)[sl] / tol[sl]).max()))
    if unrounded is not None:
        assert (np.abs(unrounded - exp_g) > tol).any()
    return float((np.abs(got - exp_g) / tol).max())


@pytest.mark.parametrize("n,H,W", [(2, 64, 80), (4, 192, 256)])
def test_logits_loss_and_gradients_match_the_oracle(n, H, W):
    """(2, 64, 80): 2 x 3 tiles per frame, the last column partial.  (4, 192, 256): 1,536 output blocks per
    convolution, so the persistent CTAs of the three tensor-memory layers walk several blocks each."""
    views = scenes.views_3x3()
    Ds, labels = frames_and_labels(n, H, W, views, 1)
    p = scenes.net_init(5)
    p = p + np.random.default_rng(6).normal(size=p.size).astype(np.float32) * 0.02
    m = occ.Net(0, max_pixels=Ds.size, max_views=8)
    m.set_params(p)
    np.testing.assert_array_equal(m.get_params(), p)
    D = torch.from_numpy(Ds).cuda()
    lab = torch.from_numpy(labels).cuda()
    logits = torch.empty(labels.shape, dtype=torch.float32, device="cuda")
    loss, g = m.loss_grad(D, views, lab, pos_weight=2.0, logits=logits)
    fw = m.forward(D, views).cpu().numpy()
    assert occ.occ_net_status() == occ.OCC_OK
    exp_loss, exp_g, exp_s, mag, unr = 0.0, np.zeros(p.size), [], np.zeros(p.size), np.zeros(p.size)
    for k in range(len(Ds)):
        lk, gk = net.loss_and_grads(p, Ds[k], views, labels[k], pos_weight=2.0)
        exp_loss += lk / len(Ds)
        exp_g += gk / len(Ds)
        mag += net.grad_magnitudes(p, Ds[k], views, labels[k], pos_weight=2.0) / len(Ds)
        unr += net.loss_and_grads(p, Ds[k], views, labels[k], 2.0, np.float64, rounding=False)[1] / len(Ds)
        exp_s.append(net.forward(p, Ds[k], views)["s"])
    exp_s = np.stack(exp_s)
    np.testing.assert_allclose(fw, exp_s, rtol=1e-3, atol=1e-3)
    np.testing.assert_allclose(logits.cpu().numpy(), exp_s, rtol=1e-3, atol=1e-3)
    assert abs(float(loss.item()) - exp_loss) <= 1e-3 * abs(exp_loss)
    got = g.cpu().numpy()
    worst = assert_gradient_elementwise(got, exp_g, mag, unrounded=unr)
    print(f"gradient: largest error {worst:.3g} of the element-wise bound")
    m.close()


def test_adam_steps_reduce_the_loss_on_plain_method_labels():
    """Labels of the plain method (per-tile hit flags) on frames of mixed noise; Adam on the GPU lowers the loss."""
    from paper_2408_14050_gb300 import learned
    views = scenes.views_3x3()
    Ds = scenes.proposer_frames(16, 96, 128, seed=12)
    D = torch.from_numpy(Ds).cuda()
    ctx = occ.occ_create(0, max_pixels=Ds.size, max_views=8)
    lab = learned.labels_for(ctx, D, views)
    ctx.close()
    frac = float(lab.float().mean().item())
    assert 0.05 < frac < 0.95, frac
    m = occ.Net(0, max_pixels=Ds.size, max_views=8)
    m.set_params(scenes.net_init(9))
    first = float(m.loss_grad(D, views, lab)[0].item())
    for step in range(1, 101):
        _, g = m.loss_grad(D, views, lab)
        m.adam(g, step, lr=3e-3)
    last = float(m.loss_grad(D, views, lab)[0].item())
    assert last < 0.8 * first, (first, last)
    s = m.forward(D, views)
    prop = occ.occ_net_propose(s, 0.0)
    np.testing.assert_array_equal(prop.cpu().numpy(), (s.cpu().numpy() > 0).astype(np.uint8))
    assert occ.occ_net_status() == occ.OCC_OK
    m.close()
