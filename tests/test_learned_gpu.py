"""The learned tile proposer end to end on the GPU: labels from the plain method, training with the library's own
kernels, calibration for a pixel recall target, and use with occ_detect_batched_tiles.  What it gains over the plain
method (tiles skipped, time) is printed; what must hold is asserted: the fallback semantics (skipping nothing is the
plain method bit for bit, skipping a tile only removes hits, so precision is 1), the calibrated recall, and that
training lowers the held-out loss."""
import numpy as np
import pytest

import paper_2408_14050_gb300 as occ
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14050_gb300 import learned
    views = scenes.views_3x3()
    H, W = 96, 128
    Dtr = torch.from_numpy(scenes.proposer_frames(768, H, W, seed=41)).cuda()
    Dva = torch.from_numpy(scenes.proposer_frames(64, H, W, seed=41, first=10 ** 6)).cuda()
    ctx = occ.occ_create(0, max_pixels=64 * H * W, max_views=8)
    Ltr = learned.labels_for(ctx, Dtr, views)
    Lva = learned.labels_for(ctx, Dva, views)
    net = occ.Net(0, max_pixels=1 << 21, max_views=8)
    net.set_params(scenes.net_init(2))
    before = float(net.loss_grad(Dva, views, Lva)[0].item())
    learned.train(net, Dtr, Ltr, views, epochs=3, batch=32, lr=2e-3)
    after = float(net.loss_grad(Dva, views, Lva)[0].item())
    yield {"net": net, "ctx": ctx, "views": views, "Dva": Dva, "before": before, "after": after}
    ctx.close()
    net.close()


def test_training_lowers_the_held_out_loss(trained):
    print(f"held-out loss {trained['before']:.4f} -> {trained['after']:.4f}")
    assert trained["after"] < 0.9 * trained["before"]


def test_calibrated_threshold_meets_the_recall_target_and_masks_are_subsets(trained):
    from paper_2408_14050_gb300 import learned
    net, ctx, views, Dva = trained["net"], trained["ctx"], trained["views"], trained["Dva"]
    frames = [Dva[i] for i in range(Dva.shape[0])]
    th, rec, skipped = learned.calibrate(net, ctx, frames, views, target_recall=0.999)
    print(f"threshold {th:.4f}: pixel recall {rec:.5f}, tiles skipped {skipped:.4f}")
    assert rec >= 0.999
    logits = learned.logits_for(net, frames, views)
    props = [occ.occ_net_propose(s, th) for s in logits]
    M_plain, O_plain = occ.occ_detect_batched(ctx, frames, views)
    M_prop, O_prop = occ.occ_detect_batched(ctx, frames, views, proposals=props)
    for a, b, oa, ob in zip(M_plain, M_prop, O_plain, O_prop):
        assert bool(((b != 0) & (a == 0)).sum().item() == 0)   # nothing new is marked
        assert bool((ob <= oa).all())                          # counts only drop
    r, p = learned.recall_precision(M_plain, M_prop)
    assert p == 1.0 and abs(r - rec) < 1e-12


def test_threshold_extremes_are_the_plain_method_and_nothing(trained):
    from paper_2408_14050_gb300 import learned
    net, ctx, views, Dva = trained["net"], trained["ctx"], trained["views"], trained["Dva"]
    frames = [Dva[i] for i in range(8)]
    logits = learned.logits_for(net, frames, views)
    M_plain, O_plain = occ.occ_detect_batched(ctx, frames, views)
    keep_all = [occ.occ_net_propose(s, -float("inf")) for s in logits]
    M_all, O_all = occ.occ_detect_batched(ctx, frames, views, proposals=keep_all)
    for a, b, oa, ob in zip(M_plain, M_all, O_plain, O_all):
        assert torch.equal(a, b) and torch.equal(oa, ob)
    skip_all = [occ.occ_net_propose(s, float("inf")) for s in logits]
    M_none, O_none = occ.occ_detect_batched(ctx, frames, views, proposals=skip_all)
    assert all(int(m.sum().item()) == 0 for m in M_none)


def test_gain_over_the_plain_method_is_measured(trained):
    """Reports the trade on mixed-noise frames of the training distribution; the numbers are printed, the checks are
    that the learned run is a valid run (recall >= target there is not guaranteed: calibration was on other frames)."""
    from paper_2408_14050_gb300 import learned
    net, ctx, views = trained["net"], trained["ctx"], trained["views"]
    frames = [torch.from_numpy(f).cuda() for f in scenes.proposer_frames(16, 96, 128, seed=43)]
    th, _, _ = learned.calibrate(net, ctx, frames, views)
    ev = learned.evaluate(net, ctx, frames, views, th, reps=3)
    print({k: (round(v, 4) if isinstance(v, float) else v) for k, v in ev.items()})
    assert ev["precision"] == 1.0 and ev["recall"] >= 0.999
    assert 0.0 <= ev["skipped_tiles"] <= 1.0 and ev["ms_plain"] > 0 and ev["ms_learned"] > 0
