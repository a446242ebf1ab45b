"""occ_detect_batched: many frames of uneven size and the same views in one batch of launches.

Every frame's M and O must equal, bit for bit, both the oracle's and occ_detect's on that frame alone; the batch must
be capturable into a CUDA graph and give the same results on replay with new inputs; statuses and statistics must
aggregate over the frames.
"""
import numpy as np
import pytest

import oracle
import paper_2408_14050_gb300 as occ
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = occ.occ_create(0, max_pixels=24 * 1024 * 1024, max_views=8)
    yield c
    c.close()


def uneven_frames(seed=0):
    sizes = [(48, 64), (100, 77), (270, 480), (31, 200), (1, 9), (129, 130)]
    out = []
    for i, (H, W) in enumerate(sizes):
        spec = scenes.SceneSpec(H=H, W=W, bg_base=(2.0, 6.0), bg_slope=(2.0, 8.0), n_objects=4, obj_disp=(8.0, 24.0),
                                obj_size=(0.1, 0.5), d_max=64.0, sigma=0.3)
        out.append(scenes.make_scene(spec, scenes.seed_of(30 + seed, i)))
    return out


def test_batch_matches_oracle_frame_by_frame(ctx):
    frames = uneven_frames()
    views = scenes.views_3x3()
    Ds = [torch.from_numpy(f).cuda() for f in frames]
    Ms, Os = occ.occ_detect_batched(ctx, Ds, views)
    assert occ.occ_get_status(ctx) == occ.OCC_OK
    stats = occ.occ_get_stats(ctx, len(views))
    exp_samples = [0] * len(views)
    for D, M, O in zip(frames, Ms, Os):
        for v, (a, r) in enumerate(views):
            Oo, Mo, st = oracle.detect_view(D, a, r)
            np.testing.assert_array_equal(O[v].cpu().numpy(), Oo)
            np.testing.assert_array_equal(M[v].cpu().numpy(), Mo)
            exp_samples[v] += st["samples"]
    assert [s["samples"] for s in stats] == exp_samples


def test_batch_of_mixed_sizes_matches_single_frame_calls(ctx):
    wl = scenes.mixed_batch(n_frames=6, sizes=[(480, 640), (720, 1280), (1080, 1920)])
    views = wl.views
    Ds = [torch.from_numpy(f).cuda() for f in wl.frames]
    Ms, Os = occ.occ_detect_batched(ctx, Ds, views)
    assert occ.occ_get_status(ctx) == occ.OCC_OK
    for D, M, O in zip(Ds, Ms, Os):
        M1, O1 = occ.occ_detect(ctx, D, views)
        assert occ.occ_get_status(ctx) == occ.OCC_OK
        assert torch.equal(O, O1) and torch.equal(M, M1)


def test_large_batch_takes_chunks_from_a_counter(ctx):
    # Above 64 Mi pixel-views per call the line kernel hands out its chunks from a counter (a kernel variant of its
    # own); the results are those of the single-frame calls, and of the oracle.
    wl = scenes.mixed_batch(n_frames=5, sizes=[(1080, 1920)])
    views = wl.views
    assert sum(f.size for f in wl.frames) * len(views) > 64 * 1024 * 1024
    Ds = [torch.from_numpy(f).cuda() for f in wl.frames]
    Ms, Os = occ.occ_detect_batched(ctx, Ds, views)
    assert occ.occ_get_status(ctx) == occ.OCC_OK
    for D, M, O in zip(Ds, Ms, Os):
        M1, O1 = occ.occ_detect(ctx, D, views)
        assert torch.equal(O, O1) and torch.equal(M, M1)
    po = oracle.default_params(gamma=1.0, zeta=2.0, beta=0.5, L=0, N=8)
    for v, (a, r) in enumerate(views):
        Oo, Mo, _ = oracle.detect_view(wl.frames[0], a, r, po)
        assert np.array_equal(Os[0][v].cpu().numpy(), Oo) and np.array_equal(Ms[0][v].cpu().numpy(), Mo)


def test_batch_captured_in_a_cuda_graph(ctx):
    views = scenes.views_3x3()
    first = uneven_frames(seed=1)
    second = uneven_frames(seed=2)
    Ds = [torch.from_numpy(f).cuda() for f in first]
    Ms = [torch.empty((len(views), *D.shape), dtype=torch.uint8, device="cuda") for D in Ds]
    Os = [torch.empty((len(views), *D.shape), dtype=torch.int32, device="cuda") for D in Ds]
    occ.occ_detect_batched(ctx, Ds, views, Ms=Ms, Os=Os)          # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        occ.occ_detect_batched(ctx, Ds, views, Ms=Ms, Os=Os)
    for f_np, D in zip(second, Ds):
        D.copy_(torch.from_numpy(f_np).cuda())
    g.replay()
    torch.cuda.synchronize()
    for f_np, M, O in zip(second, Ms, Os):
        for v, (a, r) in enumerate(views):
            Oo, Mo, _ = oracle.detect_view(f_np, a, r)
            np.testing.assert_array_equal(O[v].cpu().numpy(), Oo)
            np.testing.assert_array_equal(M[v].cpu().numpy(), Mo)


def test_batch_status_is_the_or_of_the_frames(ctx):
    frames = uneven_frames()
    frames[2] = frames[2].copy()
    frames[2][5, 7] = np.nan
    Ds = [torch.from_numpy(f).cuda() for f in frames]
    occ.occ_detect_batched(ctx, Ds, [(0.0, 1.0)])
    assert occ.occ_get_status(ctx) == occ.OCC_ERR_NONFINITE_INPUT


def test_batch_argument_checks(ctx):
    D = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(occ.OccError):
        occ.occ_detect_batched(ctx, [D] * 2, [])
    big = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
    with pytest.raises(occ.OccError):                 # 2 x 16.8 M pixels > max_pixels
        occ.occ_detect_batched(ctx, [big, big], [(0.0, 1.0)])


def test_batch_of_the_mixed_resolutions_against_the_oracle(ctx):
    """One batch holding a 4096x2160, a 640x480 and a 1280x720 map of the mixed-resolution recipe (disparity 0-64,
    eight views).  The two smaller frames are compared with the oracle whole; the 4096x2160 frame on a 24x24 window
    per view, with the oracle run on every candidate whose scan line can reach the window (all of the window's O)."""
    from test_parity_gpu import reach_mask
    wl = scenes.mixed_batch(n_frames=3, sizes=[(2160, 4096), (480, 640), (720, 1280)], config=33)
    views = wl.views
    assert sorted(f.shape for f in wl.frames) == [(480, 640), (720, 1280), (2160, 4096)]
    Ds = [torch.from_numpy(f).cuda() for f in wl.frames]
    Ms, Os = occ.occ_detect_batched(ctx, Ds, views)
    assert occ.occ_get_status(ctx) == occ.OCC_OK
    po = oracle.default_params()
    rng = np.random.default_rng(33)
    for D, M, O in zip(wl.frames, Ms, Os):
        H, W = D.shape
        O_np, M_np = O.cpu().numpy(), M.cpu().numpy()
        np.testing.assert_array_equal(M_np, (O_np > 0).astype(np.uint8))
        for v, (a, r) in enumerate(views):
            if H * W <= 1280 * 720:
                Oo, Mo, _ = oracle.detect_view(D, a, r, po)
                np.testing.assert_array_equal(O_np[v], Oo, err_msg=f"{W}x{H} view {v}")
                np.testing.assert_array_equal(M_np[v], Mo, err_msg=f"{W}x{H} view {v}")
            else:
                h = (oracle.scan_length(D, r) + 1) // 2
                c, s = (float(t) for t in oracle.direction(a))
                bx, by = int(rng.integers(0, W - 24)), int(rng.integers(0, H - 24))
                box = (bx, by, bx + 24, by + 24)
                Oo, _ = oracle.detect_view_masked(D, a, r, po, reach_mask(H, W, box, c, s, h))
                np.testing.assert_array_equal(O_np[v][by:by + 24, bx:bx + 24], Oo[by:by + 24, bx:bx + 24],
                                              err_msg=f"{W}x{H} view {v} alpha={a}")
