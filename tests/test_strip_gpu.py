"""The strip kernel (k_strip): views whose scan lines stay on one row, column, diagonal or anti-diagonal, one block
per strip of such lines with D_r and O in shared memory.  Its results must be the oracle's bit for bit, and equal
those of the candidate-list kernels (strip_px = 0), for every strip shape; frames it does not take (a side above
4096 pixels, N != 8) fall back to the list kernels; lines of three or more macro-runs go to the warp sort, in the
strip's own warps or, past what a strip keeps, through the view's list in the warp kernel, and still give the
oracle's O and M."""
import numpy as np
import pytest

import oracle
import paper_2408_14050_gb300 as occ
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OCTANT = scenes.views_3x3()


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = occ.occ_create(0, max_pixels=4100 * 600, max_views=24)
    yield c
    c.close()


def tuning(strip_px, fused=0):
    return {"line_max_runs": 2, "line_blocks_per_sm": 1, "warp_lines_per_block": 8, "strip_px": strip_px,
            "fused": fused}


def detect(ctx, D, views, strip_px, fused=0, **kw):
    occ.occ_set_tuning(ctx, tuning(strip_px, fused))
    try:
        d = dict(gamma=1.0, zeta=2.0, beta=0.5, L=0, N=8)
        d.update(kw)
        M, O = occ.occ_detect(ctx, torch.from_numpy(np.ascontiguousarray(D)).cuda(), views,
                              occ.occ_default_params(**d))
        assert occ.occ_get_status(ctx) == occ.OCC_OK
        return M.cpu().numpy(), O.cpu().numpy(), occ.occ_get_stats(ctx, len(views))
    finally:
        occ.occ_set_tuning(ctx, None)


def check_oracle(D, views, M, O, stats, **kw):
    d = dict(gamma=1.0, zeta=2.0, beta=0.5, L=0, N=8)
    d.update(kw)
    po = oracle.default_params(**d)
    for v, (a, r) in enumerate(views):
        Oo, Mo, st = oracle.detect_view(D, a, r, po)
        np.testing.assert_array_equal(O[v], Oo, err_msg=f"O view {v} alpha={a} r={r}")
        np.testing.assert_array_equal(M[v], Mo, err_msg=f"M view {v} alpha={a} r={r}")
        for k in ("candidates", "samples", "pair_tests", "L"):
            assert stats[v][k] == st[k], (v, a, k, stats[v][k], st[k])


@pytest.mark.parametrize("shape", [(270, 480), (480, 270), (97, 301), (301, 97), (1, 64), (64, 1), (5, 5)])
@pytest.mark.parametrize("strip_px", [1024, 4096, 16384])
@pytest.mark.parametrize("fused", [1, 0])
def test_strip_shapes_match_the_oracle(ctx, shape, strip_px, fused):
    """Strips of 1 to 16 lines (rows, columns and both diagonals; wide, tall, one-pixel maps; 1024 pixels is raised to
    the longest line), in the fused launch and in separate launches, against the oracle and against the
    candidate-list kernels."""
    H, W = shape
    D = scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(90, H * 7 + W)) if min(H, W) > 8 else \
        np.random.default_rng(H + W).uniform(0, 30, (H, W)).astype(np.float32)
    M, O, st = detect(ctx, D, OCTANT, strip_px, fused)
    check_oracle(D, OCTANT, M, O, st)
    M0, O0, st0 = detect(ctx, D, OCTANT, 0)
    np.testing.assert_array_equal(O, O0)
    np.testing.assert_array_equal(M, M0)
    assert st == st0


@pytest.mark.parametrize("fused", [0, 1])
def test_full_frame_strip_and_list_paths_agree(ctx, fused):
    D = scenes.array_3x3(frame=2, H=540, W=960).frames[0]
    M, O, st = detect(ctx, D, OCTANT, occ.STRIP_PX_DEFAULT, fused)
    M0, O0, st0 = detect(ctx, D, OCTANT, 0)
    np.testing.assert_array_equal(O, O0)
    np.testing.assert_array_equal(M, M0)
    assert st == st0
    check_oracle(D, OCTANT, M, O, st)


@pytest.mark.parametrize("strip_px", [1024, 4096])
@pytest.mark.parametrize("list_view", [True, False])
def test_lines_of_many_runs_go_to_the_warp_sort(ctx, strip_px, list_view):
    """Uniform noise breaks scan lines into many macro-runs, which the warp sort of the list path takes.  With a view
    off the strip directions (20 degrees) the call runs in separate launches and the strips list these lines for the
    warp kernel.  Without it the call is one fused launch: with the automatic L (h <= 100) a strip keeps up to 16 such
    lines and publishes them for the worker blocks once its O is written, and lists the rest; with a fixed L of 300
    (h = 150, the 1024 class) or 1100 (the 4096 class) it lists them all, for the workers once every strip is done.
    Strips of 1024 pixels leave the workers shared room for fewer warp buffers than strips of 4096."""
    rng = np.random.default_rng(8)
    D = rng.uniform(0, 40, (64, 160)).astype(np.float32)
    views = [(0.0, 1.0), (45.0, 2.5), (90.0, 1.0), (135.0, 1.0), (180.0, 2.0), (225.0, 1.0), (270.0, 1.0),
             (315.0, 1.5)] + ([(20.0, 1.0)] if list_view else [])
    for L in (0, 300, 1100):
        M, O, st = detect(ctx, D, views, strip_px, 0 if list_view else 1, L=L)
        check_oracle(D, views, M, O, st, L=L)


def test_frames_above_the_strip_limit_use_the_lists(ctx):
    """A side above 4096 pixels, or N != 8: every view takes the candidate-list kernels, with the same results."""
    D = scenes.make_scene(scenes.spec_array(12, 4100), scenes.seed_of(91, 0))
    M, O, st = detect(ctx, D, OCTANT[:4], occ.STRIP_PX_DEFAULT)
    check_oracle(D, OCTANT[:4], M, O, st)
    D = scenes.make_scene(scenes.spec_array(90, 130), scenes.seed_of(91, 1))
    for N in (4, 16):
        M, O, st = detect(ctx, D, OCTANT, occ.STRIP_PX_DEFAULT, N=N)
        check_oracle(D, OCTANT, M, O, st, N=N)


@pytest.mark.parametrize("fused", [0, 1])
def test_strips_in_batches_and_graphs(ctx, fused):
    """Uneven frames of one batch (strips of each frame after the previous frame's), captured in a CUDA graph and
    replayed on new inputs, in separate launches and in the fused launch (whose published-line entries carry a tag
    that changes with every launch, replays included)."""
    sizes = [(48, 64), (100, 77), (270, 480), (31, 200), (1, 9), (129, 130)]
    views = OCTANT
    first = [scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(92, i)) if min(H, W) > 8 else
             np.full((H, W), 3.0, np.float32) for i, (H, W) in enumerate(sizes)]
    second = [f[::-1, ::-1].copy() for f in first]
    Ds = [torch.from_numpy(f).cuda() for f in first]
    Ms = [torch.empty((len(views), *D.shape), dtype=torch.uint8, device="cuda") for D in Ds]
    Os = [torch.empty((len(views), *D.shape), dtype=torch.int32, device="cuda") for D in Ds]
    occ.occ_set_tuning(ctx, tuning(occ.STRIP_PX_DEFAULT, fused))
    try:
        occ.occ_detect_batched(ctx, Ds, views, Ms=Ms, Os=Os)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            occ.occ_detect_batched(ctx, Ds, views, Ms=Ms, Os=Os)
        # Two replays on different inputs: the second must not take the first one's lines.
        for inputs in (second, first):
            for f_np, D in zip(inputs, Ds):
                D.copy_(torch.from_numpy(f_np).cuda())
            g.replay()
            torch.cuda.synchronize()
            assert occ.occ_get_status(ctx) == occ.OCC_OK
            for f_np, M, O in zip(inputs, Ms, Os):
                for v, (a, r) in enumerate(views):
                    Oo, Mo, _ = oracle.detect_view(f_np, a, r)
                    np.testing.assert_array_equal(O[v].cpu().numpy(), Oo)
                    np.testing.assert_array_equal(M[v].cpu().numpy(), Mo)
    finally:
        occ.occ_set_tuning(ctx, None)


def test_fused_launch_wait_bound_and_recovery(ctx):
    """The fused launch's waits are bounded: with the plans of the frames withheld (the test hook) and a bound of
    2 ms, every strip's wait gives up, the call reports OCC_ERR_TIMEOUT and the launch ends; the next call, with the
    hook off, is exact again on the same context."""
    D = scenes.make_scene(scenes.spec_array(97, 301), scenes.seed_of(93, 0))
    occ.occ_set_tuning(ctx, tuning(4096, fused=1))
    try:
        occ.occ_set_wait_limit(ctx, 2000, hold=True)
        occ.occ_detect(ctx, torch.from_numpy(D).cuda(), OCTANT)
        assert occ.occ_get_status(ctx) == occ.OCC_ERR_TIMEOUT
    finally:
        occ.occ_set_wait_limit(ctx, 0, hold=False)
        occ.occ_set_tuning(ctx, None)
    M, O, st = detect(ctx, D, OCTANT, occ.STRIP_PX_DEFAULT, fused=1)
    check_oracle(D, OCTANT, M, O, st)
    with pytest.raises(occ.OccError):
        occ.occ_set_wait_limit(ctx, -1)


@pytest.mark.parametrize("n_frames", [5, 130])
def test_fused_batches_of_many_frames(ctx, n_frames):
    """Batches past the few frames of the small launch-parameter table (5), and past the fused launch's 128 frames
    (130, which run in separate launches): every frame against the oracle."""
    rng = np.random.default_rng(n_frames)
    sizes = [(int(rng.integers(9, 40)), int(rng.integers(9, 40))) for _ in range(n_frames)]
    frames = [scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(94, i)) for i, (H, W) in enumerate(sizes)]
    Ds = [torch.from_numpy(f).cuda() for f in frames]
    Ms = [torch.empty((len(OCTANT), *D.shape), dtype=torch.uint8, device="cuda") for D in Ds]
    Os = [torch.empty((len(OCTANT), *D.shape), dtype=torch.int32, device="cuda") for D in Ds]
    occ.occ_set_tuning(ctx, tuning(occ.STRIP_PX_DEFAULT, fused=1))
    try:
        occ.occ_detect_batched(ctx, Ds, OCTANT, Ms=Ms, Os=Os)
        torch.cuda.synchronize()
        assert occ.occ_get_status(ctx) == occ.OCC_OK
    finally:
        occ.occ_set_tuning(ctx, None)
    for f_np, M, O in zip(frames, Ms, Os):
        for v, (a, r) in enumerate(OCTANT):
            Oo, Mo, _ = oracle.detect_view(f_np, a, r)
            np.testing.assert_array_equal(O[v].cpu().numpy(), Oo)
            np.testing.assert_array_equal(M[v].cpu().numpy(), Mo)


def test_fused_option_falls_back_without_room():
    """A context too small for the fused launch's work lists (its warp buffers) takes the separate launches with
    fused = 1, with the same results."""
    D = scenes.make_scene(scenes.spec_array(64, 96), scenes.seed_of(95, 0))
    c = occ.occ_create(0, max_pixels=64 * 96, max_views=8, max_candidates=4096)
    try:
        M, O, st = detect(c, D, OCTANT, occ.STRIP_PX_DEFAULT, fused=1)
        check_oracle(D, OCTANT, M, O, st)
    finally:
        c.close()
