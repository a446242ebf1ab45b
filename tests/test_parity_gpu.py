"""Parity of the CUDA path (through the C ABI) with the CPU oracle, on the same seeded inputs.

M, O, the candidate counts, the sample counts and the pair-test counts must be bit-exact; E must be bit-exact and
A within 1e-5 relative (1e-6 absolute near 0).  Sizes span several tiles and ragged tails; full-size maps that
the oracle cannot finish in seconds are checked on sampled windows, recomputed by the oracle from exactly the
candidates whose scan lines can reach them.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2408_14050_gb300 as occ
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def both_params(**kw):
    d = dict(gamma=1.0, zeta=2.0, beta=0.5, L=0, N=8)
    d.update(kw)
    return oracle.default_params(**d), occ.occ_default_params(**d)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = occ.occ_create(0, max_pixels=4096 * 2160, max_views=24)
    yield c
    c.close()


def run_gpu(ctx, D, views, p=None, E=False, pitch_pad=0):
    Dt = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    if pitch_pad:
        wide = torch.zeros((D.shape[0], D.shape[1] + pitch_pad), dtype=torch.float32, device="cuda")
        wide[:, :D.shape[1]] = Dt
        Dt = wide[:, :D.shape[1]]
    Et = torch.empty(D.shape, dtype=torch.float32, device="cuda") if E else None
    At = torch.empty(D.shape, dtype=torch.float32, device="cuda") if E else None
    M, O = occ.occ_detect(ctx, Dt, views, p, E=Et, A=At)
    status = occ.occ_get_status(ctx)
    stats = occ.occ_get_stats(ctx, len(views))
    out = dict(M=M.cpu().numpy(), O=O.cpu().numpy(), status=status, stats=stats)
    if E:
        out["E"], out["A"] = Et.cpu().numpy(), At.cpu().numpy()
    return out


def assert_exact(ctx, D, views, kw=None, pitch_pad=0):
    po, pg = both_params(**(kw or {}))
    g = run_gpu(ctx, D, views, pg, pitch_pad=pitch_pad)
    assert g["status"] == occ.OCC_OK, occ.occ_status_string(g["status"])
    for v, (a, r) in enumerate(views):
        O, M, st = oracle.detect_view(D, a, r, po)
        np.testing.assert_array_equal(g["O"][v], O, err_msg=f"O view {v} alpha={a} r={r}")
        np.testing.assert_array_equal(g["M"][v], M, err_msg=f"M view {v}")
        for k in ("candidates", "samples", "pair_tests", "L"):
            assert g["stats"][v][k] == st[k], (v, k, g["stats"][v][k], st[k])
    return g


def noisy_map(H, W, seed, scale=6.0):
    rng = np.random.default_rng(seed)
    base = np.cumsum(rng.normal(0, 0.3, (H, W)), axis=1) * 0.2 + 10
    steps = (rng.random((H, W)) < 0.05) * rng.uniform(-scale, scale, (H, W))
    return (base + np.cumsum(steps, axis=1)).astype(np.float32)


# ---------------------------------------------------------------------------------------------------------------
# The workloads

def test_stereo_pair_exact(ctx):
    wl = scenes.stereo_pair()
    assert_exact(ctx, wl.frames[0], wl.views)


def test_array_3x3_full_size_exact(ctx):
    wl = scenes.array_3x3()
    g = assert_exact(ctx, wl.frames[0], wl.views)
    assert sum(s["samples"] for s in g["stats"]) > 50_000_000


@pytest.mark.parametrize("size", [(480, 640), (720, 1280)])
def test_mixed_batch_sizes_exact(ctx, size):
    H, W = size
    D = scenes.make_scene(scenes.spec_array(H, W), scenes.seed_of(3, 7))
    assert_exact(ctx, D, scenes.views_3x3())


def reach_mask(H, W, box, c, s, h, pad=2):
    """Candidates whose scan line (2h+1 samples along (c, s), nearest-pixel rounding) can land in box."""
    x0, y0, x1, y1 = box
    m = np.zeros((H, W), np.uint8)
    for g in range(-h - 1, h + 2):
        dx, dy = int(math.floor(c * g + 0.5)), int(math.floor(s * g + 0.5))
        xa, xb = max(0, x0 - pad - dx), min(W, x1 + pad - dx)
        ya, yb = max(0, y0 - pad - dy), min(H, y1 + pad - dy)
        if xa < xb and ya < yb:
            m[ya:yb, xa:xb] = 1
    return m


def test_stress_5x5_full_size_sampled(ctx):
    wl = scenes.stress_5x5()
    D = wl.frames[0]
    H, W = D.shape
    po, pg = both_params()
    g = run_gpu(ctx, D, wl.views, pg)
    assert g["status"] == occ.OCC_OK
    rng = np.random.default_rng(11)
    for v, (a, r) in enumerate(wl.views):
        st = g["stats"][v]
        assert st["L"] == oracle.scan_length(D, r)
        assert st["candidates"] == len(oracle.candidates(D, a, r))
        h = (st["L"] + 1) // 2
        c, s = (float(t) for t in oracle.direction(a))
        bx, by = int(rng.integers(0, W - 24)), int(rng.integers(0, H - 24))
        box = (bx, by, bx + 24, by + 24)
        O, _ = oracle.detect_view_masked(D, a, r, po, reach_mask(H, W, box, c, s, h))
        np.testing.assert_array_equal(g["O"][v][by:by + 24, bx:bx + 24], O[by:by + 24, bx:bx + 24],
                                      err_msg=f"view {v} alpha={a}")
        np.testing.assert_array_equal(g["M"][v], (g["O"][v] > 0).astype(np.uint8))


# ---------------------------------------------------------------------------------------------------------------
# Shapes, strides, angles, parameters

@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (2, 2), (5, 13), (33, 67), (70, 251), (129, 130)])
def test_ragged_shapes_exact(ctx, shape):
    H, W = shape
    D = noisy_map(H, W, seed=H * 1000 + W)
    views = [(0.0, 1.0), (90.0, 1.0), (135.0, 1.4142135), (200.5, 1.7), (333.25, 1.0)]
    assert_exact(ctx, D, views, dict(L=24))
    assert_exact(ctx, D, views)


@pytest.mark.parametrize("pad", [1, 3, 64])
def test_row_pitch(ctx, pad):
    D = noisy_map(40, 77, seed=pad)
    assert_exact(ctx, D, [(0.0, 1.0), (45.0, 1.4142135), (250.0, 1.0)], dict(L=30), pitch_pad=pad)


@pytest.mark.parametrize("runs", [2, 0])
def test_row_pitch_beyond_32_bit_offsets(ctx, runs):
    # A map whose last row starts more than 2^31 elements after its first: the kernels' element offsets into D take
    # 64 bits (the wide variants of the line, merge and warp kernels).  The rows live in one 8.7 GB buffer.
    H, W = 64, 96
    pitch = (1 << 25) + (1 << 20)
    assert (H - 1) * pitch + W > 2**31 - 1
    D = noisy_map(H, W, seed=31)
    big = torch.empty((H - 1) * pitch + W, dtype=torch.float32, device="cuda")
    try:
        Dt = big.as_strided((H, W), (pitch, 1))
        Dt.copy_(torch.from_numpy(D).cuda())
        views = [(0.0, 1.0), (45.0, 1.4142135), (160.0, 1.0), (270.0, 1.0)]
        po, pg = both_params(N=8)
        occ.occ_set_tuning(ctx, {"line_max_runs": runs, "line_blocks_per_sm": 1, "warp_lines_per_block": 8})
        try:
            M, O = occ.occ_detect(ctx, Dt, views, pg)
            assert occ.occ_get_status(ctx) == occ.OCC_OK
            stats = occ.occ_get_stats(ctx, len(views))
        finally:
            occ.occ_set_tuning(ctx, None)
        M, O = M.cpu().numpy(), O.cpu().numpy()
        for v, (a, r) in enumerate(views):
            Ov, Mv, st = oracle.detect_view(D, a, r, po)
            np.testing.assert_array_equal(O[v], Ov, err_msg=f"O view {v}")
            np.testing.assert_array_equal(M[v], Mv, err_msg=f"M view {v}")
            for k in ("candidates", "samples", "pair_tests", "L"):
                assert stats[v][k] == st[k], (v, k)
    finally:
        del big
        torch.cuda.empty_cache()


@pytest.mark.parametrize("kw", [dict(N=2), dict(N=4), dict(N=6), dict(N=16), dict(N=64), dict(zeta=0.75), dict(zeta=3.5),
                                dict(beta=0.0), dict(beta=2.0), dict(gamma=0.25), dict(gamma=3.0)])
def test_parameters_exact(ctx, kw):
    D = scenes.make_scene(scenes.SPEC_STEREO, scenes.seed_of(1, 5))[:96, :160].copy()
    assert_exact(ctx, D, [(0.0, 1.0), (45.0, 1.4142135), (180.0, 1.0), (300.0, 2.0)], kw)


@pytest.mark.parametrize("runs", [0, 1, 2])
@pytest.mark.parametrize("N", [4, 8])
def test_scan_work_mappings_exact(ctx, runs, N):
    # A noisy map whose scan lines are one, two and more macro-runs, under each mapping of the scan work: every line
    # on the warp kernel (0); the line kernel keeping lines of one macro-run (1), and of two as well (2).  The line
    # kernel streams every line, takes broken lines' counts back out of O and hands them on; O, M and the work counts
    # must not change.
    D = noisy_map(120, 200, seed=11)
    occ.occ_set_tuning(ctx, {"line_max_runs": runs, "line_blocks_per_sm": 1, "warp_lines_per_block": 8})
    try:
        assert_exact(ctx, D, [(0.0, 1.0), (45.0, 1.4142135), (160.0, 1.0), (270.0, 1.0)], dict(N=N))
    finally:
        occ.occ_set_tuning(ctx, None)


@pytest.mark.parametrize("L", [1, 2, 254, 255, 256, 600, 1022, 1023, 2000, 4094])
def test_scan_length_classes_exact(ctx, L):
    # Scan lines of 2h+1 samples run in the kernel sized for them (<= 256, <= 1024, <= 4096 samples).
    D = noisy_map(24, 300, seed=L)
    assert_exact(ctx, D, [(0.0, 1.0), (30.0, 1.0), (180.0, 1.3)], dict(L=L))


def test_many_runs_use_the_bucket_sort_exact(ctx):
    # Salt-and-pepper maps break scan lines into many monotone runs (more than the run merge handles), which the warp
    # kernel sorts by W bucket and transposition passes.
    rng = np.random.default_rng(5)
    D = rng.uniform(0, 40, (48, 200)).astype(np.float32)
    assert_exact(ctx, D, [(0.0, 1.0), (60.0, 1.0), (225.0, 2.5)], dict(L=300))
    assert_exact(ctx, D, [(10.0, 1.0)], dict(L=1500))


@pytest.mark.parametrize("alpha", list(np.arange(0.0, 360.0, 15.0)) + [7.3, 89.99, 181.0])
def test_all_angles_exact(ctx, alpha):
    D = scenes.make_scene(scenes.SPEC_STEREO, scenes.seed_of(1, 9))
    assert_exact(ctx, D, [(float(alpha), 1.0), (float(alpha), 2.25)])


def test_rectangle_band(ctx):
    D = np.full((48, 64), 3, np.float32)
    D[12:28, 20:38] = 8
    assert_exact(ctx, D, [(0.0, 1.0), (90.0, 1.0), (180.0, 2.0), (270.0, 1.0)])


def test_constant_map_is_empty(ctx):
    D = np.full((37, 53), 5.5, np.float32)
    g = run_gpu(ctx, D, scenes.views_3x3(), both_params()[1])
    assert g["status"] == occ.OCC_OK
    assert not g["O"].any() and not g["M"].any()
    assert all(s["candidates"] == 0 and s["samples"] == 0 for s in g["stats"])


def test_edge_and_angle_maps(ctx):
    D = scenes.array_3x3().frames[0]
    g = run_gpu(ctx, D, [(0.0, 1.0)], both_params()[1], E=True)
    E, A = oracle.edges(D)
    np.testing.assert_array_equal(g["E"], E)
    np.testing.assert_allclose(g["A"], A, rtol=1e-5, atol=1e-6)


def test_repeat_is_deterministic(ctx):
    D = scenes.array_3x3(frame=1, H=540, W=960).frames[0]
    a = run_gpu(ctx, D, scenes.views_3x3(), both_params()[1])
    b = run_gpu(ctx, D, scenes.views_3x3(), both_params()[1])
    np.testing.assert_array_equal(a["O"], b["O"])
    np.testing.assert_array_equal(a["M"], b["M"])
    assert a["stats"] == b["stats"]


@pytest.mark.parametrize("runs", [2, 1])
def test_profiled_call_times_its_stages(runs):
    # With profiling on, a call records its stage boundaries; the warp kernels run on the context's second stream
    # beside the merge kernel (whichever lines the line kernel keeps) and their stages count from where they start.
    # The results do not change, and they are the oracle's.
    D = scenes.array_3x3(frame=1, H=540, W=960).frames[0]
    views = scenes.views_3x3()
    c = occ.occ_create(0, max_pixels=D.size, max_views=len(views))
    try:
        occ.occ_set_tuning(c, {"line_max_runs": runs, "line_blocks_per_sm": 3, "warp_lines_per_block": 8})
        plain = run_gpu(c, D, views, both_params()[1])
        with pytest.raises(occ.OccError):
            occ.occ_get_timings(c)                # no profiled call yet
        occ.occ_set_profiling(c, True)
        try:
            prof = run_gpu(c, D, views, both_params()[1])
            t = occ.occ_get_timings(c)
        finally:
            occ.occ_set_profiling(c, False)
    finally:
        c.close()
    np.testing.assert_array_equal(prof["O"], plain["O"])
    np.testing.assert_array_equal(prof["M"], plain["M"])
    po = both_params()[0]
    for v, (a, r) in enumerate(views):
        Oo, Mo, _ = oracle.detect_view(D, a, r, po)
        np.testing.assert_array_equal(plain["O"][v], Oo, err_msg=f"O view {v}")
        np.testing.assert_array_equal(plain["M"][v], Mo, err_msg=f"M view {v}")
    assert set(t) == set(occ.STAGES)
    assert all(v >= 0.0 for v in t.values()), t
    assert t["scan_lines"] > 0.0 and t["candidates"] > 0.0 and t["mask"] > 0.0, t


def test_host_buffer_entry_point(ctx):
    D = scenes.array_3x3(frame=2, H=270, W=480).frames[0]
    views = scenes.views_3x3()
    pin_D = torch.from_numpy(D).pin_memory()
    M = torch.empty((8, 270, 480), dtype=torch.uint8).pin_memory()
    O = torch.empty((8, 270, 480), dtype=torch.int32).pin_memory()
    rc, _, _ = occ.occ_detect_host(ctx, pin_D, views, both_params()[1], M=M, O=O)
    assert rc == occ.OCC_OK
    po = both_params()[0]
    for v, (a, r) in enumerate(views):
        Oo, Mo, _ = oracle.detect_view(D, a, r, po)
        np.testing.assert_array_equal(O[v].numpy(), Oo)
        np.testing.assert_array_equal(M[v].numpy(), Mo)


def test_host_buffer_calls_queued_on_two_contexts():
    # occ_detect_host_async on two contexts and two streams, frames alternating and overlapping on the GPU: every
    # frame's M and O are those of the synchronous call.
    views = scenes.views_3x3()
    frames = [scenes.array_3x3(frame=f, H=270, W=480).frames[0] for f in range(4)]
    ctxs = [occ.occ_create(0, max_pixels=270 * 480, max_views=8) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pins = [torch.from_numpy(f).pin_memory() for f in frames]
    Ms = [torch.empty((8, 270, 480), dtype=torch.uint8).pin_memory() for _ in frames]
    Os = [torch.empty((8, 270, 480), dtype=torch.int32).pin_memory() for _ in frames]
    try:
        for i in range(len(frames)):
            j = i & 1
            if i >= 2:
                assert occ.occ_get_status(ctxs[j], streams[j]) == occ.OCC_OK
            rc, _, _ = occ.occ_detect_host(ctxs[j], pins[i], views, both_params()[1], M=Ms[i], O=Os[i],
                                           stream=streams[j], wait=False)
            assert rc == occ.OCC_OK
        for j in range(2):
            assert occ.occ_get_status(ctxs[j], streams[j]) == occ.OCC_OK
        for i, D in enumerate(frames):
            M = torch.empty((8, 270, 480), dtype=torch.uint8).pin_memory()
            O = torch.empty((8, 270, 480), dtype=torch.int32).pin_memory()
            rc, _, _ = occ.occ_detect_host(ctxs[0], pins[i], views, both_params()[1], M=M, O=O)
            assert rc == occ.OCC_OK
            assert torch.equal(M, Ms[i]) and torch.equal(O, Os[i])
    finally:
        for c in ctxs:
            c.close()


# ---------------------------------------------------------------------------------------------------------------
# Device-detected errors (status word; no fault, no trap)

def test_nonfinite_input_status(ctx):
    D = noisy_map(30, 40, seed=1)
    D[7, 9] = np.nan
    assert run_gpu(ctx, D, [(0.0, 1.0)])["status"] == occ.OCC_ERR_NONFINITE_INPUT
    D[7, 9] = np.inf
    assert run_gpu(ctx, D, [(0.0, 1.0)])["status"] == occ.OCC_ERR_NONFINITE_INPUT
    D[7, 9] = 1.0
    assert run_gpu(ctx, D, [(0.0, 1.0)])["status"] == occ.OCC_OK


def test_candidate_overflow_status():
    # A list-path view (10 degrees) with more candidates than the list holds; a strip view (0 degrees) whose scan lines
    # of three or more macro-runs (uniform noise) exceed it: with L = 300 they are longer than the strip kernel keeps
    # for its own warps, and all go to the list.  A constant map has none.
    c = occ.occ_create(0, max_pixels=64 * 64, max_views=2, max_candidates=10)
    try:
        D = noisy_map(64, 64, seed=2, scale=20)
        assert run_gpu(c, D, [(10.0, 1.0)])["status"] == occ.OCC_ERR_CAPACITY
        U = np.random.default_rng(3).uniform(0, 40, (64, 64)).astype(np.float32)
        assert run_gpu(c, U, [(0.0, 1.0)], both_params(L=300)[1])["status"] == occ.OCC_ERR_CAPACITY
        assert run_gpu(c, np.full((64, 64), 1.0, np.float32), [(0.0, 1.0)])["status"] == occ.OCC_OK
    finally:
        c.close()


@pytest.mark.parametrize("spare", [0, 64])
def test_two_run_lines_without_room_in_the_list_go_to_the_warp_kernel(spare):
    # The line kernel's list of the merge kernel holds one entry per candidate the context can hold; the pairs of the
    # two-run merges live in the entries the call's candidates leave free.  A context sized to the view's candidates
    # leaves none (every two-run line falls back to the warp kernel), or room for 32 pairs; the results must not
    # change.
    D = noisy_map(120, 200, seed=11)
    a, r = 45.0, 1.4142135
    po, pg = both_params()
    O, M, st = oracle.detect_view(D, a, r, po)
    c = occ.occ_create(0, max_pixels=D.size, max_views=1, max_candidates=st["candidates"] + spare)
    try:
        g = run_gpu(c, D, [(a, r)], pg)
        assert g["status"] == occ.OCC_OK, occ.occ_status_string(g["status"])
        np.testing.assert_array_equal(g["O"][0], O)
        np.testing.assert_array_equal(g["M"][0], M)
        for k in ("candidates", "samples", "pair_tests", "L"):
            assert g["stats"][0][k] == st[k], k
    finally:
        c.close()


def test_scan_too_long_status(ctx):
    D = np.zeros((16, 16), np.float32)
    D[3, 3] = 3000.0      # Eq. 3 gives L = 6000 > OCC_MAX_SCAN
    assert run_gpu(ctx, D, [(0.0, 1.0)])["status"] == occ.OCC_ERR_CAPACITY


def test_invalid_arguments(ctx):
    D = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    for kw in (dict(N=3), dict(N=0), dict(N=66), dict(zeta=0.0), dict(gamma=float("nan")), dict(L=5000)):
        with pytest.raises(occ.OccError) as e:
            occ.occ_detect(ctx, D, [(0.0, 1.0)], occ.occ_default_params(**kw))
        assert e.value.status == occ.OCC_ERR_INVALID_ARG
    for views in ([(0.0, 0.0)], [(0.0, -1.0)], [(float("inf"), 1.0)], [(0.0, float("nan"))], []):
        with pytest.raises(occ.OccError):
            occ.occ_detect(ctx, D, views)
    with pytest.raises(occ.OccError):
        occ.occ_detect(ctx, D, [(0.0, 1.0)] * 25)


@pytest.mark.parametrize("gamma", [0.0, 0.1, 0.25, 1.0, 3.0])
def test_edge_threshold_boundaries_exact(ctx, gamma):
    """Forward differences placed on and around the edge threshold of Eq. 2 (a few ulps either side, and pairs
    E_x, E_y whose squares sum to the boundary), so that the strict E > gamma is tested where rounding decides it."""
    rng = np.random.default_rng(int(gamma * 100) + 1)
    g = np.float32(gamma)
    near = [g]
    v = g
    for _ in range(4):
        v = np.nextafter(v, np.float32(np.inf))
        near.append(v)
    v = g
    for _ in range(4):
        v = np.nextafter(v, np.float32(-np.inf))
        near.append(v)
    near = np.array(near + [np.float32(gamma) * np.float32(np.sqrt(0.5))] * 4, dtype=np.float32)
    H, W = 40, 2 * 96
    D = np.zeros((H, W), np.float32)
    for y in range(H):
        cols = rng.choice(near, W // 2)
        D[y, 1::2] = cols
        if y % 2:                                       # vertical differences as well
            D[y] += rng.choice(near, W) * np.float32(0.5)
    D = np.abs(D).astype(np.float32)
    assert_exact(ctx, D, [(0.0, 1.0), (45.0, 1.4142135), (90.0, 1.0), (180.0, 2.0)], dict(gamma=gamma, L=12))
