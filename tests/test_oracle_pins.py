"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

The paper prints no worked example values (its figures are not available), so the oracle is pinned by:
hand-worked examples derived from Section 3 (tests/golden), closed forms for a rectangle on a flat background,
exact symmetries and monotonicity properties, brute force on tiny maps, library routines for the special cases
(cos/sin, sqrt, atan2) and an independent physical model (a z-buffer forward warp).  Each test names the passage
it pins and the reading of the paper it relies on.
"""
import math
import os

import numpy as np
import pytest

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def params(**kw):
    d = dict(L=0, N=8, gamma=1.0, zeta=2.0, beta=0.5)
    d.update(kw)
    return oracle.default_params(**d)


def small_scene(H=48, W=64, frame=0, sigma=0.25, n_objects=4):
    spec = scenes.SceneSpec(H=H, W=W, bg_base=(2.0, 6.0), bg_slope=(2.0, 8.0), n_objects=n_objects,
                            obj_disp=(8.0, 24.0), obj_size=(6.0, 20.0), d_max=64.0, sigma=sigma)
    return scenes.make_scene(spec, scenes.seed_of(101, frame))


# ---------------------------------------------------------------------------------------------------------------
# Hand-worked examples (Section 3, Eq. 1-6)

def _read_golden(name):
    blocks, cur, meta = {}, None, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head = line.split()
            if head[0] in ("alpha", "ratio"):
                meta[head[0]] = float(head[1])
            elif head[0] in ("map", "O"):
                cur = " ".join(head)
                blocks[cur] = []
            else:
                blocks[cur].append([float(t) for t in head])
    return meta, {k: np.array(v) for k, v in blocks.items()}


@pytest.mark.parametrize("name", ["rect_12x5_alpha0.txt", "rect_12x5_alpha180.txt"])
def test_golden_hand_worked(name):
    meta, blocks = _read_golden(name)
    D = blocks["map"].astype(np.float32)
    for key, expect in blocks.items():
        if not key.startswith("O"):
            continue
        N = int(key.split("N=")[1])
        O, M, st = oracle.detect_view(D, meta["alpha"], meta["ratio"], params(N=N))
        np.testing.assert_array_equal(O, expect.astype(np.int32), err_msg=f"{name} {key}")
        np.testing.assert_array_equal(M, (expect > 0).astype(np.uint8))


# ---------------------------------------------------------------------------------------------------------------
# cos / sin of the baseline angle (Eq. 4)

def test_direction_exact_on_axes_and_diagonals():
    r = np.float32(math.sqrt(0.5))
    expect = {0: (1, 0), 90: (0, 1), 180: (-1, 0), 270: (0, -1), 360: (1, 0), -90: (0, -1), 450: (0, 1),
              45: (r, r), 135: (-r, r), 225: (-r, -r), 315: (r, -r), -45: (r, -r)}
    for a, (c, s) in expect.items():
        cc, ss = oracle.direction(a)
        assert cc == np.float32(c) and ss == np.float32(s), a


def test_direction_matches_libm_elsewhere():
    rng = np.random.default_rng(0)
    for a in np.concatenate([rng.uniform(-720, 720, 400), np.arange(0, 360, 7.5)]):
        c, s = oracle.direction(a)
        rc, rs = np.float32(math.cos(math.radians(a))), np.float32(math.sin(math.radians(a)))
        # within one binary32 ulp of the float64 library value (different argument reduction)
        assert abs(float(c) - float(rc)) <= float(np.spacing(np.float32(abs(rc)))) + 1e-12, a
        assert abs(float(s) - float(rs)) <= float(np.spacing(np.float32(abs(rs)))) + 1e-12, a


# ---------------------------------------------------------------------------------------------------------------
# Eq. 1 and the E / A maps

@pytest.mark.parametrize("a,b", [(0.25, -0.5), (1.5, 2.0), (-3.0, 0.0), (0.0, 0.75)])
def test_edges_of_a_plane(a, b):
    H, W = 7, 9
    y, x = np.mgrid[0:H, 0:W]
    D = (10.0 + a * x + b * y).astype(np.float32)
    E, A = oracle.edges(D)
    ex = np.where(x + 1 < W, a, 0.0)       # forward difference, 0 on the last column (reading R4)
    ey = np.where(y + 1 < H, b, 0.0)
    np.testing.assert_array_equal(E, np.sqrt(ex * ex + ey * ey).astype(np.float32))
    np.testing.assert_allclose(A, np.arctan2(ey, ex), rtol=1e-6, atol=1e-7)


def test_scan_length_closed_form():
    # Eq. 3 (reading R13): L = ceil(2 (max D_r - min D_r))
    D = np.full((5, 6), 1.25, np.float32)
    D[2, 3] = 4.5
    assert oracle.scan_length(D) == 7                     # 2 * 3.25 = 6.5
    assert oracle.scan_length(D, 1.5) == 10               # 2 * (6.75 - 1.875) = 9.75
    D[0, 0] = -1.0
    assert oracle.scan_length(D) == 11                    # 2 * 5.5
    assert oracle.scan_length(np.full((3, 3), 7.0, np.float32)) == 0


# ---------------------------------------------------------------------------------------------------------------
# Special cases of the whole method

@pytest.mark.parametrize("alpha", [0.0, 45.0, 90.0, 135.0, 180.0, 225.0, 270.0, 315.0, 15.0, 203.5])
def test_constant_map_is_empty(alpha):
    # A uniform region has no edge (Section 3, first paragraph): no candidate, O = 0.
    D = np.full((16, 20), 13.7, np.float32)
    O, M, st = oracle.detect_view(D, alpha, 1.0, params())
    assert st["candidates"] == 0 and st["samples"] == 0
    assert not O.any() and not M.any()


def expected_rect_O(H, W, d0, d1, x0, x1, y0, y1, alpha, r, h):
    """Closed form of Eq. 4-6 for a rectangle of disparity d1 on a flat background d0 (integers), axial alpha.

    Derivation (readings R1, R2, R4, R9, R10): with b = r d0, f = r d1, Dr = f - b and u = W + b, the samples of
    the scan line through the candidate are background samples with u = g and foreground samples with
    u = g - Dr.  A background sample at u is hit by the foreground samples at u-1, u, u+1 (|dW| < zeta = 2 and
    V_b + beta < V_f); in sorted order they lie 1 before, 1 after and 3 after it, so N/2 = 4 keeps them all.
    Foreground samples are never behind anything.  For alpha = 0 the candidate is the background pixel left of
    the rectangle (E_x > 0) and the foreground spans g = 1..min(h, w); for alpha = 180 the candidate is the
    rightmost foreground pixel (E_x < 0, cos = -1) and the foreground spans g = 0..min(h, w-1).  90 / 270 are
    the same with rows and columns exchanged.
    """
    b, f = np.float32(r) * np.float32(d0), np.float32(r) * np.float32(d1)
    Dr = int(f - b)
    O = np.zeros((H, W), np.int32)
    w, hh = x1 - x0 + 1, y1 - y0 + 1

    def cnt(g, lo, hi):
        return sum(1 for u in (g - 1, g, g + 1) if lo <= u <= hi)

    if alpha == 0:
        for y in range(y0, y1 + 1):
            for g in range(-h, 1):
                px = x0 - 1 + g
                if px >= 0:
                    O[y, px] = cnt(g, 1 - Dr, min(h, w) - Dr)
    elif alpha == 180:
        for y in range(y0, y1 + 1):
            for g in range(-h, 0):
                px = x1 - g
                if px < W:
                    O[y, px] = cnt(g, -Dr, min(h, w - 1) - Dr)
    elif alpha == 90:
        for x in range(x0, x1 + 1):
            for g in range(-h, 1):
                py = y0 - 1 + g
                if py >= 0:
                    O[py, x] = cnt(g, 1 - Dr, min(h, hh) - Dr)
    elif alpha == 270:
        for x in range(x0, x1 + 1):
            for g in range(-h, 0):
                py = y1 - g
                if py < H:
                    O[py, x] = cnt(g, -Dr, min(h, hh - 1) - Dr)
    return O


RECT_CASES = [
    # (d0, d1, x0, x1, y0, y1, ratio, L)
    (3, 5, 20, 27, 12, 17, 1.0, 0),
    (3, 6, 18, 40, 10, 30, 1.0, 0),
    (4, 9, 16, 44, 14, 33, 1.0, 0),
    (2, 5, 15, 45, 14, 34, 2.0, 0),
    (3, 6, 18, 40, 10, 30, 1.0, 20),   # long scan window: the band reaches its full width on every side
    (2, 4, 22, 26, 20, 23, 1.0, 30),   # window longer than the rectangle
    (3, 8, 18, 40, 10, 30, 1.0, 9),    # odd L shorter than the band: h = ceil(L/2) = 5 (reading R6)
    (3, 8, 18, 40, 10, 30, 1.0, 7),    # h = 4 < Dr = 5
]


@pytest.mark.parametrize("case", RECT_CASES)
@pytest.mark.parametrize("alpha", [0, 90, 180, 270])
def test_rectangle_closed_form(case, alpha):
    d0, d1, x0, x1, y0, y1, r, L = case
    H, W = 48, 64
    D = np.full((H, W), d0, np.float32)
    D[y0:y1 + 1, x0:x1 + 1] = d1
    O, M, st = oracle.detect_view(D, alpha, r, params(L=L))
    Dr = int(np.float32(r) * np.float32(d1) - np.float32(r) * np.float32(d0))
    h = (L + 1) // 2 if L > 0 else Dr            # auto L = 2 Dr
    assert st["L"] == (L if L > 0 else 2 * Dr)
    expect = expected_rect_O(H, W, d0, d1, x0, x1, y0, y1, alpha, r, h)
    np.testing.assert_array_equal(O, expect)
    np.testing.assert_array_equal(M, (expect > 0).astype(np.uint8))


def test_rectangle_band_widths():
    # The occluded band lies on the background on the -alpha side of the object (Section 3, last paragraph of the
    # occlusion test: the pixel with the bigger disparity occludes).  Its width is Dr + zeta - 1 = Dr + 1 when the
    # scan window reaches it, and the mirror view (alpha + 180) puts it on the other side of the object.
    H, W, d0, d1 = 48, 64, 3, 7
    D = np.full((H, W), d0, np.float32)
    D[10:31, 20:41] = d1
    for alpha, side in [(0, "left"), (180, "right"), (90, "top"), (270, "bottom")]:
        _, M, _ = oracle.detect_view(D, alpha, 1.0, params(L=30))
        rows, cols = np.nonzero(M)
        if side == "left":
            assert cols.max() == 19 and cols.min() == 15
        elif side == "right":
            assert cols.min() == 41 and cols.max() == 45
        elif side == "top":
            assert rows.max() == 9 and rows.min() == 5
        else:
            assert rows.min() == 31 and rows.max() == 35


@pytest.mark.parametrize("alpha", [0, 90, 180, 270])
def test_edge_threshold_is_strict(alpha):
    # Eq. 2: a candidate needs E > gamma.  A step of exactly gamma is no edge; one just above gamma is.  The step is
    # a stripe across the whole map, so no corner pixel sees both gradients (E would be sqrt(2) times the step).
    H, W = 32, 40
    for step, expect_any in [(1.0, False), (1.25, True)]:
        D = np.full((H, W), 4.0, np.float32)
        if alpha in (0, 180):
            D[:, 12:30] = 4.0 + step
        else:
            D[10:20, :] = 4.0 + step
        _, M, st = oracle.detect_view(D, alpha, 1.0, params(gamma=1.0, L=8))
        assert (st["candidates"] > 0) == expect_any
        assert M.any() == expect_any


# ---------------------------------------------------------------------------------------------------------------
# Exact symmetries and monotonicity

@pytest.mark.parametrize("alpha", [0.0, 22.5, 45.0, 67.5, 90.0, 112.5, 135.0, 200.125, 300.5, 15.0])
@pytest.mark.parametrize("r", [1.0, 1.5])
def test_transpose_symmetry(alpha, r):
    # Eq. 1 and Eq. 4 treat x and y alike: O(D^T, 90 - alpha) = O(D, alpha)^T exactly (reading R14).
    D = small_scene(40, 56, frame=1)
    O1, _, s1 = oracle.detect_view(D, alpha, r, params())
    O2, _, s2 = oracle.detect_view(np.ascontiguousarray(D.T), 90.0 - alpha, r, params())
    np.testing.assert_array_equal(O2, O1.T)
    assert s1["samples"] == s2["samples"] and s1["candidates"] == s2["candidates"]


@pytest.mark.parametrize("alpha,r", [(0.0, 1.0), (45.0, 1.4142135), (250.0, 1.0)])
def test_monotonicity(alpha, r):
    # Eq. 5: O never decreases when zeta or N grows, never increases when beta grows; Eq. 2: fewer candidates
    # (larger gamma) never increase O.
    D = small_scene(40, 48, frame=2)

    def O(**kw):
        return oracle.detect_view(D, alpha, r, params(**kw))[0]

    for lo, hi in [(1.0, 2.0), (2.0, 3.5)]:
        assert (O(zeta=lo) <= O(zeta=hi)).all()
    for lo, hi in [(2, 4), (4, 8), (8, 16)]:
        assert (O(N=lo) <= O(N=hi)).all()
    for lo, hi in [(0.25, 0.5), (0.5, 1.5)]:
        assert (O(beta=lo) >= O(beta=hi)).all()
    for lo, hi in [(0.5, 1.0), (1.0, 2.0)]:
        assert (O(gamma=lo) >= O(gamma=hi)).all()


@pytest.mark.parametrize("alpha", [0.0, 30.0, 45.0, 90.0, 135.0, 290.0])
@pytest.mark.parametrize("t", [1.0, 7.0, -3.0])
def test_translation_invariance_on_dyadic_maps(alpha, t):
    # Adding a constant disparity t leaves every edge, L, and every difference W_p - W_q unchanged; on maps of
    # multiples of 1/4 all of these are exact in binary32, so O is unchanged exactly.
    D = np.round(small_scene(40, 48, frame=3) * 4) / 4
    D = D.astype(np.float32)
    O1, _, _ = oracle.detect_view(D, alpha, 1.0, params())
    O2, _, _ = oracle.detect_view((D + np.float32(t)).astype(np.float32), alpha, 1.0, params())
    np.testing.assert_array_equal(O1, O2)


# ---------------------------------------------------------------------------------------------------------------
# Brute force on tiny inputs

def test_sort_is_the_total_order_W_then_k():
    # The sort of Section 3 (reading R9): check the oracle's order against ranks obtained by counting.
    D = small_scene(48, 64, frame=4, sigma=0.6)
    rng = np.random.default_rng(1)
    for _ in range(40):
        cx, cy = int(rng.integers(0, 64)), int(rng.integers(0, 48))
        alpha = float(rng.choice([0.0, 45.0, 90.0, 135.0, 17.0, 250.0]))
        w, v, k, pix = oracle.scanline_sorted(D, alpha, 1.0, 40, cx, cy)
        n = len(w)
        rank = np.array([np.sum((w < w[i]) | ((w == w[i]) & (k < k[i]))) for i in range(n)])
        np.testing.assert_array_equal(rank, np.arange(n))
        assert len(set(k.tolist())) == n


def test_scanline_visits_the_nearest_pixels():
    # Eq. 4 with reading R7: sample k lies on the pixel nearest to C + g (cos alpha, sin alpha), g = k - h.
    D = small_scene(48, 64, frame=5)
    rng = np.random.default_rng(2)
    for _ in range(60):
        alpha = float(rng.uniform(0, 360))
        cx, cy = int(rng.integers(0, 64)), int(rng.integers(0, 48))
        L = int(rng.integers(1, 60))
        h = (L + 1) // 2
        w, v, k, pix = oracle.scanline_sorted(D, alpha, 1.0, L, cx, cy)
        got = dict(zip(k.tolist(), pix.tolist()))
        c, s = math.cos(math.radians(alpha)), math.sin(math.radians(alpha))
        for kk in range(2 * h + 1):
            g = kk - h
            fx, fy = cx + g * c, cy + g * s
            if min(abs(fx - math.floor(fx) - 0.5), abs(fy - math.floor(fy) - 0.5)) < 1e-3:
                continue                                   # near a half-pixel tie: binary32 rounding decides
            px, py = math.floor(fx + 0.5), math.floor(fy + 0.5)
            inside = 0 <= px < 64 and 0 <= py < 48
            assert (kk in got) == inside
            if inside:
                assert got[kk] == py * 64 + px
                assert v[list(k).index(kk)] == D[py, px]


def test_pair_test_count():
    # Eq. 5 tests each sorted sample against the neighbours d in {-N/2..N/2}\{0} that exist.
    D = small_scene(32, 40, frame=6)
    for N in (2, 8):
        _, _, st = oracle.detect_view(D, 45.0, 1.0, params(N=N))
        total = 0
        for p in oracle.candidates(D, 45.0, 1.0):
            cy, cx = divmod(int(p), 40)
            n = len(oracle.scanline_sorted(D, 45.0, 1.0, st["L"], cx, cy)[0])
            total += sum(min(N // 2, i) + min(N // 2, n - 1 - i) for i in range(n))
        assert st["pair_tests"] == total


@pytest.mark.parametrize("frame", [0, 1, 2])
def test_all_pairs_superset(frame):
    # Brute force: for alpha = 0 every hit of Eq. 5 is a pair of pixels of one row with |dW| < zeta and
    # V_p + beta < V_q; testing all pairs of the row (no candidate, window or N limit) can only find more.
    D = (np.round(small_scene(24, 40, frame=7 + frame) * 4) / 4).astype(np.float32)
    _, M, _ = oracle.detect_view(D, 0.0, 1.0, params())
    H, W = D.shape
    x = np.arange(W, dtype=np.float64)
    allp = np.zeros((H, W), bool)
    for y in range(H):
        V = D[y].astype(np.float64)
        Wv = x - V
        close = np.abs(Wv[:, None] - Wv[None, :]) < 2.0
        behind = V[:, None] + 0.5 < V[None, :]
        allp[y] = (close & behind).any(axis=1)
    assert not (M.astype(bool) & ~allp).any()


def zbuffer_mask(D, c, s, beta=0.5):
    """Physical model: forward-warp every center pixel by -D (c, s) into the peripheral view; a pixel is occluded
    if the surface that wins its target pixel (largest disparity) lies in front of it by more than beta."""
    H, W = D.shape
    y, x = np.mgrid[0:H, 0:W]
    tx = np.floor(x - c * D + 0.5).astype(int)
    ty = np.floor(y - s * D + 0.5).astype(int)
    key = {}
    for yy in range(H):
        for xx in range(W):
            t = (ty[yy, xx], tx[yy, xx])
            key[t] = max(key.get(t, -np.inf), D[yy, xx])
    M = np.zeros((H, W), bool)
    for yy in range(H):
        for xx in range(W):
            M[yy, xx] = key[(ty[yy, xx], tx[yy, xx])] > D[yy, xx] + beta
    return M


@pytest.mark.parametrize("alpha,dx,dy", [(0, -1, 0), (90, 0, -1), (180, 1, 0), (270, 0, 1)])
@pytest.mark.parametrize("d1", [6, 9])
def test_zbuffer_containment(alpha, dx, dy, d1):
    # Reading R1 against an independent physical model: the oracle's mask contains the z-buffer occlusion and
    # lies within it dilated by one pixel along -alpha (zeta - 1 = 1 extra pixel, Eq. 5).
    H, W, d0 = 40, 56, 3
    D = np.full((H, W), d0, np.float32)
    D[12:28, 20:38] = d1
    c, s = {0: (1, 0), 90: (0, 1), 180: (-1, 0), 270: (0, -1)}[alpha]
    Z = zbuffer_mask(D.astype(np.float64), c, s)
    _, M, _ = oracle.detect_view(D, alpha, 1.0, params())
    M = M.astype(bool)
    assert Z.any() and not (Z & ~M).any()
    dil = Z.copy()
    dil |= np.roll(Z, (dy, dx), axis=(0, 1))
    assert not (M & ~dil).any()


def test_nonfinite_input_is_rejected():
    D = np.ones((8, 8), np.float32)
    D[3, 4] = np.nan
    with pytest.raises(ValueError):
        oracle.detect_view(D, 0.0, 1.0, params())
    D[3, 4] = np.inf
    with pytest.raises(ValueError):
        oracle.detect_view(D, 0.0, 1.0, params())


# ---------------------------------------------------------------------------------------------------------------
# Disparity fusion (Section 4.2) and the backward warp of the registration (Section 1)

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9])
def test_median_matches_numpy(n):
    rng = np.random.default_rng(n)
    maps = [rng.normal(20, 5, (13, 17)).astype(np.float32) for _ in range(n)]
    got = oracle.median(maps)
    st = np.sort(np.stack(maps), axis=0)
    if n % 2:
        exp = st[n // 2]
    else:
        exp = ((st[n // 2 - 1] + st[n // 2]).astype(np.float32) * np.float32(0.5)).astype(np.float32)
    np.testing.assert_array_equal(got, exp)
    np.testing.assert_allclose(got, np.median(np.stack(maps), axis=0), rtol=1e-6)


def test_median_of_equal_maps_is_the_map():
    D = small_scene(20, 30, frame=9)
    np.testing.assert_array_equal(oracle.median([D] * 8), D)


def test_warp_constant_integer_disparity_is_a_shift():
    # d = 3 everywhere, alpha = 0: the center pixel x shows the peripheral pixel x - 3 exactly (fx = fy = 0).
    H, W = 10, 16
    img = np.arange(H * W, dtype=np.float32).reshape(H, W)
    D = np.full((H, W), 3.0, np.float32)
    out = oracle.warp_view(D, 0.0, 1.0, img)
    exp = np.zeros_like(img)
    exp[:, 3:] = img[:, :-3]
    np.testing.assert_array_equal(out, exp)
    out = oracle.warp_view(D, 90.0, 1.0, img)            # alpha = 90: rows shift
    exp = np.zeros_like(img)
    exp[3:, :] = img[:-3, :]
    np.testing.assert_array_equal(out, exp)
    np.testing.assert_array_equal(oracle.warp_view(np.zeros((H, W), np.float32), 33.0, 1.7, img), img)


def test_warp_half_pixel_is_the_mean_and_mask_zeroes():
    H, W = 6, 9
    rng = np.random.default_rng(4)
    img = rng.integers(0, 100, (H, W)).astype(np.float32)
    D = np.full((H, W), 0.5, np.float32)
    out = oracle.warp_view(D, 180.0, 1.0, img)           # alpha = 180: sample at x + 0.5
    exp = np.zeros_like(img)
    exp[:, :-1] = img[:, :-1] + np.float32(0.5) * (img[:, 1:] - img[:, :-1])
    np.testing.assert_array_equal(out, exp)
    M = np.zeros((H, W), np.uint8)
    M[2, 3] = 1
    out = oracle.warp_view(D, 180.0, 1.0, img, M)
    assert out[2, 3] == 0 and out[2, 2] == exp[2, 2]


def test_warp_vertical_half_pixel_is_the_mean_of_two_rows():
    # d = 0.5 at alpha = 90: the center pixel (x, y) takes the peripheral image at (x, y - 0.5), the mean of rows
    # y - 1 and y (fy = 0.5, fx = 0); at alpha = 270 it takes (x, y + 0.5), the mean of rows y and y + 1.  Rows whose
    # position leaves [0, H - 1] give 0.  Integer image values keep every operation exact.
    H, W = 7, 5
    rng = np.random.default_rng(12)
    img = rng.integers(0, 1000, (H, W)).astype(np.float32)
    D = np.full((H, W), 0.5, np.float32)
    mean = (img[:-1].astype(np.float64) + img[1:].astype(np.float64)) / 2
    exp = np.zeros((H, W))
    exp[1:] = mean
    np.testing.assert_array_equal(oracle.warp_view(D, 90.0, 1.0, img), exp)
    exp = np.zeros((H, W))
    exp[:-1] = mean
    np.testing.assert_array_equal(oracle.warp_view(D, 270.0, 1.0, img), exp)


@pytest.mark.parametrize("k", [1, 2])
def test_warp_diagonal_integer_shift(k):
    # alpha = 45 degrees with the binary32 disparity d whose product fl(fl(cos 45) * d) is exactly the integer k: the
    # center pixel (x, y) takes the peripheral pixel (x - k, y - k) exactly, on both axes at once.
    c, s = oracle.direction(45.0)
    assert c == s
    d = np.float32(k * np.sqrt(2.0))
    while np.float32(c * d) != np.float32(k):
        d = np.nextafter(d, np.float32(np.inf) if np.float32(c * d) < k else np.float32(-np.inf))
    H, W = 9, 11
    img = np.arange(H * W, dtype=np.float32).reshape(H, W) * 3 + 1
    out = oracle.warp_view(np.full((H, W), d, np.float32), 45.0, 1.0, img)
    exp = np.zeros_like(img)
    exp[k:, k:] = img[:-k, :-k]
    np.testing.assert_array_equal(out, exp)


@pytest.mark.parametrize("alpha,ratio", [(30.0, 1.0), (112.5, 1.7), (200.0, 1.0), (300.0, 2.25)])
def test_warp_of_a_linear_ramp_is_the_ramp_at_the_source_position(alpha, ratio):
    # Bilinear interpolation reproduces a linear function exactly, so warping the ramp I = a x + b y + c0 gives
    # a sx + b sy + c0 at the source position (sx, sy) = (x - cos(alpha) fl(r D), y - sin(alpha) fl(r D)) of every
    # pixel inside the image, up to one rounding per operation.  a != b, so swapped fx / fy weights or a wrong
    # neighbour row or column show; fractional D puts fx and fy anywhere in [0, 1).
    H, W = 12, 14
    a, b, c0 = 0.75, -1.25, 40.0
    yy, xx = np.mgrid[0:H, 0:W]
    img = (a * xx + b * yy + c0).astype(np.float32)
    rng = np.random.default_rng(int(alpha))
    D = rng.uniform(0.0, 3.0, (H, W)).astype(np.float32)
    cs, sn = oracle.direction(alpha)
    d = (np.float32(ratio) * D).astype(np.float32)
    sx = (xx.astype(np.float32) - (cs * d).astype(np.float32)).astype(np.float32)
    sy = (yy.astype(np.float32) - (sn * d).astype(np.float32)).astype(np.float32)
    inside = (sx >= 0) & (sx <= W - 1) & (sy >= 0) & (sy <= H - 1)
    assert 0.4 * H * W < inside.sum() < H * W
    frac_y = sy[inside] - np.floor(sy[inside])
    assert (frac_y > 0.1).sum() > 20
    out = oracle.warp_view(D, alpha, ratio, img)
    exp = np.where(inside, a * sx.astype(np.float64) + b * sy.astype(np.float64) + c0, 0.0)
    np.testing.assert_allclose(out, exp, rtol=0, atol=1e-4)
    assert (out[~inside] == 0).all()


def test_median_signed_zero_and_nonfinite():
    a = np.full((2, 3), -0.0, np.float32)
    b = np.full((2, 3), 0.0, np.float32)
    for maps in ([a, b, a], [a, a], [b, a]):
        got = oracle.median(maps)
        assert not np.signbit(got).any()
    c = b.copy()
    c[1, 2] = np.inf
    with pytest.raises(ValueError):
        oracle.median([b, c, b])


def test_tile_helpers_partition_the_work():
    """The proposal helpers: all tiles proposed is the plain method; the tiles' separate runs add up to it (Eq. 6 is
    a sum over scan lines); labels are 1 exactly on the tiles whose own run finds an occlusion."""
    D = small_scene(70, 100, frame=11)
    a, r = 0.0, 1.0
    O, M, _ = oracle.detect_view(D, a, r)
    ty, tx = 3, 4
    O_all, M_all = oracle.detect_view_proposed(D, a, r, None, np.ones((ty, tx), np.uint8))
    np.testing.assert_array_equal(O_all, O)
    total = np.zeros_like(O)
    labels = oracle.tile_labels(D, a, r)
    for i in range(ty):
        for j in range(tx):
            one = np.zeros((ty, tx), np.uint8)
            one[i, j] = 1
            Ot, _ = oracle.detect_view_proposed(D, a, r, None, one)
            total += Ot
            assert labels[i, j] == (1 if Ot.any() else 0)
    np.testing.assert_array_equal(total, O)
    assert oracle.tile_mask(70, 100, np.ones((3, 4))).shape == (70, 100)
    O_none, M_none = oracle.detect_view_proposed(D, a, r, None, np.zeros((ty, tx), np.uint8))
    assert not O_none.any() and not M_none.any()
