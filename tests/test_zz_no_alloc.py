"""occ_detect_noalloc, the entry point for callers that cannot allocate device memory (code inside an allocator or
memory-pool callback, a real-time loop that must not block on the allocator, a framework that only hands out its
own tensors): its results must equal occ_detect's, call after call, although every call reuses the same scratch
array built into the library.

Kept in a file of its own, collected last, so that a failure here cannot hide the other tests' results.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2408_14050_gb300 as occ
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(D, views, p):
    """M and O of the context-based entry point on the same input."""
    H, W = D.shape
    with occ.occ_create(0, max_pixels=H * W, max_views=len(views)) as ctx:
        M, O = occ.occ_detect(ctx, D, views, p)
        assert occ.occ_get_status(ctx) == occ.OCC_OK
        return M.clone(), O.clone()


def test_noalloc_matches_occ_detect_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    p = occ.occ_default_params()
    # Two different inputs in a row: the second call must not see anything the first left in the shared scratch.
    cases = [(scenes.array_3x3(frame=5, H=540, W=960).frames[0], scenes.views_3x3()),
             (scenes.stereo_pair(frame=3).frames[0], [(0.0, 1.0), (135.0, 1.4142135), (250.0, 2.0)])]
    for D_np, views in cases:
        D = torch.from_numpy(D_np).cuda()
        H, W = D_np.shape
        M = torch.empty((len(views), H, W), dtype=torch.uint8, device="cuda")
        O = torch.empty((len(views), H, W), dtype=torch.int32, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = occ.occ_detect_noalloc(D, views, p, M=M, O=O, status=st)
        assert rc == occ.OCC_OK, occ.occ_status_string(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        M_ref, O_ref = _reference(D, views, p)
        assert torch.equal(O, O_ref), "O differs from occ_detect"
        assert torch.equal(M, M_ref), "M differs from occ_detect"
        assert int(O.sum()) > 0
        # And against the oracle, bit for bit (Eq. 6: O and M).
        O_ora, M_ora, _ = oracle.detect(D_np, views, oracle.default_params())
        np.testing.assert_array_equal(O.cpu().numpy(), O_ora)
        np.testing.assert_array_equal(M.cpu().numpy(), M_ora)


def test_noalloc_at_its_largest_size():
    """H * W * views exactly at the limit (2048 x 1024, 8 views): the candidate lists fill the whole array, and the
    list of scan lines handed to the merge kernel is left no more room than the call's candidates leave free, so
    lines of two macro-runs near its end must go to the warp kernel instead.  Results equal occ_detect's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    p = occ.occ_default_params()
    views = scenes.views_3x3()
    H, W = 1024, 2048
    assert H * W * len(views) == occ.OCC_NOALLOC_MAX_PIXEL_VIEWS
    D_np = scenes.array_3x3(frame=21, H=H, W=W).frames[0]
    D = torch.from_numpy(D_np).cuda()
    M = torch.empty((len(views), H, W), dtype=torch.uint8, device="cuda")
    O = torch.empty((len(views), H, W), dtype=torch.int32, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        rc = occ.occ_detect_noalloc(D, views, p, M=M, O=O, status=st)
        assert rc == occ.OCC_OK, occ.occ_status_string(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        M_ref, O_ref = _reference(D, views, p)
        assert torch.equal(O, O_ref), "O differs from occ_detect"
        assert torch.equal(M, M_ref), "M differs from occ_detect"
    # A window of the alpha = 0 view against the oracle: at alpha = 0 a scan line stays in its row and reaches h
    # pixels to each side, so the candidates of the window's rows within h columns of it give its whole O.
    h = (oracle.scan_length(D_np, 1.0) + 1) // 2
    x0, y0, x1, y1 = 1000, 500, 1064, 532
    O_w, _, _ = oracle.detect_view(D_np, 0.0, 1.0, oracle.default_params(), region=(x0 - h, y0, x1 + h, y1))
    got = O[0, y0:y1, x0:x1].cpu().numpy()
    np.testing.assert_array_equal(got, O_w[y0:y1, x0:x1])


def test_noalloc_reports_nonfinite_input_then_recovers():
    """A NaN in D sets bit 0 of the status the call writes; the next call on good input starts from a cleared
    status word and gives occ_detect's results again."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    p = occ.occ_default_params()
    views = [(0.0, 1.0), (90.0, 1.0)]
    D_np = scenes.stereo_pair(frame=7).frames[0]
    bad = D_np.copy()
    bad[50, 60] = np.nan
    H, W = D_np.shape
    M = torch.empty((len(views), H, W), dtype=torch.uint8, device="cuda")
    O = torch.empty((len(views), H, W), dtype=torch.int32, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = occ.occ_detect_noalloc(torch.from_numpy(bad).cuda(), views, p, M=M, O=O, status=st)
    assert rc == occ.OCC_OK
    torch.cuda.synchronize()
    assert int(st.item()) & 1, "non-finite input not reported"
    D = torch.from_numpy(D_np).cuda()
    rc = occ.occ_detect_noalloc(D, views, p, M=M, O=O, status=st)
    assert rc == occ.OCC_OK
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    M_ref, O_ref = _reference(D, views, p)
    assert torch.equal(O, O_ref) and torch.equal(M, M_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = occ.load()
    views = (occ.occ_view * 8)()
    for i in range(8):
        views[i].alpha_deg, views[i].ratio = 45.0 * i, 1.0
    H, W = 2160, 4096   # 8 views of this map need 70.8 M entries > 16.8 M
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    rc = lib.occ_detect_noalloc(dummy, H, W, W, views, 8, None, dummy, dummy, None, None)
    assert rc == occ.OCC_ERR_CAPACITY
    assert H * W * 8 > occ.OCC_NOALLOC_MAX_PIXEL_VIEWS
