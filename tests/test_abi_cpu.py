"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports every entry point include/occ.h declares,
and its host-only helpers agree with the oracle's independent restatement of the same definitions."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2408_14050_gb300 as occ

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "occ.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(occ_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(occ.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = occ.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", occ.library_path()], capture_output=True, text=True)
    if nm.returncode == 0:
        exported = set(re.findall(r"\bT (occ_[a-z0-9_]+)$", nm.stdout, flags=re.M))
        assert set(declared_functions()) <= exported


def test_default_params():
    p = occ.occ_default_params()
    assert (p.gamma, p.zeta, p.beta, p.L, p.N) == (1.0, 2.0, 0.5, 0, 8)


def test_status_strings():
    for code in range(0, 6):
        assert isinstance(occ.occ_status_string(code), str) and occ.occ_status_string(code)
    assert occ.occ_status_string(99) == "unknown status"


def test_direction_agrees_with_oracle():
    rng = np.random.default_rng(3)
    angles = np.concatenate([np.arange(-720, 721, 0.5), rng.uniform(-1e4, 1e4, 2000), [1e-300, -1e-300, 359.9999999]])
    for a in angles:
        c1, s1 = occ.occ_direction(a)
        c2, s2 = oracle.direction(a)
        assert np.float32(c1) == c2 and np.float32(s1) == s2, a


def test_direction_exact_on_axes():
    for a, (c, s) in {0: (1, 0), 90: (0, 1), 180: (-1, 0), 270: (0, -1)}.items():
        assert occ.occ_direction(a) == (c, s)
    r = float(np.float32(math.sqrt(0.5)))
    assert occ.occ_direction(45) == (r, r)


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = occ.load().occ_create(ctypes.byref(h), 0, 1024, 1, 0)
    assert rc == occ.OCC_ERR_CUDA and not h.value


def test_invalid_arguments_rejected_before_any_device_work():
    lib = occ.load()
    h = ctypes.c_void_p()
    assert lib.occ_create(None, 0, 1024, 1, 0) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_create(ctypes.byref(h), 0, 0, 1, 0) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_create(ctypes.byref(h), 0, 1024, 0, 0) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_create(ctypes.byref(h), 0, 1024, 65, 0) == occ.OCC_ERR_INVALID_ARG
    v = (occ.occ_view * 1)()
    assert lib.occ_detect(None, None, 4, 4, 0, v, 1, None, None, None, None, None, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_get_status(None, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_get_stats(None, None, 1) == occ.OCC_ERR_INVALID_ARG
    # Median fusion and backward warp: argument checks come before any CUDA call (fake, never dereferenced,
    # 4-byte-aligned addresses).
    fake = ctypes.c_void_p(0x1000)
    maps = (ctypes.c_void_p * 2)(0x1000, 0x2000)
    assert lib.occ_fuse_median(None, 2, 4, 4, 0, fake, 0, None, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_fuse_median(maps, 0, 4, 4, 0, fake, 0, None, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_fuse_median(maps, 65, 4, 4, 0, fake, 0, None, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_fuse_median(maps, 2, 4, 4, 3, fake, 0, None, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_fuse_median(maps, 2, 4, 4, 0, ctypes.c_void_p(0x1002), 0, None, None) == occ.OCC_ERR_INVALID_ARG
    bad_maps = (ctypes.c_void_p * 2)(0x1000, None)
    assert lib.occ_fuse_median(bad_maps, 2, 4, 4, 0, fake, 0, None, None) == occ.OCC_ERR_INVALID_ARG
    imgs = (ctypes.c_void_p * 1)(0x3000)
    v[0].alpha_deg, v[0].ratio = 0.0, 1.0
    assert lib.occ_warp_views(None, 4, 4, 0, v, 1, imgs, 0, None, fake, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_warp_views(fake, 4, 4, 0, v, 0, imgs, 0, None, fake, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_warp_views(fake, 4, 4, 0, v, 1, None, 0, None, fake, None) == occ.OCC_ERR_INVALID_ARG
    assert lib.occ_warp_views(fake, 0, 4, 0, v, 1, imgs, 0, None, fake, None) == occ.OCC_ERR_INVALID_ARG
    v[0].ratio = 0.0
    assert lib.occ_warp_views(fake, 4, 4, 0, v, 1, imgs, 0, None, fake, None) == occ.OCC_ERR_INVALID_ARG
    v[0].ratio = float("nan")
    assert lib.occ_warp_views(fake, 4, 4, 0, v, 1, imgs, 0, None, fake, None) == occ.OCC_ERR_INVALID_ARG
    lib.occ_destroy(None)


def test_wrappers_reject_wrong_dtypes_and_shapes_before_calling_the_library():
    """The kernels write V*H*W elements of M and O: the bindings refuse buffers of another shape or dtype (and D of
    another dtype or layout) with ValueError before anything reaches the library.  Shapes are checked before the
    device, so CPU tensors show these errors."""
    torch = pytest.importorskip("torch")
    H, W, nv = 6, 9, 2
    views = [(0.0, 1.0), (90.0, 1.0)]
    D = torch.zeros((H, W), dtype=torch.float32)
    M = torch.zeros((nv, H, W), dtype=torch.uint8)
    O = torch.zeros((nv, H, W), dtype=torch.int32)
    st = torch.zeros(1, dtype=torch.int32)
    bad = [
        dict(D=D.double()),
        dict(D=torch.zeros((W, H), dtype=torch.float32).t()),          # unit row stride, not column stride
        dict(D=D[None]),
        dict(M=torch.zeros((H, W), dtype=torch.uint8)),                # one view's plane for two views
        dict(M=M.to(torch.int32)),
        dict(O=torch.zeros((nv, H, W - 1), dtype=torch.int32)),
        dict(O=O.to(torch.int64)),
        dict(O=torch.zeros((nv, W, H), dtype=torch.int32).transpose(1, 2)),
        dict(status=torch.zeros(1, dtype=torch.int64)),
        dict(status=torch.zeros(0, dtype=torch.int32)),
    ]
    for case in bad:
        args = dict(D=D, M=M, O=O, status=st)
        args.update(case)
        with pytest.raises(ValueError):
            occ.occ_detect_noalloc(args["D"], views, None, M=args["M"], O=args["O"], status=args["status"])
    with pytest.raises(ValueError):
        occ.occ_detect_noalloc(D, views, None, M=None, O=O)
    for case in bad[:8]:
        args = dict(D=D, M=M, O=O)
        args.update(case)
        with pytest.raises(ValueError):
            occ.occ_detect(None, args["D"], views, None, M=args["M"], O=args["O"])
    # Right shapes and dtypes, but on the CPU: refused for the device.
    with pytest.raises(ValueError, match="CUDA"):
        occ.occ_detect_noalloc(D, views, None, M=M, O=O, status=st)
    with pytest.raises(ValueError, match="CUDA"):
        occ.occ_detect(None, D, views, None, M=M, O=O)


def test_diagonal_scan_lines_stay_on_their_diagonal():
    """The strip kernel places sample g of a scan line t = round(fl(c g)) positions along the candidate's row, column
    or diagonal.  Eq. 4 rounds each coordinate after adding it: round(fl(fl(c g) + x)).  The two agree for every
    |g| <= 2047 and every coordinate below 4096 at the eight directions of a 3x3 array -- checked here exhaustively
    with binary32 arithmetic and round-half-away-from-zero, as both sides compute it."""
    f32 = np.float32
    xs = np.arange(4096, dtype=np.float32)
    g = np.arange(-2047, 2048, dtype=np.float32)

    def roundf(v):
        return np.sign(v) * np.floor(np.abs(v) + f32(0.5))

    for alpha in range(0, 360, 45):
        for comp in oracle.direction(float(alpha)):
            t = (f32(comp) * g).astype(f32)                       # fl(c g)
            direct = roundf(t)
            for x0 in range(0, 4096, 512):
                x = xs[x0:x0 + 512]
                v = (t[:, None] + x[None, :]).astype(f32)        # fl(fl(c g) + x)
                assert np.array_equal(roundf(v) - x[None, :], np.broadcast_to(direct[:, None], v.shape)), alpha
