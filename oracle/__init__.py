"""CPU oracle of the fast edge-aware occlusion detection (Sippel, Seiler, Kaup, ICIP 2024, Section 3).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may import
this package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in occ_oracle.c (plain C, binary32, no FMA contraction, single thread); this module
compiles it with gcc on first use and wraps it with ctypes.  Every function cites the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "occ_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libocc_oracle.so")
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE"]

OK, ERR_ARG, ERR_NONFINITE, ERR_NOMEM = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    """gamma (Eq. 2), zeta and beta (Eq. 5), L (Eq. 3; <= 0 = automatic), N (Eq. 5)."""
    _fields_ = [("gamma", ctypes.c_float), ("zeta", ctypes.c_float), ("beta", ctypes.c_float),
                ("L", ctypes.c_int32), ("N", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("samples", ctypes.c_int64), ("pair_tests", ctypes.c_int64),
                ("hits", ctypes.c_int64), ("L", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def default_params(L: int = 0, N: int = 8, gamma: float = 1.0, zeta: float = 2.0, beta: float = 0.5) -> Params:
    """The paper's thresholds gamma=1.0, zeta=2.0, beta=0.5 (Section 4.1); N=8 (the paper gives none)."""
    return Params(gamma, zeta, beta, L, N)


def build(force: bool = False) -> str:
    """Compile occ_oracle.c into oracle/_build/libocc_oracle.so (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            f32p = ctypes.POINTER(ctypes.c_float)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            L.ora_direction.argtypes = [ctypes.c_double, f32p, f32p]
            L.ora_direction.restype = None
            L.ora_edges.argtypes = [f32p, ctypes.c_int32, ctypes.c_int32, f32p, f32p]
            L.ora_edges.restype = ctypes.c_int
            L.ora_scan_length.argtypes = [f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_float]
            L.ora_scan_length.restype = ctypes.c_int32
            L.ora_detect_view_region.argtypes = [f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_float, ctypes.POINTER(Params), ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i32p, u8p,
                                                 ctypes.POINTER(Stats)]
            L.ora_detect_view_region.restype = ctypes.c_int
            L.ora_detect_view_masked.argtypes = [f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_float, ctypes.POINTER(Params), ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, u8p, i32p, u8p,
                                                 ctypes.POINTER(Stats)]
            L.ora_detect_view_masked.restype = ctypes.c_int
            L.ora_candidates.argtypes = [f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_float,
                                         ctypes.c_float, i64p, ctypes.c_int64]
            L.ora_candidates.restype = ctypes.c_int64
            L.ora_scanline_sorted.argtypes = [f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_float, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              f32p, f32p, i32p, i64p, ctypes.c_int32]
            L.ora_scanline_sorted.restype = ctypes.c_int32
            L.ora_median.argtypes = [ctypes.POINTER(f32p), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, f32p]
            L.ora_median.restype = ctypes.c_int
            L.ora_warp_view.argtypes = [f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_float, f32p,
                                        u8p, f32p]
            L.ora_warp_view.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _map(D) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.float32)
    if D.ndim != 2:
        raise ValueError("D must be [H][W]")
    return D


def direction(alpha_deg: float):
    """(cos alpha, sin alpha) rounded to binary32 after reduction to [0, 45] degrees (Eq. 4's cos/sin)."""
    c, s = ctypes.c_float(), ctypes.c_float()
    lib().ora_direction(float(alpha_deg), ctypes.byref(c), ctypes.byref(s))
    return np.float32(c.value), np.float32(s.value)


def edges(D):
    """E and A of Section 3 (Eq. 1 and the magnitude / angle maps), r = 1.  Returns (E, A) float32 [H][W]."""
    D = _map(D)
    H, W = D.shape
    E = np.empty_like(D)
    A = np.empty_like(D)
    rc = lib().ora_edges(_ptr(D, ctypes.c_float), H, W, _ptr(E, ctypes.c_float), _ptr(A, ctypes.c_float))
    if rc != OK:
        raise ValueError(f"oracle edges failed: {rc}")
    return E, A


def scan_length(D, ratio: float = 1.0) -> int:
    """Eq. 3 on D_r = fl(r*D)."""
    D = _map(D)
    return int(lib().ora_scan_length(_ptr(D, ctypes.c_float), D.shape[0], D.shape[1], float(ratio)))


def detect_view(D, alpha_deg: float, ratio: float = 1.0, params: Params | None = None, region=None):
    """The method of Section 3 for one view.  Returns (O int32 [H][W], M uint8 [H][W], stats dict).

    region = (cx0, cy0, cx1, cy1) restricts the candidates processed (O then holds only their contributions)."""
    D = _map(D)
    H, W = D.shape
    p = params or default_params()
    O = np.empty((H, W), dtype=np.int32)
    M = np.empty((H, W), dtype=np.uint8)
    st = Stats()
    cx0, cy0, cx1, cy1 = region if region is not None else (0, 0, W, H)
    rc = lib().ora_detect_view_region(_ptr(D, ctypes.c_float), H, W, float(alpha_deg), float(ratio),
                                      ctypes.byref(p), cx0, cy0, cx1, cy1, _ptr(O, ctypes.c_int32),
                                      _ptr(M, ctypes.c_uint8), ctypes.byref(st))
    if rc != OK:
        raise ValueError(f"oracle detect failed: {rc}")
    return O, M, st.as_dict()


def detect_view_masked(D, alpha_deg: float, ratio: float, params: Params | None, cand_mask):
    """detect_view restricted to the candidates where cand_mask (uint8 [H][W]) is non-zero: O then holds exactly
    their contributions.  Returns (O, stats)."""
    D = _map(D)
    H, W = D.shape
    p = params or default_params()
    mask = np.ascontiguousarray(cand_mask, dtype=np.uint8)
    if mask.shape != (H, W):
        raise ValueError("mask shape")
    O = np.empty((H, W), dtype=np.int32)
    st = Stats()
    rc = lib().ora_detect_view_masked(_ptr(D, ctypes.c_float), H, W, float(alpha_deg), float(ratio),
                                      ctypes.byref(p), 0, 0, W, H, _ptr(mask, ctypes.c_uint8),
                                      _ptr(O, ctypes.c_int32), None, ctypes.byref(st))
    if rc != OK:
        raise ValueError(f"oracle detect failed: {rc}")
    return O, st.as_dict()


def detect(D, views, params: Params | None = None):
    """All views of one frame: O int32 [V][H][W], M uint8 [V][H][W], list of per-view stats."""
    D = _map(D)
    outs = [detect_view(D, a, r, params) for (a, r) in views]
    return (np.stack([o[0] for o in outs]), np.stack([o[1] for o in outs]), [o[2] for o in outs])


def candidates(D, alpha_deg: float, ratio: float = 1.0, gamma: float = 1.0) -> np.ndarray:
    """Eq. 2's candidate list, row-major, as flat pixel indices y*W + x."""
    D = _map(D)
    H, W = D.shape
    cap = H * W
    out = np.empty(cap, dtype=np.int64)
    n = lib().ora_candidates(_ptr(D, ctypes.c_float), H, W, float(alpha_deg), float(ratio), float(gamma),
                             _ptr(out, ctypes.c_int64), cap)
    return out[:n].copy()


def scanline_sorted(D, alpha_deg: float, ratio: float, L: int, cx: int, cy: int):
    """Sorted samples (W, V, k, pixel) of the scan line through (cx, cy) (Eq. 4, the warp and the sort)."""
    D = _map(D)
    H, W = D.shape
    cap = L + 2
    w = np.empty(cap, np.float32)
    v = np.empty(cap, np.float32)
    k = np.empty(cap, np.int32)
    pix = np.empty(cap, np.int64)
    n = lib().ora_scanline_sorted(_ptr(D, ctypes.c_float), H, W, float(alpha_deg), float(ratio), int(L), int(cx),
                                  int(cy), _ptr(w, ctypes.c_float), _ptr(v, ctypes.c_float),
                                  _ptr(k, ctypes.c_int32), _ptr(pix, ctypes.c_int64), cap)
    if n < 0:
        raise ValueError("scan line longer than expected")
    return w[:n], v[:n], k[:n], pix[:n]


def median(maps):
    """Pixel-wise median of n maps [H][W] (Section 4.2); even n: fl(a + b) * 0.5 of the two middle values."""
    maps = [_map(m) for m in maps]
    H, W = maps[0].shape
    arr = (ctypes.POINTER(ctypes.c_float) * len(maps))(*[_ptr(m, ctypes.c_float) for m in maps])
    out = np.empty((H, W), np.float32)
    rc = lib().ora_median(arr, len(maps), H, W, _ptr(out, ctypes.c_float))
    if rc != OK:
        raise ValueError(f"oracle median failed: {rc}")
    return out


def warp_view(D, alpha_deg: float, ratio: float, img, M=None):
    """Backward warp of a peripheral image into the center view, bilinear, occluded / outside pixels 0 (Section 1)."""
    D = _map(D)
    img = _map(img)
    H, W = D.shape
    out = np.empty((H, W), np.float32)
    Mp = None
    if M is not None:
        M = np.ascontiguousarray(M, dtype=np.uint8)
        Mp = _ptr(M, ctypes.c_uint8)
    rc = lib().ora_warp_view(_ptr(D, ctypes.c_float), H, W, float(alpha_deg), float(ratio), _ptr(img, ctypes.c_float),
                             Mp, _ptr(out, ctypes.c_float))
    if rc != OK:
        raise ValueError(f"oracle warp failed: {rc}")
    return out


def tile_mask(H: int, W: int, table, T: int = 32) -> np.ndarray:
    """uint8 [H][W] pixel mask that is 1 on the tiles where table [ceil(H/T)][ceil(W/T)] is non-zero."""
    table = np.asarray(table)
    return np.kron(table != 0, np.ones((T, T), dtype=bool))[:H, :W].astype(np.uint8)


def detect_view_proposed(D, alpha_deg: float, ratio: float, params: Params | None, proposal, T: int = 32):
    """The method with the candidate list of Eq. 2 restricted to the tiles where proposal [tiles_y][tiles_x] is
    non-zero (a candidate belongs to the tile of its pixel).  Returns (O, M)."""
    D = _map(D)
    O, _ = detect_view_masked(D, alpha_deg, ratio, params, tile_mask(*D.shape, proposal, T))
    return O, (O > 0).astype(np.uint8)


def tile_labels(D, alpha_deg: float, ratio: float, params: Params | None = None, T: int = 32) -> np.ndarray:
    """uint8 [tiles_y][tiles_x]: 1 where the scan lines of the tile's candidates (Eq. 2, Eq. 4) add a non-zero count
    to O (Eq. 5-6), each tile run on its own."""
    D = _map(D)
    H, W = D.shape
    ty, tx = (H + T - 1) // T, (W + T - 1) // T
    out = np.zeros((ty, tx), np.uint8)
    for i in range(ty):
        for j in range(tx):
            one = np.zeros((ty, tx), np.uint8)
            one[i, j] = 1
            O, _ = detect_view_masked(D, alpha_deg, ratio, params, tile_mask(H, W, one, T))
            out[i, j] = 1 if O.any() else 0
    return out
