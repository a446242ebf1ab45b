"""Autotuner of the mapping of the scan work (occ_tuning): the strip kernel's tile shape (pixels per strip, hence
lines per strip and blocks per multiprocessor; or no strip kernel), whether an all-strip call runs as one fused launch
or as separate launches, how many macro-runs the line-per-thread kernel takes (0, 1, 2), its resident blocks per
multiprocessor, and the warps per block of the one-warp-per-line kernel.

Every choice gives bit-identical M and O; the tuner times each candidate with CUDA events on sample frames of the
caller's workload, keeps the fastest, and caches it in a JSON file keyed by device and workload class (size class of
the frames, scan-length bucket, and whether the views are axial only), so that later processes reuse it.
"""
from __future__ import annotations

import json
import os

import paper_2408_14050_gb300 as occ

DEFAULT_CACHE = os.environ.get("OCC_TUNING_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "occ_tuning.json"))


def size_class(shapes) -> str:
    m = max(max(h, w) for h, w in shapes)
    return "small" if m <= 1024 else ("medium" if m <= 2048 else "large")


def scan_bucket(L: int) -> str:
    return "L<=254" if L <= 254 else ("L<=1022" if L <= 1022 else "L>1022")


def angle_class(views) -> str:
    def multiple(a, m):
        r = a % m
        return abs(r) < 1e-9 or abs(r - m) < 1e-9
    if all(multiple(a, 90.0) for a, _ in views):
        return "axial"
    return "octant" if all(multiple(a, 45.0) for a, _ in views) else "general"


def workload_key(device_name: str, shapes, views, L: int, N: int) -> str:
    return f"{device_name}|{size_class(shapes)}|{scan_bucket(L)}|{angle_class(views)}|N{N}"


# Pixels per strip of the strip kernel.  4352 holds two 2160-pixel columns or diagonals (4096x2160 frames) at five
# blocks per multiprocessor.
STRIP_SHAPES = (2048, 3072, 4096, 4352, 6144)


def candidates(max_line_bps: int):
    """Strip shapes, fused and not, with the default list-path mapping; then every list-path mapping without the strip
    kernel."""
    out = [{"line_max_runs": 2, "line_blocks_per_sm": max_line_bps, "warp_lines_per_block": 8, "strip_px": px,
            "fused": fused} for px in STRIP_SHAPES for fused in (1, 0)]
    for runs in (2, 1, 0):
        for bps in sorted({max_line_bps, max(1, max_line_bps - 1)}, reverse=True):
            for wpb in (8, 4):
                if runs == 0 and bps != max_line_bps:
                    continue      # the line kernel does not run: its grid is irrelevant
                out.append({"line_max_runs": runs, "line_blocks_per_sm": bps, "warp_lines_per_block": wpb,
                            "strip_px": 0, "fused": 0})
    return out


def tuning_name(t: dict) -> str:
    return (f"strip{t['strip_px']}{'f' if t.get('fused', 0) else ''}_runs{t['line_max_runs']}"
            f"_bps{t['line_blocks_per_sm']}_wpb{t['warp_lines_per_block']}")


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_call(run, reps: int) -> float:
    import torch
    for _ in range(2):
        run()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(reps):
        run()
    stop.record()
    torch.cuda.synchronize()
    return start.elapsed_time(stop) / reps


def autotune(ctx, Ds, views, params=None, reps: int = 5, cache_path: str | None = DEFAULT_CACHE,
             use_cache: bool = True):
    """Pick the fastest tuning for detecting `views` on the CUDA maps Ds (one map: occ_detect, several:
    occ_detect_batched), apply it to ctx and return (tuning, {candidate key: ms}).  With use_cache, a cached choice
    for the same device and workload class is applied without timing."""
    import torch
    p = params or occ.occ_default_params()
    Ms = [torch.empty((len(views), *D.shape), dtype=torch.uint8, device=D.device) for D in Ds]
    Os = [torch.empty((len(views), *D.shape), dtype=torch.int32, device=D.device) for D in Ds]

    def run():
        if len(Ds) == 1:
            occ.occ_detect(ctx, Ds[0], views, p, M=Ms[0], O=Os[0])
        else:
            occ.occ_detect_batched(ctx, Ds, views, p, Ms=Ms, Os=Os)

    run()
    if occ.occ_get_status(ctx) != occ.OCC_OK:
        raise RuntimeError("autotune: the sample frames do not run cleanly")
    L = max(s["L"] for s in occ.occ_get_stats(ctx, len(views)))
    key = workload_key(torch.cuda.get_device_name(Ds[0].device), [tuple(D.shape) for D in Ds], views, L, p.N)
    cache = load_cache(cache_path) if cache_path else {}
    if use_cache and key in cache:
        occ.occ_set_tuning(ctx, cache[key]["tuning"])
        return cache[key]["tuning"], cache[key].get("ms", {})
    _, max_bps = occ.occ_get_tuning(ctx)
    timings = {}
    best, best_ms = None, float("inf")
    for t in candidates(max_bps):
        occ.occ_set_tuning(ctx, t)
        ms = _time_call(run, reps)
        timings[tuning_name(t)] = round(ms, 4)
        if ms < best_ms:
            best, best_ms = t, ms
    occ.occ_set_tuning(ctx, best)
    if cache_path:
        cache[key] = {"tuning": best, "ms": timings}
        save_cache(cache, cache_path)
    return best, timings
