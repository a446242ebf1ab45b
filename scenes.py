"""Seeded synthetic disparity scenes: the input generator shared by the tests, the oracle runs and bench.py.

This module only makes inputs.  It holds none of the occlusion method's arithmetic: it draws piecewise-planar
disparity maps (a sloped background plane plus slanted rectangles and ellipses painted far-to-near, Gaussian
noise, optional salt outliers) that stand in for the paper's workloads (SceneFlow, the synthetic hyperspectral
database and the real CAMSI recording of Section 4, none of which are available here).

Randomness is counter-based: every draw is splitmix64(seed + counter * golden_gamma), so a scene depends only on
(config id, frame id) and on nothing else (no global RNG state, no library RNG whose stream could change between
numpy versions).  Gaussians use the Box-Muller transform in float64; the map is rounded to float32 once, at the end.
The float64 log/cos of different libms can differ in the last bit, so the same seed may give maps that differ in a
few low-order bits between machines; every parity check generates its input on the machine it runs on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array; wraps modulo 2**64."""
    z = (z ^ (z >> np.uint64(30))) * _MIX1
    z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def seed_of(config_id: int, frame: int) -> int:
    """Stream seed for (config id, frame id)."""
    x = np.array([(int(config_id) << 32) | (int(frame) & 0xFFFFFFFF)], dtype=np.uint64)
    return int(_mix(x + _GOLDEN)[0])


class CounterRng:
    """splitmix64 in counter mode: draw i of stream `key` is mix(seed ^ key*C + (i+1)*golden)."""

    def __init__(self, seed: int, key: int = 0):
        base = np.array([seed], dtype=np.uint64) ^ (np.array([key], dtype=np.uint64) * _MIX2)
        self._base = base
        self._next = 0

    def bits(self, n: int, offset: int | None = None) -> np.ndarray:
        start = self._next if offset is None else offset
        idx = np.arange(start + 1, start + 1 + n, dtype=np.uint64)
        if offset is None:
            self._next += n
        return _mix(self._base + idx * _GOLDEN)

    def uniform(self, n: int, offset: int | None = None) -> np.ndarray:
        """n float64 uniforms in (0, 1)."""
        b = self.bits(n, offset)
        return ((b >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)

    def normal(self, n: int, offset: int | None = None) -> np.ndarray:
        """n standard normals by Box-Muller (one pair of uniforms per draw, cosine branch)."""
        start = self._next if offset is None else offset
        u = self.uniform(2 * n, offset=2 * start)
        if offset is None:
            self._next += n
        u1, u2 = u[0::2], u[1::2]
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def scalar(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * float(self.uniform(1)[0])


@dataclass(frozen=True)
class SceneSpec:
    """Statistics of one synthetic piecewise-planar scene."""
    H: int
    W: int
    bg_base: tuple = (0.0, 8.0)          # background disparity at its lowest corner
    bg_slope: tuple = (2.0, 8.0)         # total background change across the image, px
    n_objects: int = 20
    obj_disp: tuple = (8.0, 64.0)        # base disparity of an object
    obj_size: tuple = (0.05, 0.25)       # object width/height; fractions of H if <= 1, else pixels
    obj_slope: float = 2.0               # max disparity change across one object, px
    d_max: float = 64.0                  # objects are clamped to [0, d_max] before noise
    sigma: float = 0.25                  # Gaussian noise std, px
    salt: float = 0.0                    # probability that a pixel is replaced by U[0, d_max]
    quantum: float = 0.0                 # if > 0: round the noise-free map to multiples of this (dyadic maps)


def make_scene(spec: SceneSpec, seed: int) -> np.ndarray:
    """Draw one float32 [H][W] disparity map (row-major, x = column, y = row pointing down)."""
    H, W = spec.H, spec.W
    rng = CounterRng(seed, key=1)
    ys = np.arange(H, dtype=np.float64)[:, None]
    xs = np.arange(W, dtype=np.float64)[None, :]

    # Background plane d0 + |gx|*fx + |gy|*fy, with fx, fy running 0->1 or 1->0 by a random sign.
    d0 = rng.scalar(*spec.bg_base)
    total = rng.scalar(*spec.bg_slope)
    split = rng.scalar(0.0, 1.0)
    gx, gy = total * split, total * (1.0 - split)
    fx = xs / W if rng.scalar(0, 1) < 0.5 else 1.0 - xs / W
    fy = ys / H if rng.scalar(0, 1) < 0.5 else 1.0 - ys / H
    d = d0 + gx * fx + gy * fy
    d = np.broadcast_to(d, (H, W)).copy()

    # Objects: drawn first, painted in ascending base disparity (near objects last, so the map is z-consistent).
    objs = []
    for _ in range(spec.n_objects):
        lo, hi = spec.obj_size
        if hi <= 1.0:
            lo, hi = lo * H, hi * H
        ow, oh = rng.scalar(lo, hi), rng.scalar(lo, hi)
        ocx, ocy = rng.scalar(0, W), rng.scalar(0, H)
        base = rng.scalar(*spec.obj_disp)
        t = rng.scalar(0.0, spec.obj_slope)
        f = rng.scalar(0.0, 1.0)
        sx = t * f * (1 if rng.scalar(0, 1) < 0.5 else -1)
        sy = t * (1 - f) * (1 if rng.scalar(0, 1) < 0.5 else -1)
        ellipse = rng.scalar(0, 1) < 0.5
        objs.append((base, ow, oh, ocx, ocy, sx, sy, ellipse))
    objs.sort(key=lambda o: o[0])
    for base, ow, oh, ocx, ocy, sx, sy, ellipse in objs:
        x0, x1 = max(0, int(math.floor(ocx - ow / 2))), min(W, int(math.ceil(ocx + ow / 2)) + 1)
        y0, y1 = max(0, int(math.floor(ocy - oh / 2))), min(H, int(math.ceil(ocy + oh / 2)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        bx = xs[:, x0:x1]
        by = ys[y0:y1, :]
        rx, ry = (bx - ocx) / (ow / 2), (by - ocy) / (oh / 2)
        if ellipse:
            inside = rx * rx + ry * ry <= 1.0
        else:
            inside = (np.abs(rx) <= 1.0) & (np.abs(ry) <= 1.0)
        plane = base + sx * rx / 2 + sy * ry / 2
        plane = np.clip(plane, 0.0, spec.d_max)
        region = d[y0:y1, x0:x1]
        region[inside] = np.broadcast_to(plane, inside.shape)[inside]

    if spec.quantum > 0:
        d = np.round(d / spec.quantum) * spec.quantum
    if spec.sigma > 0:
        d = d + spec.sigma * CounterRng(seed, key=2).normal(H * W).reshape(H, W)
    if spec.salt > 0:
        r = CounterRng(seed, key=3).uniform(2 * H * W).reshape(H, W, 2)
        hit = r[..., 0] < spec.salt
        d = np.where(hit, r[..., 1] * spec.d_max, d)
    return np.ascontiguousarray(d.astype(np.float32))


# ---------------------------------------------------------------------------------------------------------------
# Views of a camera array: baseline direction alpha (degrees, from +x toward +y, y pointing down) and baseline
# ratio r (this camera's baseline over the axial neighbour's).

def views_3x3():
    """The eight peripheral cameras of a 3x3 array: axial at ratio 1, diagonal at ratio sqrt(2)."""
    out = []
    for k in range(8):
        a = 45.0 * k
        out.append((a, 1.0 if k % 2 == 0 else float(np.float32(math.sqrt(2.0)))))
    return out


def views_5x5_ring():
    """24 views at 15 degree steps on the square rings of a 5x5 array: r = ring / max(|cos a|, |sin a|)."""
    out = []
    for k in range(24):
        a = 15.0 * k
        ring = 1.0 if k % 2 == 0 else 2.0
        rad = math.radians(a)
        out.append((a, float(np.float32(ring / max(abs(math.cos(rad)), abs(math.sin(rad)))))))
    return out


# ---------------------------------------------------------------------------------------------------------------
# The workloads.  Each returns a list of (name, D) frames and the view table.

SPEC_STEREO = SceneSpec(H=192, W=256, bg_base=(2.0, 6.0), bg_slope=(2.0, 8.0), n_objects=6,
                        obj_disp=(10.0, 40.0), obj_size=(12.0, 60.0), d_max=64.0, sigma=0.25)


def spec_array(H: int, W: int) -> SceneSpec:
    return SceneSpec(H=H, W=W, bg_base=(0.0, 8.0), bg_slope=(2.0, 8.0), n_objects=20, obj_disp=(8.0, 64.0),
                     obj_size=(0.05, 0.25), d_max=64.0, sigma=0.25)


def spec_stress(H: int = 2160, W: int = 4096) -> SceneSpec:
    return SceneSpec(H=H, W=W, bg_base=(0.0, 16.0), bg_slope=(4.0, 16.0), n_objects=20, obj_disp=(16.0, 128.0),
                     obj_size=(0.05, 0.25), d_max=128.0, sigma=0.5, salt=0.02)


MIXED_SIZES = [(480, 640), (720, 1280), (1080, 1920), (2160, 4096)]


@dataclass
class Workload:
    name: str
    frames: list = field(default_factory=list)     # list of float32 [H][W] arrays
    views: list = field(default_factory=list)      # list of (alpha_deg, ratio)

    @property
    def pixel_views(self) -> int:
        return sum(int(f.size) for f in self.frames) * len(self.views)


def stereo_pair(frame: int = 0) -> Workload:
    """One 256x192 map, horizontal stereo pair (alpha = 0, ratio 1)."""
    return Workload("stereo_256x192_1view", [make_scene(SPEC_STEREO, seed_of(1, frame))], [(0.0, 1.0)])


def array_3x3(frame: int = 0, H: int = 1080, W: int = 1920) -> Workload:
    """One center-view map of a 3x3 array, eight peripheral views."""
    return Workload(f"array3x3_{W}x{H}_8views", [make_scene(spec_array(H, W), seed_of(2, frame))], views_3x3())


def _array_scene(H: int, W: int, seed: int) -> np.ndarray:
    return make_scene(spec_array(H, W), seed)


def mixed_batch(n_frames: int = 64, sizes=None, config: int = 3, workers: int = 0) -> Workload:
    """n_frames maps of uneven resolution (equal counts of each size, seeded shuffle), eight views each.  Another
    `config` draws other frames of the same recipe (e.g. held-out frames for calibration).  workers > 1 draws them
    in a pool of spawned processes (same frames)."""
    sizes = sizes or MIXED_SIZES
    order = [sizes[i % len(sizes)] for i in range(n_frames)]
    perm = np.argsort(CounterRng(seed_of(config, 1 << 20), key=4).uniform(n_frames), kind="stable")
    jobs = [(*order[i], seed_of(config, f)) for f, i in enumerate(perm)]
    if workers > 1 and n_frames > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            frames = pool.starmap(_array_scene, jobs, chunksize=1)
    else:
        frames = [_array_scene(*j) for j in jobs]
    return Workload(f"mixed_{n_frames}frames_8views", frames, views_3x3())


def stress_5x5(frame: int = 0, H: int = 2160, W: int = 4096) -> Workload:
    """4096x2160 map with salt outliers, 24 views on the rings of a 5x5 array."""
    return Workload(f"array5x5_{W}x{H}_24views", [make_scene(spec_stress(H, W), seed_of(4, frame))],
                    views_5x5_ring())


def stereo_maps(D: np.ndarray, n: int, seed: int, sigma: float = 0.25, salt: float = 0.01,
                d_max: float = 64.0) -> list:
    """n per-camera estimates of the center map D, as the stereo matches of n peripheral cameras would give them
    before fusion: D plus independent Gaussian noise (sigma px) and, with probability `salt` per pixel, a wrong match
    drawn from U[0, d_max]."""
    H, W = D.shape
    out = []
    for k in range(n):
        e = D.astype(np.float64) + sigma * CounterRng(seed, key=16 + 2 * k).normal(H * W).reshape(H, W)
        if salt > 0:
            r = CounterRng(seed, key=17 + 2 * k).uniform(2 * H * W).reshape(H, W, 2)
            e = np.where(r[..., 0] < salt, r[..., 1] * d_max, e)
        out.append(np.ascontiguousarray(e.astype(np.float32)))
    return out


def peripheral_images(H: int, W: int, n: int, seed: int) -> list:
    """n smooth-plus-texture float32 images standing in for the peripheral cameras' spectral images (values in
    [0, 1]): a low-frequency pattern plus uniform texture."""
    ys = np.arange(H, dtype=np.float64)[:, None]
    xs = np.arange(W, dtype=np.float64)[None, :]
    out = []
    for k in range(n):
        rng = CounterRng(seed, key=64 + k)
        fx, fy, ph = rng.scalar(0.005, 0.05), rng.scalar(0.005, 0.05), rng.scalar(0.0, 6.28)
        base = 0.5 + 0.3 * np.sin(fx * xs + ph) * np.cos(fy * ys)
        tex = 0.2 * rng.uniform(H * W).reshape(H, W)
        out.append(np.ascontiguousarray((base + tex).astype(np.float32)))
    return out


# ---------------------------------------------------------------------------------------------------------------
# Initial parameters of the learned tile proposer (seeded; the network's own arithmetic lives elsewhere).
# Layout of the flat float32 parameter vector: for each 3x3 convolution (c_in -> c_out) the weights
# [c_out][9][c_in] (tap = (dy + 1) * 3 + (dx + 1)) then the bias [c_out]; then the view encoding's weights [16][3]
# and bias [16], then the output bias [1].

NET_LAYERS = [(8, 16), (16, 16), (16, 32), (32, 16)]
NET_FEATURES = 16
NET_ENC = 3


def net_param_count() -> int:
    n = sum(co * 9 * ci + co for ci, co in NET_LAYERS)
    return n + NET_FEATURES * NET_ENC + NET_FEATURES + 1


def net_init(seed: int) -> np.ndarray:
    """He-normal convolution weights (fan-in = 9 x the input channels that carry data: 1 for the first layer, whose
    input has the disparity in channel 0 and zeros elsewhere), zero biases, N(0, 0.5) view-encoding weights."""
    rng = CounterRng(seed, key=200)
    out = []
    off = 0
    for li, (ci, co) in enumerate(NET_LAYERS):
        fan = 9 * (1 if li == 0 else ci)
        w = rng.normal(co * 9 * ci, offset=off) * np.sqrt(2.0 / fan)
        off += co * 9 * ci
        if li == 0:
            w = w.reshape(co, 9, ci)
            w[:, :, 1:] = 0.0
            w = w.reshape(-1)
        out += [w, np.zeros(co)]
    out += [rng.normal(NET_FEATURES * NET_ENC, offset=off) * 0.5, np.zeros(NET_FEATURES), np.zeros(1)]
    return np.concatenate(out).astype(np.float32)


def proposer_spec(frame: int, H: int, W: int, seed: int) -> SceneSpec:
    """Scene statistics of one training frame of the learned tile proposer: the 3x3-array recipe with the noise
    level drawn from [0, 0.3] px and 4 to 20 objects, so that both noisy and clean maps are seen."""
    rng = CounterRng(seed_of(seed, frame), key=300)
    return SceneSpec(H=H, W=W, bg_base=(0.0, 8.0), bg_slope=(2.0, 8.0), n_objects=int(rng.scalar(4, 21)),
                     obj_disp=(8.0, 64.0), obj_size=(0.05, 0.35), d_max=64.0, sigma=rng.scalar(0.0, 0.3))


def proposer_frame(frame: int, H: int, W: int, seed: int) -> np.ndarray:
    return make_scene(proposer_spec(frame, H, W, seed), seed_of(seed + 1, frame))


def proposer_frames(n: int, H: int, W: int, seed: int, first: int = 0, workers: int = 0) -> np.ndarray:
    """Frames first .. first + n - 1 of the proposer's training stream as one float32 array [n][H][W].  workers > 1
    draws them in a pool of spawned processes (safe after CUDA has been initialised)."""
    idx = list(range(first, first + n))
    if workers > 1 and n > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            out = pool.starmap(proposer_frame, [(i, H, W, seed) for i in idx], chunksize=max(1, n // (4 * workers)))
    else:
        out = [proposer_frame(i, H, W, seed) for i in idx]
    return np.stack(out)
