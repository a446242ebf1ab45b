"""TEST INFRASTRUCTURE ONLY: a plain numpy restatement of the learned tile proposer, for the GPU kernels' parity tests.

The paper ends (Section 5) with the remark that thinning the candidate list would cut the runtime further.  The
learned tile proposer is a small convolutional network that, for each 32x32 tile of the center disparity map D and
each peripheral view (alpha, r), predicts whether the scan lines of the tile's candidates (Eq. 2, Eq. 4) find an
occlusion (Eq. 5-6), so that the tiles it rules out need not be scanned.  It is trained on labels produced by the plain
method.  This file computes its forward pass, loss and gradients the slow, obvious way:

  input      x0[y][x] = bf16(fl(D * 1/32) - 1) in channel 0 of 8 (channels 1..7 are zero)
  4 layers   a_l = bf16(relu(conv3x3_same(a_{l-1}, bf16(W_l)) + b_l)), channels 8 -> 16 -> 16 -> 32 -> 16,
             zero padding, products of bf16 values summed in binary32
  view code  g(v) = We (cos alpha, sin alpha, r) + be        (16 values; cos and sin as the detection rounds them)
  pixel      z_v[y][x] = sum_c a_4[y][x][c] g_c(v) + b0
  tile       s_v(t) = log(mean over the tile's pixels of exp(z_v))   (log-sum-exp pooling; partial tiles average
             over their own pixels)
  loss       mean over (view, tile) of -(w y log sigmoid(s) + (1 - y) log(1 - sigmoid(s))), w = positive weight

and the gradients by the chain rule, with the tensors the GPU keeps in bf16 rounded at the same points: the
activations a_l, the weights, and the back-propagated pre-activation gradients (gated by a_l > 0).  Every other
quantity is binary32 (or binary64 with rounding switched off, for the finite-difference pin).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module; the CUDA library never does.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(8, 16), (16, 16), (16, 32), (32, 16)]
FEATURES = 16
ENC = 3
TILE = 32


def param_count() -> int:
    return sum(co * 9 * ci + co for ci, co in LAYERS) + FEATURES * ENC + FEATURES + 1


def bf16(x) -> np.ndarray:
    """Round binary32 values to the nearest bfloat16 (ties to even), returned as binary32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def _identity(x):
    return x


def unpack(params, dtype=np.float32):
    """Flat parameter vector -> ([(W [co][9][ci], b [co]) per layer], We [16][3], be [16], b0)."""
    p = np.asarray(params, dtype=dtype)
    off = 0
    layers = []
    for ci, co in LAYERS:
        w = p[off:off + co * 9 * ci].reshape(co, 9, ci)
        off += co * 9 * ci
        b = p[off:off + co]
        off += co
        layers.append((w, b))
    We = p[off:off + FEATURES * ENC].reshape(FEATURES, ENC)
    off += FEATURES * ENC
    be = p[off:off + FEATURES]
    off += FEATURES
    return layers, We, be, p[off]


def pack(layers, We, be, b0, dtype=np.float32) -> np.ndarray:
    parts = []
    for w, b in layers:
        parts += [np.ravel(w), np.ravel(b)]
    parts += [np.ravel(We), np.ravel(be), np.ravel([b0])]
    return np.concatenate(parts).astype(dtype)


def shifted(X, dy: int, dx: int):
    """S[y][x] = X[y + dy][x + dx], zero outside the image (X is [H][W][C])."""
    H, W = X.shape[:2]
    S = np.zeros_like(X)
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    S[yd, xd] = X[ys, xs]
    return S


TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]   # tap index (dy + 1) * 3 + (dx + 1)


def conv3x3_same(X, Wt, b):
    """Y[y][x][co] = b[co] + sum over taps and ci of Wt[co][tap][ci] X[y + dy][x + dx][ci] (zero padding)."""
    H, W, _ = X.shape
    Y = np.zeros((H, W, Wt.shape[0]), dtype=X.dtype) + b.astype(X.dtype)
    for t, (dy, dx) in enumerate(TAPS):
        Y = Y + shifted(X, dy, dx) @ Wt[:, t, :].T.astype(X.dtype)
    return Y


def tiles(H: int, W: int):
    """(ty, tx, y-slice, x-slice) of every tile, row-major."""
    for ty in range((H + TILE - 1) // TILE):
        for tx in range((W + TILE - 1) // TILE):
            yield ty, tx, slice(ty * TILE, min(H, (ty + 1) * TILE)), slice(tx * TILE, min(W, (tx + 1) * TILE))


def encodings(views, dtype=np.float32):
    """(cos alpha, sin alpha, r) of every view, cos and sin as the detection computes them."""
    from . import direction
    return np.array([[*direction(a), r] for a, r in views], dtype=dtype)


def forward(params, D, views, dtype=np.float32, rounding: bool = True):
    """Activations a_0..a_4, the view codes g [V][16], the pixel scores z [V][H][W] and the tile logits
    s [V][ty][tx]."""
    rnd = bf16 if rounding else _identity
    layers, We, be, b0 = unpack(params, dtype)
    D = np.asarray(D, dtype=np.float32)
    H, W = D.shape
    x0 = np.zeros((H, W, LAYERS[0][0]), dtype=dtype)
    x0[..., 0] = rnd((D * np.float32(0.03125) - np.float32(1.0)).astype(dtype))
    acts = [x0]
    for w, b in layers:
        pre = conv3x3_same(acts[-1], rnd(w).astype(dtype), b)
        acts.append(rnd(np.maximum(pre, 0).astype(dtype)))
    f = acts[-1]
    enc = encodings(views, dtype)
    g = enc @ We.T + be                                   # [V][16]
    z = np.einsum("yxc,vc->vyx", f, g) + b0               # [V][H][W]
    ty, tx = (H + TILE - 1) // TILE, (W + TILE - 1) // TILE
    s = np.zeros((len(views), ty, tx), dtype=dtype)
    for i, j, ys, xs in tiles(H, W):
        zt = z[:, ys, xs].reshape(len(views), -1)
        m = zt.max(axis=1, keepdims=True)
        s[:, i, j] = (np.log(np.exp(zt - m).sum(axis=1)) + m[:, 0] - np.log(zt.shape[1])).astype(dtype)
    return {"acts": acts, "g": g, "z": z, "s": s, "enc": enc}


def loss_and_grads(params, D, views, labels, pos_weight: float = 1.0, dtype=np.float32, rounding: bool = True):
    """Loss and its gradient with respect to the flat parameter vector (same layout)."""
    rnd = bf16 if rounding else _identity
    layers, We, be, b0 = unpack(params, dtype)
    fw = forward(params, D, views, dtype, rounding)
    acts, g, z, s, enc = fw["acts"], fw["g"], fw["z"], fw["s"], fw["enc"]
    y = np.asarray(labels, dtype=dtype)
    V, H, W = z.shape
    n = s.size
    sig = 1.0 / (1.0 + np.exp(-s))
    pw = dtype(pos_weight)
    # log sigmoid(s) and log(1 - sigmoid(s)) in their stable forms.
    log_p = -np.logaddexp(0.0, -s)
    log_q = -np.logaddexp(0.0, s)
    loss = float(np.mean(-(pw * y * log_p + (1 - y) * log_q)))
    ds = ((pw * y * (sig - 1) + (1 - y) * sig) / n).astype(dtype)

    dz = np.zeros_like(z)
    for i, j, ys, xs in tiles(H, W):
        zt = z[:, ys, xs]
        e = np.exp(zt - zt.reshape(V, -1).max(axis=1)[:, None, None])
        dz[:, ys, xs] = ds[:, i, j][:, None, None] * e / e.reshape(V, -1).sum(axis=1)[:, None, None]
    f = acts[-1]
    df = np.einsum("vyx,vc->yxc", dz, g)
    dg = np.einsum("vyx,yxc->vc", dz, f)
    dWe = dg.T @ enc
    dbe = dg.sum(axis=0)
    db0 = dz.sum()

    grads = [None] * len(layers)
    dpre = rnd((df * (f > 0)).astype(dtype))
    for li in range(len(layers) - 1, -1, -1):
        w, _ = layers[li]
        X = acts[li]
        dW = np.zeros_like(w)
        for t, (dy, dx) in enumerate(TAPS):
            dW[:, t, :] = np.einsum("yxo,yxi->oi", dpre, shifted(X, dy, dx))
        grads[li] = (dW, dpre.sum(axis=(0, 1)))
        if li > 0:
            wb = rnd(w).astype(dtype)
            dX = np.zeros_like(X)
            for t, (dy, dx) in enumerate(TAPS):
                dX = dX + shifted(dpre, -dy, -dx) @ wb[:, t, :]
            dpre = rnd((dX * (X > 0)).astype(dtype))
    return loss, pack(grads, dWe, dbe, db0, dtype)


def grad_magnitudes(params, D, views, labels, pos_weight: float = 1.0):
    """For every gradient element, the sum of the absolute values of the terms that loss_and_grads adds up for it:
    the same chain rule, in float64, with every factor replaced by its absolute value and every ReLU gate open.

    A parity test bounds the difference between two evaluations of the gradient that round differently (other
    summation order, a bf16 rounding that lands on the other side) by a small multiple of 2^-8 times this sum, element
    by element: each of the roundings on a path through the network moves a term by at most that fraction of its
    magnitude, and a gate that flips drops or adds a term that this sum already counts."""
    layers, We, be, b0 = unpack(params, np.float64)
    fw = forward(params, D, views, np.float64, rounding=True)
    acts, g, z, s, enc = fw["acts"], fw["g"], fw["z"], fw["s"], fw["enc"]
    y = np.asarray(labels, dtype=np.float64)
    V, H, W = z.shape
    n = s.size
    sig = 1.0 / (1.0 + np.exp(-s))
    ds = np.abs(pos_weight * y * (sig - 1)) / n + np.abs((1 - y) * sig) / n
    dz = np.zeros_like(z)
    for i, j, ys, xs in tiles(H, W):
        zt = z[:, ys, xs]
        e = np.exp(zt - zt.reshape(V, -1).max(axis=1)[:, None, None])
        dz[:, ys, xs] = ds[:, i, j][:, None, None] * e / e.reshape(V, -1).sum(axis=1)[:, None, None]
    f = acts[-1]
    ag = np.abs(g)
    df = np.einsum("vyx,vc->yxc", dz, ag)
    dg = np.einsum("vyx,yxc->vc", dz, np.abs(f))
    dWe = dg.T @ np.abs(enc)
    dbe = dg.sum(axis=0)
    db0 = dz.sum()
    grads = [None] * len(layers)
    dpre = df
    for li in range(len(layers) - 1, -1, -1):
        w, _ = layers[li]
        X = np.abs(acts[li])
        dW = np.zeros_like(w)
        for t, (dy, dx) in enumerate(TAPS):
            dW[:, t, :] = np.einsum("yxo,yxi->oi", dpre, shifted(X, dy, dx))
        grads[li] = (dW, dpre.sum(axis=(0, 1)))
        if li > 0:
            wa = np.abs(bf16(w.astype(np.float32))).astype(np.float64)
            dX = np.zeros_like(X)
            for t, (dy, dx) in enumerate(TAPS):
                dX = dX + shifted(dpre, -dy, -dx) @ wa[:, t, :]
            dpre = dX
    return pack(grads, dWe, dbe, db0, np.float64)
