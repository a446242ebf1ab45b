"""The learned tile proposer end to end: labels from the plain method, training on the GPU with the library's own
forward / backward / Adam kernels, calibration of the skip threshold for a pixel recall target, and use.

Labels.  For a frame and a view, tile t is labelled 1 when the scan lines walked from the candidates of t (Eq. 2,
Eq. 4) add a non-zero count to O (Eq. 5-6): the tile_hits output of occ_detect_batched_tiles.

Proposal.  A tile is skipped only where the network is confident it is empty: logit <= threshold.  Every other tile
runs the plain method (the fallback for uncertain tiles).  Skipping only removes scan lines, so O can only decrease
and the mask of the proposed run is a subset of the plain mask: precision against the plain mask is 1 by
construction, and the threshold is chosen on held-out frames as the largest one whose pixel recall reaches the
target (0.999 by default).
"""
from __future__ import annotations


import numpy as np

from . import Net, occ_detect_batched, occ_net_propose, tiles_of


def labels_for(ctx, D, views, chunk: int = 64):
    """uint8 labels [n][V][tiles_y][tiles_x] of the frames D ([n][H][W] CUDA tensor) from the plain method."""
    import torch
    n, H, W = D.shape
    ty, tx = tiles_of(H, W)
    V = len(views)
    out = torch.empty((n, V, ty, tx), dtype=torch.uint8, device=D.device)
    M = [torch.empty((V, H, W), dtype=torch.uint8, device=D.device) for _ in range(chunk)]
    O = [torch.empty((V, H, W), dtype=torch.int32, device=D.device) for _ in range(chunk)]
    for s in range(0, n, chunk):
        k = min(chunk, n - s)
        occ_detect_batched(ctx, [D[s + i] for i in range(k)], views, Ms=M[:k], Os=O[:k],
                           hits=[out[s + i] for i in range(k)])
    return out


def train(net: Net, D, labels, views, epochs: int = 1, batch: int = 32, lr: float = 2e-3, pos_weight: float = 1.0,
          seed: int = 0, log_every: int = 0):
    """Adam on mini-batches of whole frames, shuffled per epoch.  Returns the loss of every step."""
    import torch
    n = D.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    step = 0
    bufD = torch.empty((batch, *D.shape[1:]), dtype=D.dtype, device=D.device)
    bufL = torch.empty((batch, *labels.shape[1:]), dtype=labels.dtype, device=D.device)
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).to(D.device)
        for s in range(0, n - batch + 1, batch):
            idx = order[s:s + batch]
            torch.index_select(D, 0, idx, out=bufD)
            torch.index_select(labels, 0, idx, out=bufL)
            step += 1
            loss, g = net.loss_grad(bufD, views, bufL, pos_weight=pos_weight)
            net.adam(g, step, lr=lr)
            losses.append(loss)
            if log_every and step % log_every == 0:
                print(f"epoch {ep} step {step} loss {float(loss.item()):.4f}", flush=True)
    return [float(x.item()) for x in losses]


def logits_for(net: Net, frames, views):
    """Tile logits of a list of [H][W] CUDA maps (frames of one size are run together, as many per call as the
    network's activation scratch holds)."""
    import torch
    out = [None] * len(frames)
    by_size = {}
    for i, f in enumerate(frames):
        by_size.setdefault(tuple(f.shape), []).append(i)
    for (H, W), idx in by_size.items():
        per_call = max(1, net.max_pixels // (H * W))
        for s0 in range(0, len(idx), per_call):
            part = idx[s0:s0 + per_call]
            D = torch.stack([frames[i] for i in part]) if len(part) > 1 else frames[part[0]].unsqueeze(0)
            s = net.forward(D.contiguous(), views)
            for k, i in enumerate(part):
                out[i] = s[k]
    return out


def masks(ctx, frames, views, proposals=None):
    """Masks of the plain (or, with proposals, the proposed) run, in batches that fit the context."""
    Ms = []
    s = 0
    while s < len(frames):
        e, px = s, 0
        while e < len(frames) and e - s < 1024 and px + frames[e].numel() <= ctx.max_pixels:
            px += frames[e].numel()
            e += 1
        if e == s:
            raise ValueError("a frame is larger than the context")
        part, _ = occ_detect_batched(ctx, frames[s:e], views, proposals=None if proposals is None else proposals[s:e])
        Ms += part
        s = e
    return Ms


def recall_precision(M_plain, M_prop):
    """Pixel recall and precision of the proposed run's masks against the plain masks (lists of uint8 tensors)."""
    tp = sum(int(((a != 0) & (b != 0)).sum().item()) for a, b in zip(M_plain, M_prop))
    pos = sum(int((a != 0).sum().item()) for a in M_plain)
    pred = sum(int((b != 0).sum().item()) for b in M_prop)
    return (tp / pos if pos else 1.0), (tp / pred if pred else 1.0)


def calibrate(net: Net, ctx, frames, views, target_recall: float = 0.999, iters: int = 14):
    """Largest threshold whose proposals keep pixel recall >= target on `frames` (bisection over the logits' range;
    recall does not increase with the threshold).  Returns (threshold, recall, skipped tile fraction)."""
    import torch
    logits = logits_for(net, frames, views)
    M_plain = masks(ctx, frames, views)
    allv = torch.cat([s.flatten() for s in logits])
    lo, hi = float(allv.min().item()) - 1.0, float(allv.max().item())
    best = (lo, 1.0, 0.0)

    def run(th):
        props = [occ_net_propose(s, th) for s in logits]
        rec, _ = recall_precision(M_plain, masks(ctx, frames, views, props))
        skipped = 1.0 - float(sum(int(p.sum().item()) for p in props)) / allv.numel()
        return rec, skipped

    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        rec, sk = run(mid)
        if rec >= target_recall:
            best = (mid, rec, sk)
            lo = mid
        else:
            hi = mid
    return best


def evaluate(net: Net, ctx, frames, views, threshold: float, reps: int = 5):
    """Recall, precision, skipped tiles and device times of the plain and the proposed runs on `frames`."""
    import torch
    M_plain = masks(ctx, frames, views)

    def plain():
        occ_detect_batched(ctx, frames, views, Ms=M_plain)

    M_prop = [torch.empty_like(m) for m in M_plain]
    state = {}

    def learned():
        logits = logits_for(net, frames, views)
        props = [occ_net_propose(s, threshold) for s in logits]
        occ_detect_batched(ctx, frames, views, Ms=M_prop, proposals=props)
        state["props"] = props

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_plain = timed(plain)
    t_learned = timed(learned)
    # Net alone (inference of all frames), for the breakdown.
    t_net = timed(lambda: logits_for(net, frames, views))
    rec, prec = recall_precision(M_plain, M_prop)
    tiles = sum(p.numel() for p in state["props"])
    kept = sum(int(p.sum().item()) for p in state["props"])
    return {"recall": rec, "precision": prec, "tiles": tiles, "skipped_tiles": 1.0 - kept / tiles,
            "ms_plain": t_plain, "ms_learned": t_learned, "ms_net": t_net, "speedup": t_plain / t_learned}
