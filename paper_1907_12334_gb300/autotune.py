"""Launch-shape autotuner for msg_solve_batch.

The solver's results do not depend on its launch shapes; its speed does.  Three
shapes are tuned per call through msg_params: the threads per CTA of the
per-visit kernels (``tune_block``), the items per CTA of the warp-resident
kernel (``tune_low_warps``) and the largest relative diagonal whose grids are
visited one warp per grid (``tune_warp_visit``).  ``tune`` times
msg_solve_batch on a sub-batch of the caller's own samples (CUDA events on the
launching stream) over a small grid of candidates by coordinate descent and
caches the best triple per batch composition.  It runs outside any timed
region.
"""
from __future__ import annotations

import collections
import dataclasses

import numpy as np

_cache: dict = {}


def _key(PQ, prm):
    cnt = collections.Counter(map(tuple, np.asarray(PQ).reshape(-1, 2).tolist()))
    return (tuple(sorted(cnt.items())), prm.precision, prm.mu, prm.nu1, prm.nu2, prm.eps)


def _time_solve(msg, torch, PQ, Z, prm, ws, Q, st):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    msg.msg_solve_batch(PQ, prm, Z, Q, st, workspace=ws)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def tune(PQ, Z, prm, blocks=(128, 256, 512), warps=(2, 4, 8), warp_visit=(4, 6, 8), sample=256, verbose=False):
    """Return a copy of prm with the fastest (tune_block, tune_low_warps, tune_warp_visit) for this batch.

    PQ: [S][2] shapes; Z: device tensor of the packed fields (as msg_solve_batch takes)."""
    import torch

    from . import msg

    pq = np.ascontiguousarray(np.asarray(PQ, dtype=np.int32).reshape(-1, 2))
    key = _key(pq, prm)
    if key in _cache:
        b, w, v = _cache[key]
        return dataclasses.replace(prm, tune_block=b, tune_low_warps=w, tune_warp_visit=v)
    n = min(sample, pq.shape[0])
    sub = pq[:n]
    _, nf = msg.packed_sizes(sub)
    Zs = Z[:nf]
    nq, _ = msg.packed_sizes(sub)
    Q = torch.empty(nq, dtype=torch.float64, device=Z.device)
    st = torch.empty(n, dtype=torch.int32, device=Z.device)
    ws = torch.empty(max(msg.msg_workspace_bytes(sub, dataclasses.replace(prm, tune_low_warps=w))
                         for w in warps), dtype=torch.uint8, device=Z.device)
    best_b, best_w, best_v = 256, 4, 4
    trials = {}

    def run(b, w, v):
        if (b, w, v) not in trials:
            trials[(b, w, v)] = _time_solve(msg, torch, sub, Zs, dataclasses.replace(
                prm, tune_block=b, tune_low_warps=w, tune_warp_visit=v), ws, Q, st)
        return trials[(b, w, v)]

    run(best_b, best_w, best_v)  # warm-up of the default shape (first call pays one-time costs)
    trials.clear()
    best_v = min(warp_visit, key=lambda v: run(best_b, best_w, v))
    best_b = min(blocks, key=lambda b: run(b, best_w, best_v))
    best_w = min(warps, key=lambda w: run(best_b, w, best_v))
    if verbose:
        print("autotune:", {f"{b}x{w}x{v}": round(t, 2) for (b, w, v), t in trials.items()})
    _cache[key] = (best_b, best_w, best_v)
    return dataclasses.replace(prm, tune_block=best_b, tune_low_warps=best_w, tune_warp_visit=best_v)
