"""Launch-shape autotuner for msg_solve_batch.

The solver's results do not depend on its launch shapes; its speed does.  Two
shapes are tuned per call through msg_params: the threads per CTA of the
per-visit kernels (``tune_block``) and the items per CTA of the low-diagonal
kernel (``tune_low_warps``).  ``tune`` times msg_solve_batch on a sub-batch of
the caller's own samples (CUDA events on the launching stream) over a small
grid of candidates by coordinate descent and caches the best pair per batch
composition.  It runs outside any timed region.
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


def tune(PQ, Z, prm, blocks=(128, 256), warps=(2, 4), sample=256, verbose=False):
    """Return a copy of prm with the fastest (tune_block, tune_low_warps) for this batch.

    PQ: [S][2] shapes; Z: device tensor of the packed fields (as msg_solve_batch takes)."""
    import torch

    from . import msg

    pq = np.ascontiguousarray(np.asarray(PQ, dtype=np.int32).reshape(-1, 2))
    key = _key(pq, prm)
    if key in _cache:
        b, w = _cache[key]
        return dataclasses.replace(prm, tune_block=b, tune_low_warps=w)
    n = min(sample, pq.shape[0])
    sub = pq[:n]
    nq, nf = msg.packed_sizes(sub)
    Zs = Z[:nf]
    Q = torch.empty(nq, dtype=torch.float64, device=Z.device)
    st = torch.empty(n, dtype=torch.int32, device=Z.device)
    ws = torch.empty(max(msg.msg_workspace_bytes(sub, dataclasses.replace(prm, tune_low_warps=w))
                         for w in warps), dtype=torch.uint8, device=Z.device)
    best_b, best_w = 128, 2
    trials = {}

    def run(b, w):
        if (b, w) not in trials:
            trials[(b, w)] = _time_solve(msg, torch, sub, Zs, dataclasses.replace(
                prm, tune_block=b, tune_low_warps=w), ws, Q, st)
        return trials[(b, w)]

    run(best_b, best_w)  # warm-up of the default shape (first call pays one-time costs)
    trials.clear()
    best_b = min(blocks, key=lambda b: run(b, best_w))
    best_w = min(warps, key=lambda w: run(best_b, w))
    if verbose:
        print("autotune:", {f"{b}x{w}": round(t, 2) for (b, w), t in trials.items()})
    _cache[key] = (best_b, best_w)
    return dataclasses.replace(prm, tune_block=best_b, tune_low_warps=best_w)
