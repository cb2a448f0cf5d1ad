"""Launch-shape autotuner for msg_solve_batch.

The solver's results do not depend on its launch shapes; its speed does.  The
shapes tuned here, per call through msg_params, are the threads per CTA of the
per-visit kernels (``tune_block``) and the items per warp and warps per CTA of
the low-diagonal kernel (``tune_low_items``, ``tune_low_warps``).  ``tune``
times msg_solve_batch on a sub-batch of the caller's own samples (CUDA events
on the launching stream) over a small set of candidates by coordinate descent,
starting from the library defaults, and caches the best per batch composition.
It runs outside any timed region.  Schedule parameters that change rounding
(``tune_low_cut``, ``tune_visit_smem``) stay as the caller set them.
"""
from __future__ import annotations

import collections
import dataclasses

import numpy as np

_cache: dict = {}

BLOCKS = (0, 64, 256)              # 0: library default
LOW_SHAPES = ((0, 0), (4, 8), (1, 16))  # (items per warp, warps per CTA); (0, 0): library default


def _key(PQ, prm):
    cnt = collections.Counter(map(tuple, np.asarray(PQ).reshape(-1, 2).tolist()))
    return (tuple(sorted(cnt.items())), prm.precision, prm.mu, prm.nu1, prm.nu2, prm.eps, prm.tune_low_cut,
            prm.tune_visit_smem)


def _time_solve(msg, torch, PQ, Z, prm, ws, Q, st):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    msg.msg_solve_batch(PQ, prm, Z, Q, st, workspace=ws)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def _with(prm, b, low):
    return dataclasses.replace(prm, tune_block=b, tune_low_items=low[0], tune_low_warps=low[1])


def tune(PQ, Z, prm, blocks=BLOCKS, low_shapes=LOW_SHAPES, sample=256, verbose=False):
    """Return a copy of prm with the fastest launch shapes for this batch.

    PQ: [S][2] shapes; Z: device tensor of the packed fields (as msg_solve_batch takes)."""
    import torch

    from . import msg

    pq = np.ascontiguousarray(np.asarray(PQ, dtype=np.int32).reshape(-1, 2))
    key = _key(pq, prm)
    if key in _cache:
        return _with(prm, *_cache[key])
    n = min(sample, pq.shape[0])
    sub = pq[:n]
    nq, nf = msg.packed_sizes(sub)
    Zs = Z[:nf]
    Q = torch.empty(nq, dtype=torch.float64, device=Z.device)
    st = torch.empty(n, dtype=torch.int32, device=Z.device)
    sizes = [msg.msg_workspace_bytes(sub, _with(prm, b, lw)) for b in blocks for lw in low_shapes]
    ws = torch.empty(max(sizes), dtype=torch.uint8, device=Z.device)
    trials = {}

    def run(b, lw):
        if (b, lw) not in trials:
            trials[(b, lw)] = _time_solve(msg, torch, sub, Zs, _with(prm, b, lw), ws, Q, st)
        return trials[(b, lw)]

    run(blocks[0], low_shapes[0])  # warm-up (the first call pays one-time costs)
    trials.clear()
    best_b = min(blocks, key=lambda b: run(b, low_shapes[0]))
    best_l = min(low_shapes, key=lambda lw: run(best_b, lw))
    if verbose:
        print("autotune:", {f"{b}/{lw}": round(t, 2) for (b, lw), t in trials.items()})
    _cache[key] = (best_b, best_l)
    return _with(prm, best_b, best_l)
