"""The multi-GPU path is replicas only (samples are independent): each rank solves
its own batch and the run reduces two host numbers.  Checked here on CPU with two
gloo ranks, no GPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_steps_and_ranks_tile_the_sample_stream():
    bench = _bench()
    S, world, steps = 5, 3, 4
    seen = []
    for k in range(steps):
        for r in range(world):
            s0 = bench.step_offset(k, world, r, S)
            seen.extend(range(s0, s0 + S))
    assert sorted(seen) == list(range(steps * world * S))


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    # rank r took (r + 1) seconds and converged 10 (r + 1) samples
    el, conv = bench.job_totals(1.0 + rank, 10 * (rank + 1), tdist, "cpu")
    out[rank] = (el, conv)
    tdist.barrier()
    tdist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_totals_max_time_and_summed_count_over_two_gloo_ranks():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (2.0, 30)


def test_job_totals_single_process_is_identity():
    bench = _bench()
    assert bench.job_totals(1.5, 7) == (1.5, 7)
