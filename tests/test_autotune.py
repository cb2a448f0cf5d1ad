"""Host logic of the launch-shape autotuner (paper_1907_12334_gb300/autotune.py):
coordinate descent over the thread-block candidates, then over the low-kernel
shapes at the best block, one measurement per candidate pair, and a cache per
batch composition.  The timing call is replaced by a synthetic cost; the
library is only asked for workspace sizes (host arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1907_12334_gb300 import autotune, msg  # noqa: E402


@pytest.fixture(autouse=True)
def _fresh_cache():
    autotune._cache.clear()
    yield
    autotune._cache.clear()


def _run(monkeypatch, cost, PQ=None, prm=None):
    calls = []

    def fake_time(msg_, torch_, PQ_, Z_, prm_, ws_, Q_, st_):
        calls.append((prm_.tune_block, prm_.tune_low_items, prm_.tune_low_warps))
        return cost(prm_.tune_block, (prm_.tune_low_items, prm_.tune_low_warps))

    monkeypatch.setattr(autotune, "_time_solve", fake_time)
    PQ = np.array([[4, 3]] * 6 + [[3, 5]] * 2, dtype=np.int32) if PQ is None else PQ
    _, nf = msg.packed_sizes(PQ)
    Z = torch.zeros(nf, dtype=torch.float64)
    prm = prm or msg.SolverParams()
    return autotune.tune(PQ, Z, prm, sample=8), calls


def test_picks_the_fastest_block_then_the_fastest_low_shape(monkeypatch):
    msg.load()
    best_block, best_low = 256, (4, 8)

    def cost(b, lw):
        return 1.0 + (0.0 if b == best_block else 0.5) + (0.0 if lw == best_low else 0.25)

    out, calls = _run(monkeypatch, cost)
    assert out.tune_block == best_block
    assert (out.tune_low_items, out.tune_low_warps) == best_low
    # warm-up of the default pair, then len(blocks) + len(low shapes) - 1 distinct measurements
    assert len(calls) == 1 + len(autotune.BLOCKS) + len(autotune.LOW_SHAPES) - 1
    assert len(set(calls[1:])) == len(calls) - 1


def test_result_is_cached_per_batch_composition(monkeypatch):
    msg.load()
    out1, calls1 = _run(monkeypatch, lambda b, lw: 1.0 + (b == 64) * -0.5)
    assert out1.tune_block == 64
    out2, calls2 = _run(monkeypatch, lambda b, lw: 1.0)  # same composition: no new measurement
    assert calls2 == [] and out2.tune_block == 64
    # a different composition, or another schedule parameter, is tuned again
    _, calls3 = _run(monkeypatch, lambda b, lw: 1.0, PQ=np.array([[5, 5]] * 4, dtype=np.int32))
    assert calls3
    _, calls4 = _run(monkeypatch, lambda b, lw: 1.0, prm=msg.SolverParams(tune_low_cut=3))
    assert calls4


def test_tuning_leaves_the_rounding_parameters_alone(monkeypatch):
    msg.load()
    prm = msg.SolverParams(tune_low_cut=3, tune_visit_smem=8, eps=1e-9)
    out, _ = _run(monkeypatch, lambda b, lw: 1.0, prm=prm)
    assert (out.tune_low_cut, out.tune_visit_smem, out.eps) == (3, 8, 1e-9)
