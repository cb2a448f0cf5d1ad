"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
the pins in test_oracle_pins.py catch every one of them."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "msg_oracle.c")

# (name, original text, mutated text, pins expected to fail)
MUTATIONS = [
    ("west/east face swapped", "double aw = g->ax[j * g->nx + i - 1], ae = g->ax[j * g->nx + i];\n    double as = g->ay[(j - 1) * W + i], an = g->ay[j * W + i];\n    double idx2 = 1.0 / (g->dx * g->dx), idy2 = 1.0 / (g->dy * g->dy);\n    return",
     "double ae = g->ax[j * g->nx + i - 1], aw = g->ax[j * g->nx + i];\n    double as = g->ay[(j - 1) * W + i], an = g->ay[j * W + i];\n    double idx2 = 1.0 / (g->dx * g->dx), idy2 = 1.0 / (g->dy * g->dy);\n    return",
     "symmetric_positive or manufactured"),
    ("dy^2 dropped", "- (an * (v[c + W] - v[c]) - as * (v[c] - v[c - W])) * idy2;",
     "- (an * (v[c + W] - v[c]) - as * (v[c] - v[c - W])) * idx2;", "sine_solution or printed_values"),
    ("full weighting centre weight", "return 0.25 * (f[c - 1] + 2.0 * f[c] + f[c + 1]);",
     "return 0.25 * (f[c - 1] + 1.0 * f[c] + f[c + 1]);", "restriction or rhs_restriction"),
    ("restriction average weights", "else v = 0.5 * Rx_at(fx, src ? fx->b : fx->r, i, j) + 0.5 * Ry_at(",
     "else v = 0.75 * Rx_at(fx, src ? fx->b : fx->r, i, j) + 0.25 * Ry_at(", "restriction"),
    ("kappa transposed", "*kx = lx * lx / (lx * lx + ly * ly);", "*kx = ly * ly / (lx * lx + ly * ly);", "kappa"),
    ("cubic weight", "return (-cm1 + 9.0 * c0 + 9.0 * c1 - c2) / 16.0;", "return (-cm1 + 8.0 * c0 + 9.0 * c1 - c2) / 16.0;",
     "cubic"),
    ("cubic boundary ghost sign", "double cm1 = (k - 1 >= 0) ? c[(k - 1) * stride] : -c[1 * stride];",
     "double cm1 = (k - 1 >= 0) ? c[(k - 1) * stride] : c[1 * stride];", "cubic"),
    ("residual sign", "for (int c = 0; c < n; ++c) g->r[c] = g->b[c] - g->r[c];",
     "for (int c = 0; c < n; ++c) g->r[c] = g->b[c] + g->r[c];", "dense_solves or contraction"),
    ("face placement", "a = exp(Z[row + (2 * i + 1) * sx]);", "a = exp(Z[row + (2 * i) * sx]);", "injection"),
    ("series mean segment", "for (int k = 0; k < sx; ++k) s += exp(-Z[row + 2 * (i * sx + k) + 1]);",
     "for (int k = 0; k < sx; ++k) s += exp(-Z[row + 2 * (i * sx + k)]);", "series_mean"),
    ("integral weight", "return g->dx * g->dy * s;", "return g->dx * s;", "printed_values or qoi_closed"),
    ("mixed difference term", "if (t1 > 0) d1_at_t2m1 -= Qgrid[(p0 + t1 - 2) * Qn + (q0 + t2 - 2)];",
     "", "worked_example or telescoping"),
    ("philox multiplier", "0xD2E7470EE14C6C93ULL * x0", "0xD2E7470EE14C6C95ULL * x0", "philox"),
    ("flux boundary column", "double a = exp(Z[(int64_t)(2 * j * sy) * NFx + (NFx - 1)]);",
     "double a = exp(Z[(int64_t)(2 * j * sy) * NFx + (NFx - 2)]);", "boundary_column"),
    ("flux boundary row", "double a = exp(Z[(int64_t)(2 * j * sy) * NFx + (NFx - 1)]);",
     "double a = exp(Z[(int64_t)(2 * j * sy + 1) * NFx + (NFx - 1)]);", "boundary_column"),
    ("divergence against the zero guess only",
     "while (!(rr <= H->eps) && n < H->max_cycles && rr == rr && (rr <= 1.0 || rr <= rr0));",
     "while (!(rr <= H->eps) && n < H->max_cycles && rr == rr && rr <= 1.0);", "keeps_cycling"),
    ("box-muller radius", "double rad = sqrt(-2.0 * log(1.0 - ua));", "double rad = sqrt(-1.0 * log(1.0 - ua));",
     "normals_distribution"),
    ("standard restriction corner weight", "return (4.0 * r[c] + 2.0 * edge + corner) / 16.0;",
     "return (4.0 * r[c] + 2.0 * edge + 2.0 * corner) / 16.0;", "std_transfer"),
    ("bilinear cell-centre weight",
     "return 0.25 * (v[j0 * W + i0] + v[j0 * W + i0 + 1] + v[(j0 + 1) * W + i0] + v[(j0 + 1) * W + i0 + 1]);",
     "return 0.25 * (v[j0 * W + i0] + v[j0 * W + i0 + 1] + v[(j0 + 1) * W + i0] + v[(j0 + 1) * W + i0]);",
     "std_transfer"),
    ("line solve elimination", "double d = diag_at(g, i, j) - (k > 0 ? lo * cp[k - 1] : 0.0);",
     "double d = diag_at(g, i, j);", "line_solve"),
]


@pytest.mark.parametrize("name,orig,mut,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, mut, pins):
    src = open(SRC).read()
    assert orig in src, f"mutation anchor for '{name}' not found in the oracle"
    bad = src.replace(orig, mut, 1)
    c = tmp_path / "bad.c"
    so = tmp_path / "libbad.so"
    c.write_text(bad)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", pins],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"planted mistake '{name}' was not caught:\n{r.stdout[-2000:]}"
