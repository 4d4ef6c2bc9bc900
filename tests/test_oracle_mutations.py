"""Planted mistakes in a copy of the CPU oracle must fail its pins.

Each mutation is a plausible slip (a dropped term, a wrong sign, a swapped
index, a transposed operand) applied to a temporary copy of smoe_oracle.c,
compiled with the same flags; the pin suite then runs against the copy in a
subprocess and must fail.  Nothing here touches a GPU."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "smoe_oracle.c")

MUTATIONS = {
    "transposed_L": ("float z0 = fmaf(a, dx, t);", "float z0 = fmaf(a, dx, 0.0f);"),
    "wrong_cross_term": ("double z0 = (double)a * dx + (double)b * dy;",
                         "double z0 = (double)a * dx - (double)b * dy;"),
    "missing_half": ("pr->e = exp(lp - 0.5 * q);", "pr->e = exp(lp - q);"),
    "gate_weight_ignored": ("double lp = m->logpi ? (double)m->logpi[k] : 0.0;",
                            "double lp = 0.0;"),
    "gate_weight_grad_sign": ("gpi += sv;", "gpi -= sv;"),
    "rbf_normalised": ("double nrm = m->rbf ? 1.0 : D;", "double nrm = D;"),
    "rbf_grad_keeps_y": ("r += G[ch * HW + p] * (pr.mexp[ch] - (m->rbf ? 0.0 : Y[ch * HW + p]));",
                         "r += G[ch * HW + p] * (pr.mexp[ch] - Y[ch * HW + p]);"),
    "swapped_slope_index": ("v += w0 * dx + w1 * dy;", "v += w1 * dx + w0 * dy;"),
    "dropped_expert_mu_term": ("gmx -= gG * w[ch][0];", "gmx -= 0.0;"),
    "sign_grad_c": ("gc += -sv * pr.z1 * pr.dy;", "gc += sv * pr.z1 * pr.dy;"),
    "no_chain_rule_W": ("g_mu[2 * s] = gmx * (double)m->W;", "g_mu[2 * s] = gmx;"),
    "box_uses_min_axis": ("float lmax_p = half_tr + rt;", "float lmax_p = half_tr - rt;"),
    "adam_no_bias_correction": ("double bc1 = 1.0 - pow(b1, (double)step);", "double bc1 = 1.0;"),
    "predicate_strict": ("return q32 <= m->qmax;", "return q32 < m->qmax - 1e-3f;"),
    "empty_rule": ("y[ch * n + p] = D > 0.0 ? N[ch] / nrm : 0.0;",
                   "y[ch * n + p] = D > 0.0 ? N[ch] / nrm : 0.5;"),
    "points_swapped_xy": ("float x = xy[2 * p], yy = xy[2 * p + 1];",
                          "float x = xy[2 * p + 1], yy = xy[2 * p];"),
    "points_no_raster_bounds": ("if (x >= 0.0f && x < (float)m->W && yy >= 0.0f && yy < (float)m->H)",
                                "if (x == x && yy == yy)"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name        # every occurrence is mutated
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-fopenmp", str(mut), "-o", str(lib), "-lm"])
    env = dict(os.environ, SMOE_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"
