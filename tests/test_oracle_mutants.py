"""Planted mistakes: each mutant copy of the oracle source (a dropped term, a wrong sign or
index, a transposed operand) must fail at least one pin in test_oracle_pins.py.  Runs on the
CPU only; the committed oracle is untouched."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lhf_oracle.c")

MUTANTS = {
    "mass_cross_sign": ("mass += 4.0 * fg + cross;", "mass += 4.0 * fg - cross;"),
    "kinetic_diag": ("kin += 2.0 * fg - cross;", "kin += 1.0 * fg - cross;"),
    "kinetic_half": ("Hb[e] = 0.5 * tk - v;", "Hb[e] = tk - v;"),
    "potential_sign": ("Hb[e] = 0.5 * tk - v;", "Hb[e] = 0.5 * tk + v;"),
    "laplacian_term_dropped": ("M[0][e] * M[1][e] * K[2][e];", "0.0;"),
    "half_weight_window": ("? 0.5 : 1.0;\n            double c = c0 + k * s->b[l];", "? 1.0 : 1.0;\n            double c = c0 + k * s->b[l];"),
    "image_shift_sign": ("double c = c0 + k * s->b[l];\n            double dmin", "double c = c0 - 2 * k * s->b[l];\n            double dmin"),
    "p_factor_direction": ("if (s->kind[mu] == 1 + l)", "if (s->kind[mu] == 2 - l)"),
    "dft_sign": ("double ph = -2.0 * ORC_PI *", "double ph = -1.0 * ORC_PI *"),
    "embedding_transpose": ("Xe[(size_t)i * n + j + m] = -xi;", "Xe[(size_t)i * n + j + m] = xi;"),
    "lindep_scale": ("X[(size_t)i * nk + a] = V[(size_t)i * n + kept[a]] / sqrt(", "X[(size_t)i * nk + a] = V[(size_t)i * n + kept[a]] * sqrt("),
    "drop_rule": ("if (Sk[2 * ((size_t)i * m + i)] > tau * s0[i]) keep[mr++] = i;", "keep[mr++] = i;"),
    "drop_threshold_x100": ("> tau * s0[i]) keep[mr++] = i;", "> 100.0 * tau * s0[i]) keep[mr++] = i;"),
    "drop_threshold_div100": ("> tau * s0[i]) keep[mr++] = i;", "> 0.01 * tau * s0[i]) keep[mr++] = i;"),
    "s0_from_kappa_0_only": ("s0[i] += Sbar[k * mm2 + 2 * ((size_t)i * m + i)];", "s0[i] += Sbar[2 * ((size_t)i * m + i)];"),
    "first_weight_tail": ("w[0] = w[0] / (1.0 - exp(-du));", "w[0] = w[0];"),
    "cell_shift": ("double A = s->centre[3 * mu + l] + cell * s->b[l];", "double A = s->centre[3 * mu + l] - cell * s->b[l];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, f"mutation anchor missing for {name}"
    mutant = tmp_path / "lhf_oracle_mutant.c"
    mutant.write_text(src.replace(old, new, 1))
    sys.path.insert(0, ROOT)
    import oracle

    lib = oracle.compile_source(str(mutant), str(tmp_path / "liblhf_oracle_mutant.so"))
    env = dict(os.environ, LHF_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived every pin:\n{r.stdout[-2000:]}"
