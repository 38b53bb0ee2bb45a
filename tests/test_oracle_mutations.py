"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped factor, a wrong exponent, a swapped
weight or index, a wrong plane) in a temporary copy of the C oracle, on the
CPU, and checks that the pin suites fail on it.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "caxsi_oracle.c")

MUTATIONS = {
    "G_so exponent": ("pow(x * x + y * y, 1.5)", "pow(x * x + y * y, 1.0)"),
    "G_od power of s": ("(slen * slen * slen)", "(slen * slen)"),
    "dtheta edge offset": ("double h = 0.5 * g->p_z;", "double h = g->p_z;"),
    "Bragg half angle": ("o->u = sin(0.5 * o->theta);", "o->u = sin(o->theta);"),
    "dropped cos(theta/2)": ("* cos(0.5 * o->theta);", ";"),
    "dropped Jacobian E": ("phi[k] * E * dE / (g->hc * g->hc);\n        acc",
                           "phi[k] * dE / (g->hc * g->hc);\n        acc"),
    "swapped interpolation weights": ("return (1.0 - a) * f0 + a * f1;",
                                      "return a * f0 + (1.0 - a) * f1;"),
    "mask plane parameter": ("double t = (g->X_mask - x) / (g->X_det - x);",
                             "double t = (g->X_det - g->X_mask) / (g->X_det - x);"),
    "mask row/col transposed": ("mask[(long)rf * g->mask_cols + (long)cf]",
                                "mask[(long)cf * g->mask_rows + (long)rf]"),
    "object y pitch": ("* g->rho_y * g->p_y; }", "* g->p_y; }"),
    "adjoint weight": ("frow[l + 1] += base * ck * a;", "frow[l + 1] += base * ck * (1.0 - a);"),
    "energy bin centre": ("(k + 0.5) * dE", "(k + 1.0) * dE"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTATIONS[name]
    src = open(SRC).read()
    assert before in src
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    (tmp_path / "oracle" / "caxsi_oracle.c").write_text(src.replace(before, after, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "tests/test_oracle_recon.py"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation '{name}' survived the pins:\n{r.stdout[-2000:]}"
