"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped factor, a wrong exponent, a swapped
weight or index, a wrong plane, a wrong sign or root in the update, a subset
step that leaks outside its subset)
in a temporary copy of the oracle, on the CPU, and checks that the pin suites
fail on it.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C_SRC = "oracle/caxsi_oracle.c"
PY_SRC = "oracle/__init__.py"

MUTATIONS = {
    "G_so exponent": (C_SRC, "pow(x * x + y * y, 1.5)", "pow(x * x + y * y, 1.0)"),
    "G_od power of s": (C_SRC, "(slen * slen * slen)", "(slen * slen)"),
    "dtheta edge offset": (C_SRC, "double h = 0.5 * g->p_z;", "double h = g->p_z;"),
    "Bragg half angle": (C_SRC, "o->u = sin(0.5 * o->theta);", "o->u = sin(o->theta);"),
    "dropped cos(theta/2)": (C_SRC, "* cos(0.5 * o->theta);", ";"),
    "dropped Jacobian E": (C_SRC, "phi[k] * E * dE / (g->hc * g->hc);\n        acc",
                           "phi[k] * dE / (g->hc * g->hc);\n        acc"),
    "swapped interpolation weights": (C_SRC, "return (1.0 - a) * f0 + a * f1;",
                                      "return a * f0 + (1.0 - a) * f1;"),
    "mask plane parameter": (C_SRC, "double t = (g->X_mask - x) / (g->X_det - x);",
                             "double t = (g->X_det - g->X_mask) / (g->X_det - x);"),
    "mask row/col transposed": (C_SRC, "mask[(long)rf * g->mask_cols + (long)cf]",
                                "mask[(long)cf * g->mask_rows + (long)rf]"),
    "object y pitch": (C_SRC, "* g->rho_y * g->p_y; }", "* g->p_y; }"),
    "adjoint weight": (C_SRC, "frow[l + 1] += base * ck * a;", "frow[l + 1] += base * ck * (1.0 - a);"),
    "energy bin centre": (C_SRC, "(k + 0.5) * dE", "(k + 1.0) * dE"),
    "angular factor": (C_SRC, "(1.0 + cos(o->theta) * cos(o->theta))", "(1.0 + cos(o->theta))"),
    "G_od from s_y": (C_SRC, "o->God = fabs(s[0]) /", "o->God = fabs(s[1]) /"),
    "mask ray from y = 0": (C_SRC, "double ym = y + t * (yp - y);", "double ym = t * yp;"),
    "G_so without the voxel's y": (C_SRC, "pow(x * x + y * y, 1.5)", "pow(x * x, 1.5)"),
    "dtheta across y": (C_SRC, [("double sp[3] = {s[0], s[1], s[2] + h};", "double sp[3] = {s[0], s[1] + h, s[2]};"),
                                ("double sm[3] = {s[0], s[1], s[2] - h};", "double sm[3] = {s[0], s[1] - h, s[2]};")]),
    "pixel y half pitch": (C_SRC, "return (n - 0.5 * (g->N - 1)) * g->p_y;", "return (n - 0.5 * g->N) * g->p_y;"),
    "mask z unscaled": (C_SRC, "double zm = t * zp;", "double zm = zp;"),
    # the same mistake in the forward and the adjoint (the adjoint identity cannot see it)
    "q step range / Q": (C_SRC, [("double dq = (g->q_max - g->q_min) / (g->Q - 1);",
                                  "double dq = (g->q_max - g->q_min) / g->Q;")] * 2),
    "no zero sample past the q grid": (C_SRC, [
        ("if (!(tau > -1.0 && tau < (double)Q)) return 0.0;",
         "if (!(tau >= 0.0 && tau <= (double)(Q - 1))) return 0.0;"),
        ("if (!(tau > -1.0 && tau < (double)g->Q)) continue;",
         "if (!(tau >= 0.0 && tau <= (double)(g->Q - 1))) continue;")]),
    "C dropped": (C_SRC, [("out[t] = g->C * acc;", "out[t] = acc;"), ("frow[l] *= g->C;", "frow[l] *= 1.0;"),
                          ("H[p * cols + v * g->Q + l] = g->C * pr.Gso", "H[p * cols + v * g->Q + l] = pr.Gso")]),
    "spectrum dropped": (C_SRC, [("double ck = phi[k] * E * dE / (g->hc * g->hc);",
                                  "double ck = E * dE / (g->hc * g->hc);")] * 2),
    "pixel z half pitch": (C_SRC, "return (m - 0.5 * (g->M - 1)) * g->p_z;", "return (m - 0.5 * g->M) * g->p_z;"),
    "dtheta one-sided": (C_SRC, "double sm[3] = {s[0], s[1], s[2] - h};", "double sm[3] = {s[0], s[1], s[2]};"),
    "EM mean without background": (PY_SRC, "    z = A(f_hat) + r\n    if np.any",
                                   "    z = A(f_hat)\n    if np.any"),
    # the update of Eq. 10 and its penalty terms (Appendices B-C)
    "Huber weight beyond delta": (PY_SRC, "1.0, delta / np.where(a > 0, a, 1.0))",
                                  "1.0, 1.0 / np.where(a > 0, a, 1.0))"),
    "psi_dot sign": (PY_SRC, "b5 += np.where(ok, huber_grad(d, delta), 0.0)",
                     "b5 += np.where(ok, huber_grad(-d, delta), 0.0)"),
    "b3 factor 2": (PY_SRC, "b3 += np.where(ok, 2.0 * huber_curv(d, delta), 0.0)",
                    "b3 += np.where(ok, huber_curv(d, delta), 0.0)"),
    "chi2 penalty sign": (PY_SRC, "chi2 = b1 + beta * (-f_hat * (b3 + b4) + b5 + b6)",
                          "chi2 = b1 + beta * (f_hat * (b3 + b4) + b5 + b6)"),
    "Lemma minus root": (PY_SRC, "root = (-b + np.sqrt(b * b + 4.0 * a * c)) / (2.0 * a)",
                         "root = (-b - np.sqrt(b * b + 4.0 * a * c)) / (2.0 * a)"),
    "q form: sin instead of sin^2": (PY_SRC, "np.cos(0.5 * theta) / s2 ** 2 * phi_fn", "np.cos(0.5 * theta) / s2 * phi_fn"),
    "q form: angular factor": (PY_SRC, "return q * (1.0 + np.cos(theta) ** 2)", "return q * (1.0 + np.cos(theta))"),
    "likelihood: ln y! off by one": (PY_SRC, "math.lgamma(v + 1.0)", "math.lgamma(v + 2.0)"),
    "likelihood: sign of y ln z": (PY_SRC, "np.sum(z - ylogz + _lgamma1(y))", "np.sum(z + ylogz + _lgamma1(y))"),
    "chi3 without f_hat": (PY_SRC, "chi3 = f_hat * b2\n", "chi3 = b2\n"),
    "Lemma linear case": (PY_SRC, "lin = np.where(b > 0, c / b, np.inf)", "lin = np.where(b > 0, b / c, np.inf)"),
    "Huber quadratic half": (PY_SRC, "np.where(a <= delta, 0.5 * t * t,", "np.where(a <= delta, t * t,"),
    # ordered subsets (Algorithm 5)
    "OS ratio outside the subset": (PY_SRC, "ok = in_subset & (z > 0)", "ok = z > 0"),
    "OS sensitivity of all pixels": (PY_SRC, "return At(np.asarray(in_subset, dtype=np.float64))",
                                     "return At(np.ones(np.shape(in_subset)))"),
}


def _run_mutant(name, work, env):
    """Plant one mutation in a copy of the oracle under `work` and run the pin
    suites on it: (pytest return code, end of its output), or (None, why) when
    the mutation's text is not in the source any more."""
    rel, *edit = MUTATIONS[name]
    edits = edit[0] if len(edit) == 1 else [tuple(edit)]
    src = open(os.path.join(ROOT, rel)).read()
    for before, after in edits:        # each pair replaces one occurrence, in order
        if before not in src:
            return None, f"text not found: {before!r}"
        src = src.replace(before, after, 1)
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), work / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), work / "pytest.ini")
    (work / rel).write_text(src)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "tests/test_oracle_recon.py"],
                       cwd=work, capture_output=True, text=True, timeout=600, env=env)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    # the mutants are independent: run them side by side, each oracle on 2 threads
    base = tmp_path_factory.mktemp("mutants")
    env = dict(os.environ, OMP_NUM_THREADS="2")
    names = sorted(MUTATIONS)
    workers = max(1, min(len(names), (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        futs = {n: ex.submit(_run_mutant, n, base / f"m{i}", env) for i, n in enumerate(names)}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, outcomes):
    rc, out = outcomes[name]
    assert rc is not None, f"mutation '{name}': {out}"
    assert rc != 0, f"mutation '{name}' survived the pins:\n{out}"
