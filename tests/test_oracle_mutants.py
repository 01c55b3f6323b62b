"""Planted mistakes in copies of the oracle: each one must fail at least one pin.

The pins (tests/test_oracle_pins.py) are meant to tie the oracle to what the paper and the
mathematics fix, so that a plausible slip anywhere in it -- a flipped sign, a wrong or
transposed index, a dropped term, a wrong normalisation, a loosened stopping rule, a changed
tie rule -- cannot pass unnoticed.  This test plants one slip at a time in a copy of
oracle/ot_oracle.c (on the CPU, in a temporary directory), rebuilds that copy, runs the pin
suite against it and requires a failure; the unmodified copy must pass.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name: (text in the oracle, the slip that replaces it)
MUTANTS = {
    "rates_sign": ("interference += P[k] * g[k];", "interference -= P[k] * g[k];"),
    "rates_index": ("if (k != j) interference += P[k] * g[k];", "if (k != j) interference += P[j] * g[k];"),
    "rates_log": ("log1p(sinr) / log(2.0)", "log1p(sinr)"),
    "rates_total_own": ("const double interference = ((t - own) + c) + N0;",
                        "const double interference = (t + c) + N0;"),
    "cost_mu": ("C_out[t] = 1.0 / (mu * R[t]);", "C_out[t] = mu / R[t];"),
    "row_sign": ("y[j] = (g[j] - C[i * J + j]) / eps;", "y[j] = (g[j] + C[i * J + j]) / eps;"),
    "row_drop_logp": ("f[i] = eps * log(p[i]) - eps * lse_row(y, J);", "f[i] = - eps * lse_row(y, J);"),
    "col_transpose": ("s += exp((f[i] - C[i * J + j]) / eps - m);",
                      "s += exp((f[i] - C[(j % I) * J + (i % J)]) / eps - m);"),
    "col_drop_max": ("g[j] = eps * log(q[j]) - eps * (m + log(s));", "g[j] = eps * log(q[j]) - eps * (log(s));"),
    "lse_no_shift": ("return m + log(s);", "return log(s);"),
    "plan_sign": ("return exp((f[i] + g[j] - C[i * J + j]) / eps);",
                  "return exp((f[i] - g[j] - C[i * J + j]) / eps);"),
    "median_even": ("m = 0.5 * (lo + hi);", "m = lo;"),
    "stop_early": ("if (err <= tol || k >= max_iter) break;", "if (err <= 10*tol || k >= max_iter) break;"),
    "norm_shift": ("double shift = eps * log(sp);", "double shift = 0.0;"),
    "finalize_rho": ("rho_out[j] = c;", "rho_out[j] = s;"),
    "finalize_row_mass": ("*err_row_out = er / mass;", "*err_row_out = er;"),
    "finalize_col_mass": ("*err_col_out = ec / mass;", "*err_col_out = ec;"),
    "maxsinr_tie": ("if (R[i * J + j] > R[i * J + best]) best = j;",
                    "if (R[i * J + j] >= R[i * J + best]) best = j;"),
    "adaptive_split": ("q[j] + d / (double)(J - 1);", "q[j] + d / (double)(J);"),
    "completion_queue": ("Ti += pij * C[i * J + j] / (1.0 - rho[j]);", "Ti += pij * C[i * J + j];"),
    "completion_mean": ("*T_out = T / (double)I;", "*T_out = T;"),
    "euclid_axis": ("const double dy = dev_xy[2 * i + 1] - rrh_xy[2 * j + 1];",
                    "const double dy = dev_xy[2 * i + 1] - rrh_xy[2 * j];"),
}


def _copy_tree(dst: str) -> None:
    skip = shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.o")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=skip)
    os.makedirs(os.path.join(dst, "paper_1805_01559_gb300"))
    for f in ("__init__.py", "instances.py"):  # the pins draw their inputs from the generators
        shutil.copy(os.path.join(ROOT, "paper_1805_01559_gb300", f), os.path.join(dst, "paper_1805_01559_gb300", f))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)


def _pins_pass(dst: str) -> bool:
    env = dict(os.environ)
    env.pop("PYTHONPATH", None)
    env["OMP_NUM_THREADS"] = "2"
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=dst, env=env, capture_output=True, text=True,
                       timeout=900)
    return r.returncode == 0


def _run(tmp: str, name: str, slip) -> bool:
    dst = os.path.join(tmp, name)
    _copy_tree(dst)
    if slip is not None:
        path = os.path.join(dst, "oracle", "ot_oracle.c")
        src = open(path).read()
        a, b = slip
        assert src.count(a) >= 1, f"{name}: the text to mutate is not in the oracle"
        open(path, "w").write(src.replace(a, b, 1))
    return _pins_pass(dst)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    jobs = {"unmodified": None, **MUTANTS}
    workers = max(1, min(6, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(_run, str(tmp_path), name, slip) for name, slip in jobs.items()}
        passed = {name: f.result() for name, f in futs.items()}
    assert passed.pop("unmodified"), "the pins fail on the unmodified oracle"
    missed = sorted(name for name, ok in passed.items() if ok)
    assert not missed, f"planted mistakes the pins do not catch: {missed}"
