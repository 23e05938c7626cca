"""Plants one mistake at a time in a copy of the oracle and checks that a pin fails.

Each mutant is a textual edit of oracle/oracle.c compiled into a temporary
library; the pins of test_oracle_fft.py / test_oracle_estimator.py then run in a
subprocess against it and must fail.  This shows that a dropped term, a wrong
sign, index or exponent anywhere in the oracle is caught by something other
than the oracle itself.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "twiddle_sign": ("tw[j].im = sign * sin(a);", "tw[j].im = -sign * sin(a);", "test_oracle_fft.py"),
    "fft_index": ("cplx y = out[(size_t)r * m + (k % m)];", "cplx y = out[(size_t)r * m + (k % p)];",
                  "test_oracle_fft.py"),
    "shell_edge_unsquared": ("if (edges[s] * edges[s] <= d &&", "if (edges[s] <= d &&",
                             "test_oracle_estimator.py -k shell_map"),
    "dropped_factor": ("for (int t = 0; t < c->order; t++) p *= f[t][x];",
                       "for (int t = 0; t < c->order - 1; t++) p *= f[t][x];",
                       "test_oracle_estimator.py -k direct_sampling"),
    "normalisation_power": ("double norm = pow(L * L * L, order - 1) / pow(n3d, order);\n        for (int64_t b = 0; b < nbins; b++) {\n            double v",
                            "double norm = pow(L * L * L, order) / pow(n3d, order);\n        for (int64_t b = 0; b < nbins; b++) {\n            double v",
                            "test_oracle_estimator.py -k 'textbook or iid'"),
    "count_scale": ("double v = C[b] / n3d;", "double v = C[b] / n3d * 0.5;",
                    "test_oracle_estimator.py -k 'counts_match_golden'"),
    "closure_sign": ("int la = ((-sa) % N + N) % N,", "int la = ((sa) % N + N) % N,",
                     "test_oracle_estimator.py -k 'direct'"),
    "polygon_strict": ("if (rule == 1 || centre[cur[0] - 1] <= rest + 1e-9 * centre[cur[0] - 1])",
                       "if (rule == 1 || centre[cur[0] - 1] < rest)", "test_oracle_estimator.py -k bin_enumeration"),
    "adjoint_all_factors": ("if (u != t) p *= D[(size_t)(k[u] - 1) * n3 + x];", "p *= D[(size_t)(k[u] - 1) * n3 + x];",
                            "test_oracle_estimator.py -k gradient"),
    "adjoint_no_mask": ("if (smap[q] == m) H[q] = work[q];", "if (smap[q] >= 0) H[q] = work[q];",
                        "test_oracle_estimator.py -k gradient"),
    "group_dropped_factor": ("for (int f = 1; f < nf; f++) {", "for (int f = 1; f < nf - 1; f++) {",
                             "test_oracle_estimator.py -k n5_n6"),
    "group_wrong_partner": ("c.b = G + n3 * (size_t)bg[2 * b + 1];", "c.b = G + n3 * (size_t)bg[2 * b];",
                            "test_oracle_estimator.py -k n5_n6"),
    "disconnected_pairing": ("if (k[0] == k[1] && k[2] == k[3]) sd += p1 * p3;", "if (k[0] == k[1]) sd += p1 * p3;",
                             "test_oracle_estimator.py -k disconnected"),
    "disconnected_power": ("P[smap[i]] += dhat[2 * i] * dhat[2 * i] + dhat[2 * i + 1] * dhat[2 * i + 1];",
                           "P[smap[i]] += dhat[2 * i] * dhat[2 * i];", "test_oracle_estimator.py -k disconnected"),
    "legendre_sign": ("((2.0 * n + 1.0) * mu * p1 - n * p0) / (n + 1.0);", "((2.0 * n + 1.0) * mu * p1 + n * p0) / (n + 1.0);",
                      "test_oracle_estimator.py -k multipole"),
    "multipole_axis": ("legendre(ell, qz / sqrt(qx * qx + qy * qy + qz * qz));",
                       "legendre(ell, qx / sqrt(qx * qx + qy * qy + qz * qz));", "test_oracle_estimator.py -k multipole"),
    "full_shape_diagonal": ("const double w0 = signed_freq(x1, N) - signed_freq(x3, N),",
                            "const double w0 = signed_freq(x1, N) - signed_freq(x2, N),",
                            "test_oracle_estimator.py -k full_shape"),
    "multipole_factor": ("norm = (2.0 * ell + 1.0) * pow(L * L * L, order - 1)", "norm = pow(L * L * L, order - 1)",
                         "test_oracle_estimator.py -k multipole"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new, target = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(lib), str(mutated), "-lm",
                           "-lpthread"])
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=str(lib))
    parts = target.split(" ", 1)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", os.path.join(ROOT, "tests", parts[0])]
    if len(parts) > 1:
        cmd += ["-k", parts[1].split("-k ", 1)[1].strip("'")]
    res = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 1, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"
