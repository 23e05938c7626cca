"""Exact polygon counts from integer closure maps on the device (count_b of App. A / Eq. Ncalc).

Plans whose FP64 counting-field sums can no longer be rounded safely (large n = 5, 6
plans) take the closure-map route; POLY_COUNTS_EXACT=1 forces it, which these tests
use (in a child process, since counts are cached per process) to compare the route
with the oracle's exact counts bit for bit on plans of every order.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import fieldgen
import oracle

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1904_11055_gb300 import build

    build.build()
    oracle.set_threads(os.cpu_count() or 1)


def forced_exact_counts(N, order, nshell, width=1.0, flags=0):
    """Counts of a plan created in a child process with the closure-map route forced."""
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import fieldgen, paper_1904_11055_gb300 as ps; "
            f"p = ps.Plan({N}, 1000.0, {order}, fieldgen.unit_edges({nshell}, {width}), 'fp32', {flags}); "
            f"print(json.dumps(p.counts.tolist()))")
    env = dict(os.environ, POLY_COUNTS_EXACT="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return np.array(json.loads(out.stdout.strip().splitlines()[-1]), dtype=np.int64)


@pytest.mark.parametrize("N,order,nshell,width", [(48, 3, 12, 1.0), (32, 4, 7, 1.0), (48, 4, 7, 1.5),
                                                  (48, 5, 6, 1.0), (64, 6, 5, 1.0)])
def test_closure_map_route_matches_the_oracle(N, order, nshell, width):
    e = fieldgen.unit_edges(nshell, width)
    exact = forced_exact_counts(N, order, nshell, width)
    plan = ps.Plan(N, 1000.0, order, e, "fp32")  # this process: the FP64 counting-field route
    assert np.array_equal(exact, plan.counts)
    ref = oracle.counts_exact(N, e, order, plan.bins)
    assert np.array_equal(exact, ref)
    plan.close()


def test_large_order5_plan_gets_exact_counts():
    """128^3, 20 unit shells, n = 5: counts up to 1e13, beyond what the FP64 counting-field sum rounds
    safely (plan creation used to refuse it); the closure-map counts of the largest bins against the
    oracle's exact counts."""
    N, e = 128, fieldgen.unit_edges(20)
    plan = ps.Plan(N, 1000.0, 5, e, "fp32")
    assert plan.counts.max() > 10 ** 12
    idx = np.argsort(plan.counts)[-6:]
    ref = oracle.counts_exact(N, e, 5, plan.bins[idx])
    assert np.array_equal(plan.counts[idx], ref)
    plan.close()
