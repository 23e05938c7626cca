"""Full-shape trispectrum T(k1..k4; d1, d2) on the device (Eq. Tkfull, Sec. 2.1) against the FP64 oracle.

Counts are compared bit for bit.  T is compared element by element against
oracle.trispectrum_full on the same seeded field, in units of the oracle's
scale c_4 sum prod_t |dhat(q_t)| / count: |T_gpu - T_ref| <= tol * scale with
tol 1e-4 for FP32 plans (the FP32 forward transform and FP32 per-bin sums) and
1e-10 for FP64 plans.  At sizes the oracle cannot enumerate in seconds the
sums over all diagonal bins are checked against the angle-averaged estimator
of the same bin (counts exact, sums within the same bar).
"""
import os

import numpy as np
import pytest

import fieldgen
import oracle

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "split_bf16": 1e-4, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1904_11055_gb300 import build

    build.build()
    oracle.set_threads(os.cpu_count() or 1)


def unit_diagonals(top):
    """Diagonal bins [0, 0.5), [0.5, 1.5), ... up to top + 0.5."""
    return np.concatenate([[0.0], np.arange(top + 1) + 0.5])


def device_tfull(delta, L, edges, k, dedges, prec, order=2, flags=0):
    N = delta.shape[0]
    plan = ps.Plan(N, L, order, edges, prec, flags)
    d = torch.from_numpy(np.ascontiguousarray(delta)).to("cuda", plan.real_dtype)
    T, C, sc = plan.trispectrum_full(d, k, dedges, scale=True)
    torch.cuda.synchronize()
    return plan, T.cpu().numpy(), C.cpu().numpy(), sc.cpu().numpy()


def compare(T, C, ref, tol):
    assert np.array_equal(C, ref["counts"]), "counts differ from the oracle"
    assert np.array_equal(T == 0.0, ref["counts"] == 0)
    live = ref["counts"] > 0
    err = np.abs(T[live] - ref["T"][live]) / ref["scale"][live]
    assert err.max() <= tol, err.max()
    return err.max()


CASES = [
    # N, L, nshell, k, dedges, prec, seed
    (16, 300.0, 4, (4, 4, 4, 4), unit_diagonals(9), "fp32", 61),  # sums of three q wrap around the grid
    (24, 400.0, 5, (5, 4, 3, 2), unit_diagonals(10), "fp32", 62),
    (32, 500.0, 7, (7, 6, 5, 4), unit_diagonals(15), "fp32", 63),
    (32, 500.0, 7, (5, 7, 4, 6), np.linspace(0.0, 15.0, 41), "fp32", 64),  # 40 diagonal bins
    (24, 400.0, 5, (5, 4, 3, 2), np.linspace(0.0, 10.5, 101), "fp64", 74),  # tables too large for shared memory
    (32, 500.0, 7, (6, 6, 6, 6), np.array([1.0, 3.0, 4.5, 6.0, 9.0, 11.5]), "fp32", 65),  # ranges outside every bin
    (32, 500.0, 7, (7, 6, 5, 4), unit_diagonals(15), "split_bf16", 66),
    (32, 500.0, 5, (5, 5, 4, 3), unit_diagonals(11), "fp32", 73),  # 3K <= (N - 1) / 2: no sum needs reducing
    (24, 400.0, 5, (5, 5, 3, 3), unit_diagonals(10), "fp64", 67),
    (32, 500.0, 5, (5, 4, 4, 2), unit_diagonals(11), "fp64", 68),
]


@pytest.mark.parametrize("N,L,nshell,k,dedges,prec,seed", CASES)
def test_full_shape_matches_oracle(N, L, nshell, k, dedges, prec, seed):
    e = fieldgen.unit_edges(nshell)
    delta = fieldgen.field("lognormal", N, seed, np.float64 if prec == "fp64" else np.float32)
    plan, T, C, sc = device_tfull(delta, L, e, k, dedges, prec)
    ref = oracle.trispectrum_full(delta.astype(np.float64), L, e, k, dedges)
    compare(T, C, ref, TOL[prec])
    live = C > 0
    assert np.allclose(sc[live], ref["scale"][live], rtol=1e-4 if prec != "fp64" else 1e-10, atol=0.0)
    assert np.count_nonzero(C) > 3
    plan.close()


@pytest.mark.parametrize("order,prec,ell", [(3, "split_bf16", 0), (4, "fp32", 0), (3, "fp32", 2), (3, "fp64", 0)])
def test_any_plan_serves(order, prec, ell):
    """The full-shape trispectrum takes only the plan's shells, grid and forward transform from it: plans of
    other orders, the split-BF16 precision and a multipole plan give the oracle's T and counts."""
    N, L, nshell, k = 24, 400.0, 5, (5, 4, 3, 3)
    e = fieldgen.unit_edges(nshell)
    delta = fieldgen.field("lognormal", N, 75, np.float64 if prec == "fp64" else np.float32)
    de = unit_diagonals(10)
    plan = ps.Plan(N, L, order, e, prec, 0, ell)
    d = torch.from_numpy(np.ascontiguousarray(delta)).to("cuda", plan.real_dtype)
    T, C, sc = plan.trispectrum_full(d, k, de, scale=True)
    torch.cuda.synchronize()
    ref = oracle.trispectrum_full(delta.astype(np.float64), L, e, k, de)
    compare(T.cpu().numpy(), C.cpu().numpy(), ref, TOL[prec])
    plan.close()


def test_aliased_quadrilaterals_are_counted():
    """On 16^3 with shells up to 4.5, q1 = q2 = q3 = (4, 0, 0) closes with q4 = (4, 0, 0) only
    through the grid's periodicity: the device counts must include such quadrilaterals, as the
    oracle (which closes modulo N) does."""
    N, e, k = 16, fieldgen.unit_edges(4), (4, 4, 4, 4)
    plan = ps.Plan(N, 300.0, 2, e, "fp32")
    de = unit_diagonals(9)
    C = plan.trispectrum_full(None, k, de).cpu().numpy()
    ref = oracle.trispectrum_full(None, 300.0, e, k, de, N=N)
    assert np.array_equal(C, ref["counts"])
    # the same shells on 32^3 cannot wrap: the wrapped configurations are extra
    C32 = ps.Plan(32, 300.0, 2, e, "fp32").trispectrum_full(None, k, de).cpu().numpy()
    assert C.sum() > C32.sum()
    plan.close()


def test_counts_only_matches_oracle_at_48cube():
    N, e, k = 48, fieldgen.unit_edges(9), (9, 8, 7, 6)
    de = unit_diagonals(19)
    plan = ps.Plan(N, 700.0, 2, e, "fp32")
    C = plan.trispectrum_full(None, k, de).cpu().numpy()
    ref = oracle.trispectrum_full(None, 700.0, e, k, de, N=N)
    assert np.array_equal(C, ref["counts"])
    plan.close()


@pytest.mark.parametrize("N,L,nshell,k,prec,seed", [
    (32, 500.0, 7, (7, 6, 5, 4), "fp32", 69),
    (64, 800.0, 10, (10, 9, 8, 8), "fp32", 70),
    (256, 1000.0, 14, (14, 13, 12, 11), "fp32", 71),
    (64, 800.0, 10, (9, 9, 7, 5), "fp64", 72),
])
def test_sums_over_diagonals_give_the_angle_averaged_bin(N, L, nshell, k, prec, seed):
    """Eq. Tkfull: summed over diagonal bins covering every |q1 - q2| and |q1 - q3|, counts equal the
    angle-averaged estimator's count_b exactly and sum_j T_j count_j equals B_b count_b within the bar
    (both measured in units of sum_j scale_j count_j >= the scale of either sum)."""
    e = fieldgen.unit_edges(nshell)
    plan = ps.Plan(N, L, 4, e, prec)
    b = np.flatnonzero((plan.bins == np.asarray(k)).all(axis=1))
    assert b.size == 1
    d = torch.from_numpy(fieldgen.field("lognormal", N, seed, np.float64 if prec == "fp64" else np.float32)).cuda()
    B = plan.estimate(d).cpu().numpy()
    de = unit_diagonals(2 * nshell + 1)
    T, C, sc = plan.trispectrum_full(d, k, de, scale=True)
    torch.cuda.synchronize()
    T, C, sc = T.cpu().numpy(), C.cpu().numpy(), sc.cpu().numpy()
    assert C.sum() == plan.counts[b[0]]
    err = abs((T * C).sum() - B[b[0]] * plan.counts[b[0]]) / (sc * C).sum()
    assert err <= TOL[prec], err
    plan.close()


def test_full_shape_argument_checks():
    e = fieldgen.unit_edges(4)
    plan = ps.Plan(16, 300.0, 2, e, "fp32")
    d = torch.zeros((16, 16, 16), dtype=torch.float32, device="cuda")
    de = unit_diagonals(5)
    for k, dd in [((0, 1, 1, 1), de), ((5, 1, 1, 1), de), ((1, 1, 1, 1), np.array([1.0, 1.0, 2.0])),
                  ((1, 1, 1, 1), np.arange(130.0)), ((1, 1, 1, 1), np.array([-1.0, 2.0]))]:
        with pytest.raises(ps.PolyError) as ei:
            plan.trispectrum_full(d, k, dd)
        assert ei.value.status == 1  # POLY_ERR_ARG
    out = torch.empty((5, 5), dtype=torch.float64, device="cuda")
    with pytest.raises(ps.PolyError):  # T without delta
        ps.poly_trispectrum_full(plan.handle, None, (1, 1, 1, 1), de, out.data_ptr(), None, None, None)
    with pytest.raises(ps.PolyError):  # outputs alias
        ps.poly_trispectrum_full(plan.handle, d.data_ptr(), (1, 1, 1, 1), de, out.data_ptr(), out.data_ptr(), None,
                                 None)
    plan.close()
