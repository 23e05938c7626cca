"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Error measure (the stated tolerance bound, same physical prefactor on
both sides): err_b = |B_gpu - B_ref| / (c_n * scale_ref_b) with
scale_ref_b = sum_x |prod D| / (N^3 count_b) from the oracle and
c_n = V^{n-1} / N^{3n}.  Bars: 1e-4 for the plain FP32 path, 1e-5 for the
split-BF16 tensor-core path, 1e-10 for the FP64 plain method; counts bit-exact.
"""
import os

import numpy as np
import pytest

import fieldgen
import oracle

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {"fp32": 1e-4, "split_bf16": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1904_11055_gb300 import build

    build.build()
    oracle.set_threads(os.cpu_count() or 1)


def norm(L, N, n):
    return (L ** 3) ** (n - 1) / float(N ** 3) ** n


def gpu_estimate(delta, L, edges, order, prec, flags=0, bins=None):
    N = delta.shape[0]
    plan = ps.Plan(N, L, order, edges, prec, flags)
    dt = torch.float64 if prec == "fp64" else torch.float32
    d = torch.from_numpy(np.ascontiguousarray(delta)).to("cuda", dt)
    B = plan.estimate(d)
    plan.sync()  # a device-side timeout raises here instead of returning partial sums
    return plan, B.cpu().numpy()


def check_against_oracle(delta, L, edges, order, prec, sample=None, flags=0):
    N = delta.shape[0]
    plan, B = gpu_estimate(delta, L, edges, order, prec, flags)
    idx = np.arange(plan.nbins) if sample is None else np.asarray(sample)
    ref = oracle.estimate(np.asarray(delta, dtype=np.float64), L, edges, order, bins=plan.bins[idx])
    assert np.array_equal(plan.counts[idx], ref["counts"]), "counts differ from the oracle"
    with np.errstate(invalid="ignore", divide="ignore"):  # bins with no polygon have no scale (0 / 0)
        err = np.abs(B[idx] - ref["B"]) / (norm(L, N, order) * ref["scale"])
    return plan, B, ref, err


# ------------------------------------------------------------------ counts
def test_counts_match_golden_enumeration():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "counts_n3_N16_unit6.txt")) if not ln.startswith("#")]
    g = np.array([[int(v) for v in r] for r in rows if r], dtype=np.int64)
    plan = ps.Plan(16, 1.0, 3, fieldgen.unit_edges(6), "fp32", ps.POLY_BINS_ALL_SORTED | ps.POLY_ALLOW_ALIAS)
    assert np.array_equal(plan.bins, g[:, :3])
    assert np.array_equal(plan.counts, g[:, 3])


def read_golden_counts(name):
    rows = np.loadtxt(os.path.join(GOLDEN, name), dtype=np.int64, comments="#")
    return rows[:, :-1].astype(np.int32), rows[:, -1]


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_counts_of_the_256cube_benchmark_plan_match_the_golden_file(prec):
    """Every one of the 24,432 triangle counts of the 256^3 / 64-shell plan, bit for bit, against the
    oracle's exact pair-convolution counts (tests/golden/counts_n3_64shells.txt)."""
    bins, counts = read_golden_counts("counts_n3_64shells.txt")
    plan = ps.Plan(256, 1000.0, 3, fieldgen.unit_edges(64), prec)
    assert plan.nbins == len(counts) == 24432
    assert np.array_equal(plan.bins, bins)
    assert np.array_equal(plan.counts, counts)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
@pytest.mark.parametrize("N,order,nshell,seed", [(48, 3, 12, 51), (32, 4, 7, 52)])
def test_all_sorted_bins_match_oracle(prec, N, order, nshell, seed):
    """POLY_BINS_ALL_SORTED: every sorted tuple (Sec. 4.2 order), including those outside the polygon
    rule; bins with no closed polygon have count 0 and must come out as exactly 0."""
    e = fieldgen.unit_edges(nshell)
    delta = fieldgen.field("lognormal", N, seed, np.float32)
    plan, B, ref, err = check_against_oracle(delta, 1000.0, e, order, prec, flags=ps.POLY_BINS_ALL_SORTED)
    assert np.array_equal(plan.bins, oracle.enumerate_bins(e, order, oracle.RULE_ALL_SORTED))
    zero = ref["counts"] == 0
    assert zero.any() and (~zero).any()
    assert np.all(B[zero] == 0.0) and np.all(ref["B"][zero] == 0.0)
    assert err[~zero].max() <= TOL[prec], err[~zero].max()


@pytest.mark.parametrize("N,order,nshell,width,flags", [(32, 3, 10, 1.0, 0), (48, 3, 10, 1.5, 0), (32, 4, 7, 1.0, 0),
                                                        (24, 2, 11, 1.0, 1), (64, 3, 16, 1.0, 0),
                                                        (96, 3, 32, 1.0, 2)])
def test_counts_bit_exact(N, order, nshell, width, flags):
    e = fieldgen.unit_edges(nshell, width)
    plan = ps.Plan(N, 1.0, order, e, "fp32", flags)
    ref = oracle.estimate(np.zeros((N, N, N)), 1.0, e, order, bins=plan.bins)
    assert np.array_equal(plan.bins, oracle.enumerate_bins(e, order, flags & 1))
    assert np.array_equal(plan.counts, ref["counts"])


# ------------------------------------------------------------------ the plain FP64 method (64^3 Gaussian, 16 shells)
def test_fp64_plain_method_64cube():
    d = fieldgen.field("gaussian_cut16", 64, 1, np.float64)
    plan, B, ref, err = check_against_oracle(d, 1000.0, fieldgen.unit_edges(16), 3, "fp64")
    assert plan.nbins == 508
    assert err.max() <= TOL["fp64"], err.max()


# ------------------------------------------------------------------ FP32 path, several tiles and ragged tails
CASES = [(48, 3, 12, "lognormal", 7), (32, 4, 7, "lognormal", 8), (24, 2, 11, "gaussian", 9),
         (64, 3, 16, "gaussian_cut16", 1), (16, 3, 4, "white", 10), (96, 3, 20, "lognormal", 11),
         (48, 4, 11, "lognormal", 13)]


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
@pytest.mark.parametrize("N,order,nshell,kind,seed", CASES)
def test_matches_oracle(prec, N, order, nshell, kind, seed):
    d = fieldgen.field(kind, N, seed, np.float32).astype(np.float64)
    _, _, _, err = check_against_oracle(d, 1000.0, fieldgen.unit_edges(nshell), order, prec)
    assert err.max() <= TOL[prec], err.max()


# ------------------------------------------------------------------ orders 5 and 6 (CUDA-core path: pairs or
# triples of fields against triples)
@pytest.mark.parametrize("prec", ["fp32", "fp64", "split_bf16"])
@pytest.mark.parametrize("N,order,nshell,seed", [(32, 5, 5, 21), (48, 6, 6, 22), (48, 5, 8, 23)])
def test_higher_orders_match_oracle(prec, N, order, nshell, seed):
    d = fieldgen.field("lognormal", N, seed, np.float32).astype(np.float64)
    plan, _, _, err = check_against_oracle(d, 1000.0, fieldgen.unit_edges(nshell), order, prec)
    assert plan.nbins > 50
    assert err.max() <= TOL[prec], err.max()


# ------------------------------------------------------------------ disconnected part of the trispectrum
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("split_bf16", 1e-5)])
@pytest.mark.parametrize("N,nshell,width,seed", [(32, 7, 1.0, 31), (48, 7, 1.5, 32)])
def test_disconnected_trispectrum_matches_oracle(prec, tol, N, nshell, width, seed):
    e = fieldgen.unit_edges(nshell, width)
    d64 = fieldgen.field("lognormal", N, seed, np.float32).astype(np.float64)
    plan = ps.Plan(N, 1000.0, 4, e, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    d = torch.from_numpy(d64).to("cuda", dt)
    Bd, P = plan.disconnected(d, power=True)
    torch.cuda.synchronize()
    ref, Pref = oracle.disconnected(d64, 1000.0, e, plan.bins, plan.counts)
    assert np.allclose(P.cpu().numpy(), Pref, rtol=tol, atol=0.0)
    got = Bd.cpu().numpy()
    assert np.array_equal(got == 0.0, ref == 0.0)
    nz = ref != 0.0
    assert nz.sum() >= nshell
    assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) <= 2 * tol


def test_disconnected_part_is_refused_below_order_4():
    plan = ps.Plan(32, 1000.0, 3, fieldgen.unit_edges(6), "fp32")
    d = torch.from_numpy(fieldgen.field("lognormal", 32, 3, np.float32)).cuda()
    with pytest.raises(ps.PolyError) as ei:
        plan.disconnected(d)
    assert ei.value.status == 6


# ------------------------------------------------------------------ redshift-space multipoles (first leg L_ell)
@pytest.mark.parametrize("prec", ["fp32", "fp64", "split_bf16"])
@pytest.mark.parametrize("N,order,nshell,ell,seed", [(32, 3, 8, 2, 41), (48, 3, 12, 4, 42), (32, 4, 6, 2, 43)])
def test_multipoles_match_oracle(prec, N, order, nshell, ell, seed):
    e = fieldgen.unit_edges(nshell)
    d64 = fieldgen.field("lognormal", N, seed, np.float32).astype(np.float64)
    plan = ps.Plan(N, 1000.0, order, e, prec, ell=ell)
    dt = torch.float64 if prec == "fp64" else torch.float32
    B = plan.estimate(torch.from_numpy(d64).to("cuda", dt)).cpu().numpy()
    ref = oracle.estimate_ell(d64, 1000.0, e, order, ell, plan.bins)
    assert np.array_equal(plan.counts, ref["counts"])
    err = np.abs(B - ref["B"]) / ((2 * ell + 1) * norm(1000.0, N, order) * ref["scale"])
    assert err.max() <= TOL[prec], err.max()
    assert np.abs(ref["B"]).max() > 0


def test_multipole_zero_is_the_plain_plan_and_refuses_the_adjoint():
    e = fieldgen.unit_edges(6)
    d = torch.from_numpy(fieldgen.field("lognormal", 32, 5, np.float32)).cuda()
    plain, m0 = ps.Plan(32, 1000.0, 3, e, "fp32"), ps.Plan(32, 1000.0, 3, e, "fp32", ell=0)
    assert torch.equal(plain.estimate(d), m0.estimate(d))
    m2 = ps.Plan(32, 1000.0, 3, e, "fp32", ell=2)
    with pytest.raises(ps.PolyError) as ei:
        m2.backward(d, torch.ones(m2.nbins, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 6


def test_higher_orders_refuse_the_adjoint():
    """No order above 4 has an adjoint."""
    e = fieldgen.unit_edges(4)
    plan = ps.Plan(32, 1000.0, 5, e, "fp32")
    d = torch.from_numpy(fieldgen.field("lognormal", 32, 3, np.float32)).cuda()
    with pytest.raises(ps.PolyError) as ei:
        plan.backward(d, torch.ones(plan.nbins, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 6


# every contraction shape poly_plan_set_config accepts: M tiles per group 1..4, CTA budget 1/2..4 x the SMs
TC_SHAPES = [mt | (mult << 4) for mt in (1, 2, 3, 4) for mult in (1, 2, 4, 6, 8)]


@pytest.mark.parametrize("N,order,nshell,width,seed,sample", [
    (128, 3, 40, 1.0, 81, {40, 39, 27, 26, 20, 13, 7, 2}),  # 1 to 4 groups; two producer teams at 4 M tiles
    (48, 4, 7, 1.5, 82, None),
])
def test_every_contraction_shape_matches_oracle(N, order, nshell, width, seed, sample):
    """The tuner's shapes change the groups, their A/B slots, the producer team count (two or three) and the
    CTA split of the chunks; every one of them gives the oracle's B within the split-BF16 bar (on the bins
    among the sampled shells where given)."""
    L = 700.0
    e = fieldgen.unit_edges(nshell, width)
    bins = oracle.enumerate_bins(e, order)
    idx = np.arange(len(bins)) if sample is None else np.array(
        [i for i, b in enumerate(bins) if set(b.tolist()) <= sample])
    delta = fieldgen.field("lognormal", N, seed, np.float32)
    ref = oracle.estimate(delta.astype(np.float64), L, e, order, bins=bins[idx])
    plan = ps.Plan(N, L, order, e, "split_bf16")
    assert np.array_equal(plan.bins[idx], bins[idx])
    d = torch.from_numpy(delta).cuda()
    live = ref["counts"] > 0
    for code in TC_SHAPES:
        plan.set_config(code)
        B = plan.estimate(d).cpu().numpy()[idx]
        plan.sync()
        err = np.abs(B[live] - ref["B"][live]) / (norm(L, N, order) * ref["scale"][live])
        assert err.max() <= TOL["split_bf16"], (hex(code), err.max())
    plan.close()


@pytest.fixture(scope="module")
def field256():
    return fieldgen.field("lognormal", 256, 2, np.float32)


@pytest.fixture(scope="module")
def oracle256(field256):
    """Oracle on the bins among ten shells of the 256^3, 64-shell workload."""
    e = fieldgen.unit_edges(64)
    bins = oracle.enumerate_bins(e, 3)
    shells = {64, 63, 41, 40, 33, 32, 31, 17, 9, 2}
    idx = np.array([i for i, b in enumerate(bins) if set(b.tolist()) <= shells])
    return idx, oracle.estimate(field256.astype(np.float64), 1000.0, e, 3, bins=bins[idx])


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_full_size_256cube_sampled(prec, field256, oracle256):
    """256^3 lognormal, 64 unit shells (24,432 triangles), the configuration bench.py times."""
    e = fieldgen.unit_edges(64)
    plan, B = gpu_estimate(field256, 1000.0, e, 3, prec)
    assert plan.nbins == 24432
    idx, ref = oracle256
    assert len(idx) >= 30
    assert np.array_equal(plan.counts[idx], ref["counts"])
    err = np.abs(B[idx] - ref["B"]) / (norm(1000.0, 256, 3) * ref["scale"])
    assert err.max() <= TOL[prec], err.max()


@pytest.fixture(scope="module")
def oracle256_n4(field256):
    """Oracle on the quadrilaterals among six shells of the 256^3 trispectrum workload (32 x 1.5 k_F)."""
    e = fieldgen.unit_edges(32, 1.5)
    bins = oracle.enumerate_bins(e, 4)
    shells = {32, 31, 22, 13, 6, 1}
    idx = np.array([i for i, b in enumerate(bins) if set(b.tolist()) <= shells])
    return idx, oracle.estimate(field256.astype(np.float64), 1000.0, e, 4, bins=bins[idx])


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_full_size_trispectrum_256cube_sampled(prec, field256, oracle256_n4):
    """256^3 lognormal, 32 shells of width 1.5 k_F (45,135 quadrilaterals): the Gram of pair products."""
    e = fieldgen.unit_edges(32, 1.5)
    plan, B = gpu_estimate(field256, 1000.0, e, 4, prec)
    assert plan.nbins == 45135
    idx, ref = oracle256_n4
    assert len(idx) >= 30
    assert np.array_equal(plan.counts[idx], ref["counts"])
    err = np.abs(B[idx] - ref["B"]) / (norm(1000.0, 256, 4) * ref["scale"])
    assert err.max() <= TOL[prec], err.max()


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_order5_128cube_sampled(prec):
    """n = 5 at the size bench.py measures it (128^3, 16 unit shells, 15,056 bins), FP32 and split-BF16, on the
    bins among five shells; counts bit-exact."""
    e = fieldgen.unit_edges(16)
    d = fieldgen.field("lognormal", 128, 2, np.float32)
    plan, B = gpu_estimate(d, 1000.0, e, 5, prec)
    assert plan.nbins == 15056
    shells = {16, 15, 9, 4, 1}
    idx = np.array([i for i, b in enumerate(plan.bins) if set(b.tolist()) <= shells])
    assert len(idx) >= 30
    ref = oracle.estimate(d.astype(np.float64), 1000.0, e, 5, bins=plan.bins[idx])
    assert np.array_equal(plan.counts[idx], ref["counts"])
    err = np.abs(B[idx] - ref["B"]) / (norm(1000.0, 128, 5) * ref["scale"])
    assert err.max() <= TOL[prec], err.max()


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_quadrupole_256cube_sampled(prec, field256):
    """ell = 2 multipole bispectrum at 256^3 with 64 unit shells (the size bench.py measures), FP32 and
    split-BF16, on the triangles among five shells."""
    e = fieldgen.unit_edges(64)
    plan = ps.Plan(256, 1000.0, 3, e, prec, ell=2)
    B = plan.estimate(torch.from_numpy(field256).cuda()).cpu().numpy()
    shells = {64, 40, 33, 17, 2}
    idx = np.array([i for i, b in enumerate(plan.bins) if set(b.tolist()) <= shells])
    assert len(idx) >= 10
    ref = oracle.estimate_ell(field256.astype(np.float64), 1000.0, e, 3, 2, plan.bins[idx])
    assert np.array_equal(plan.counts[idx], ref["counts"])
    err = np.abs(B[idx] - ref["B"]) / (5 * norm(1000.0, 256, 3) * ref["scale"])
    assert err.max() <= TOL[prec], err.max()


def test_matches_an_independent_cufft_route():
    """The estimate against the same estimator built from cuFFT shell fields (torch.fft) and plain torch
    reductions: an independent GPU route, FP64 throughout, 48^3 and 10 shells."""
    N, L, e = 48, 1000.0, fieldgen.unit_edges(10)
    d = fieldgen.field("lognormal", N, 17, np.float32)
    plan = ps.Plan(N, L, 3, e, "fp32")
    B = plan.estimate(torch.from_numpy(d).cuda()).cpu().numpy()
    dt = torch.from_numpy(d.astype(np.float64)).cuda()
    f = torch.fft.fftfreq(N, d=1.0 / N, device="cuda", dtype=torch.float64)
    fz = torch.fft.rfftfreq(N, d=1.0 / N, device="cuda", dtype=torch.float64)
    q2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2
    F = torch.fft.rfftn(dt)
    D = []
    for s in range(10):
        m = (q2 >= e[s] ** 2) & (q2 < e[s + 1] ** 2) & (q2 > 0)
        D.append(torch.fft.irfftn(torch.where(m, F, 0), s=(N, N, N), norm="forward").reshape(-1))
    D = torch.stack(D)
    b = torch.from_numpy(plan.bins.astype(np.int64) - 1).cuda()
    S = (D[b[:, 0]] * D[b[:, 1]] * D[b[:, 2]]).sum(dim=1)
    A = (D[b[:, 0]] * D[b[:, 1]] * D[b[:, 2]]).abs().sum(dim=1)
    cnt = torch.from_numpy(plan.counts).cuda().double()
    ref = (norm(L, N, 3) * S / (N ** 3 * cnt)).cpu().numpy()
    scale = (A / (N ** 3 * cnt)).cpu().numpy()
    err = np.abs(B - ref) / (norm(L, N, 3) * scale)
    assert err.max() <= TOL["fp32"], err.max()


# ------------------------------------------------------------------ entry points agree bit for bit
def test_host_entry_matches_device_entry():
    d = fieldgen.field("lognormal", 32, 5, np.float32)
    plan, B = gpu_estimate(d, 500.0, fieldgen.unit_edges(10), 3, "fp32")
    Bh = plan.estimate_host(d)
    assert np.array_equal(B, Bh)


def test_batched_matches_single_calls():
    cases = [(32, 8, 21), (48, 12, 22), (32, 8, 23), (24, 7, 24)]
    plans, fields, singles = [], [], []
    for N, ns, seed in cases:
        p = ps.Plan(N, 500.0, 3, fieldgen.unit_edges(ns), "fp32")
        f = torch.from_numpy(fieldgen.field("lognormal", N, seed, np.float32)).cuda()
        plans.append(p)
        fields.append(f)
        singles.append(p.estimate(f).cpu().numpy())
    outs = ps.estimate_batched(plans, fields)
    torch.cuda.synchronize()
    for o, s in zip(outs, singles):
        assert np.array_equal(o.cpu().numpy(), s)


def test_scale_output_matches_oracle_scale():
    d = fieldgen.field("lognormal", 32, 12, np.float32).astype(np.float64)
    e = fieldgen.unit_edges(9)
    plan = ps.Plan(32, 1000.0, 3, e, "fp32")
    B, sc = plan.estimate(torch.from_numpy(d).to("cuda", torch.float32), scale=True)
    ref = oracle.estimate(d, 1000.0, e, 3, bins=plan.bins)
    assert np.allclose(sc.cpu().numpy(), ref["scale"], rtol=1e-5, atol=0)


# ------------------------------------------------------------------ robustness on the host side
@pytest.mark.parametrize("k", [1, 2, 5, 9, 14])
def test_allocation_failure_is_reported_and_cleaned_up(k):
    e = fieldgen.unit_edges(8)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ps.poly_debug_fail_alloc_after(k)
    try:
        with pytest.raises(ps.PolyError) as ei:
            ps.Plan(32, 100.0, 3, e, "fp32")
        assert ei.value.status == 3
    finally:
        ps.poly_debug_fail_alloc_after(0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 8 << 20
