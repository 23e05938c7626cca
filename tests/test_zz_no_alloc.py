"""poly_estimate_noalloc: the bispectrum entry point that allocates no device memory.

It is meant for callers that cannot call cudaMalloc when they need an
estimate: programs whose device-memory budget is already fixed, or code
running inside a framework that owns the device allocator.  It keeps its
intermediates in a static device array inside the library, so these checks
call it several times in a row, on different fields and on problems whose
intermediates are laid out differently in that array (a later call must not
see anything an earlier one left behind), and compare each result with
poly_estimate's and with the FP64 oracle, within the FP32 bar the other parity
tests use.  They also check that a call leaves the device's free memory
unchanged.  This file is collected last so that a failure here never hides
another test.
"""
import numpy as np
import pytest

import fieldgen
import oracle

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4  # |B - B_ref| <= 1e-4 * c_n * sum_x |prod D| / (N^3 count), as for the plain FP32 path


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_11055_gb300 import build

    build.build()


def _noalloc(N, L, edges, d, counts, nbins):
    out = torch.full((nbins,), float("nan"), dtype=torch.float64, device="cuda")
    ps.poly_estimate_noalloc(N, L, edges, d.data_ptr(), counts, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_poly_estimate_on_calls_in_a_row():
    """Two fields on one layout, then a grid and shell set with another layout of the static array,
    then the first layout again."""
    cases = [(32, 500.0, 9, 31), (32, 500.0, 9, 32), (48, 700.0, 14, 33), (32, 500.0, 9, 34)]
    for N, L, nshell, seed in cases:
        edges = fieldgen.unit_edges(nshell)
        plan = ps.Plan(N, L, 3, edges, "fp32")
        c_n = (L ** 3) ** 2 / float(N ** 3) ** 3
        d = torch.from_numpy(fieldgen.field("lognormal", N, seed, np.float32)).cuda()
        ref, scale = plan.estimate(d, scale=True)
        out = _noalloc(N, L, edges, d, plan.counts, plan.nbins)
        err = ((out - ref).abs() / (c_n * scale)).max().item()
        assert err <= TOL_FP32, (N, nshell, seed, err)
        plan.close()


def test_noalloc_matches_the_oracle():
    N, L, nshell = 32, 500.0, 9
    edges = fieldgen.unit_edges(nshell)
    delta = fieldgen.field("lognormal", N, 35, np.float32)
    bins = oracle.enumerate_bins(edges, 3)
    ref = oracle.estimate(delta.astype(np.float64), L, edges, 3, bins=bins)
    out = _noalloc(N, L, edges, torch.from_numpy(delta).cuda(), ref["counts"], len(bins)).cpu().numpy()
    c_n = (L ** 3) ** 2 / float(N ** 3) ** 3
    err = np.max(np.abs(out - ref["B"]) / (c_n * ref["scale"]))
    assert err <= TOL_FP32, err


def test_noalloc_leaves_free_device_memory_unchanged():
    """After a first call (which looks up the static array's address), a further call changes the
    device's free memory by nothing: no allocation, by the library or by anything it calls."""
    N, L, nshell = 32, 500.0, 9
    edges = fieldgen.unit_edges(nshell)
    plan = ps.Plan(N, L, 3, edges, "fp32")
    counts, nbins = plan.counts.copy(), plan.nbins
    plan.close()
    d = torch.from_numpy(fieldgen.field("lognormal", N, 36, np.float32)).cuda()
    out = torch.empty(nbins, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ps.poly_estimate_noalloc(N, L, edges, d.data_ptr(), counts, out.data_ptr(), stream)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ps.poly_estimate_noalloc(N, L, edges, d.data_ptr(), counts, out.data_ptr(), stream)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)
    assert torch.isfinite(out).all()


def test_noalloc_rejects_problems_beyond_its_static_scratch():
    N, nshell = 256, 64
    edges = fieldgen.unit_edges(nshell)
    d = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
    out = torch.empty(24432, dtype=torch.float64, device="cuda")
    with pytest.raises(ps.PolyError) as ei:
        ps.poly_estimate_noalloc(N, 1000.0, edges, d.data_ptr(), np.ones(24432, np.int64), out.data_ptr(), None)
    assert ei.value.status == 6  # POLY_ERR_UNSUPPORTED
    assert "32 MiB" in str(ei.value)


def test_noalloc_wrapper_checks_the_counts_length():
    N, nshell = 32, 9
    edges = fieldgen.unit_edges(nshell)
    d = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ps.poly_estimate_noalloc(N, 500.0, edges, d.data_ptr(), np.ones(8, np.int64), out.data_ptr(), None)
