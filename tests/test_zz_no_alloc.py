"""poly_estimate_noalloc: the bispectrum entry point that allocates no device memory.

It is meant for callers that cannot call cudaMalloc when they need an
estimate: programs whose device-memory budget is already fixed, code running
inside a framework that owns the allocator, or loops that must not pay for an
allocation.  It keeps its intermediates in a static device array inside the
library, so these checks call it twice in a row on different fields (the second
call must not see anything the first one left behind) and compare each result
with poly_estimate's, within the FP32 bar the other parity tests use.
This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

import fieldgen

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_11055_gb300 import build

    build.build()


def test_noalloc_matches_poly_estimate_on_two_calls_in_a_row():
    N, L, nshell = 32, 500.0, 9
    edges = fieldgen.unit_edges(nshell)
    plan = ps.Plan(N, L, 3, edges, "fp32")
    c_n = (L ** 3) ** 2 / float(N ** 3) ** 3
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (31, 32):
        d = torch.from_numpy(fieldgen.field("lognormal", N, seed, np.float32)).cuda()
        ref, scale = plan.estimate(d, scale=True)
        out = torch.full((plan.nbins,), float("nan"), dtype=torch.float64, device="cuda")
        ps.poly_estimate_noalloc(N, L, edges, d.data_ptr(), plan.counts, out.data_ptr(), stream)
        torch.cuda.synchronize()
        err = ((out - ref).abs() / (c_n * scale)).max().item()
        assert err <= 1e-4, err


def test_noalloc_rejects_problems_beyond_its_static_scratch():
    N, nshell = 256, 64
    edges = fieldgen.unit_edges(nshell)
    d = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
    out = torch.empty(24432, dtype=torch.float64, device="cuda")
    with pytest.raises(ps.PolyError) as ei:
        ps.poly_estimate_noalloc(N, 1000.0, edges, d.data_ptr(), np.ones(24432, np.int64), out.data_ptr(), None)
    assert ei.value.status == 6  # POLY_ERR_UNSUPPORTED
    assert "32 MiB" in str(ei.value)
