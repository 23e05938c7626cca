"""The hand-written adjoint (poly_backward) for L = sum_b w_b B_b.

Checks: against the FP64 oracle gradient (analytic adjoint, itself pinned by
central differences in test_oracle_estimator.py); against central finite
differences of the GPU estimator on 64 random voxels of a 64^3 / 16-shell
field (FP64 plain method); a full-size 256^3 / 64-shell directional derivative
(FP64 finite difference of L along a random direction vs <grad, v>, for the
FP32 adjoint and the tensor-core split-BF16 one); and
the torch.autograd wrapper.
"""
import os

import numpy as np
import pytest

import fieldgen
import oracle

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1904_11055_gb300 import build

    build.build()
    oracle.set_threads(os.cpu_count() or 1)


def gpu_grad(plan, delta, w):
    dt = torch.float64 if plan.prec == ps.POLY_FP64 else torch.float32
    d = torch.from_numpy(np.ascontiguousarray(delta)).to("cuda", dt)
    g = plan.backward(d, torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    return g.double().cpu().numpy()


@pytest.mark.parametrize("N,order,nshell,prec,tol", [(32, 3, 8, "fp64", 1e-9), (32, 3, 8, "fp32", 2e-5),
                                                     (24, 4, 5, "fp64", 1e-9), (24, 2, 9, "fp32", 2e-5),
                                                     (48, 3, 14, "split_bf16", 2e-5),
                                                     (96, 3, 30, "split_bf16", 2e-5)])
def test_gradient_matches_oracle(N, order, nshell, prec, tol):
    e = fieldgen.unit_edges(nshell)
    d = fieldgen.field("lognormal", N, 40 + N, np.float32).astype(np.float64)
    plan = ps.Plan(N, 500.0, order, e, prec)
    w = np.random.default_rng(5).standard_normal(plan.nbins)
    g = gpu_grad(plan, d, w)
    ref = oracle.gradient(d, 500.0, e, order, plan.bins, plan.counts, w)
    err = np.abs(g - ref).max() / np.abs(ref).max()
    assert err < tol, err


def test_gradient_central_differences_64cube():
    """64 random voxels of a 64^3 field, 16 unit shells, FP64 plain method on the GPU."""
    N, L = 64, 1000.0
    e = fieldgen.unit_edges(16)
    d = fieldgen.field("gaussian_cut16", N, 4, np.float64)
    plan = ps.Plan(N, L, 3, e, "fp64")
    w = np.random.default_rng(5).standard_normal(plan.nbins)
    g = gpu_grad(plan, d, w)
    dev = torch.from_numpy(d).cuda()
    wt = torch.from_numpy(w).cuda()
    vox = np.random.default_rng(6).choice(N ** 3, size=64, replace=False)
    h = 1e-3 * float(d.std())
    flat = dev.view(-1)
    for v in vox:
        flat[v] += h
        lp = float(torch.dot(plan.estimate(dev), wt))
        flat[v] -= 2 * h
        lm = float(torch.dot(plan.estimate(dev), wt))
        flat[v] += h
        fd = (lp - lm) / (2 * h)
        gv = g.reshape(-1)[v]
        assert abs(fd - gv) <= 1e-6 * np.abs(g).max(), (v, fd, gv)


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_gradient_directional_derivative_full_size(prec):
    """256^3 lognormal, 64 unit shells: <grad, v> from the FP32 / split-BF16 adjoint vs an FP64 central difference."""
    N, L = 256, 1000.0
    e = fieldgen.unit_edges(64)
    d = fieldgen.field("lognormal", N, 4, np.float32)
    p32 = ps.Plan(N, L, 3, e, prec)
    w = np.random.default_rng(5).standard_normal(p32.nbins)
    g = gpu_grad(p32, d.astype(np.float64), w)
    p32.close()
    v = np.random.default_rng(6).standard_normal((N, N, N))
    dirderiv = float(np.sum(g * v))
    p64 = ps.Plan(N, L, 3, e, "fp64")
    wt = torch.from_numpy(w).cuda()
    h = 1e-3
    base = torch.from_numpy(d.astype(np.float64)).cuda()
    vt = torch.from_numpy(v).cuda()
    lp = float(torch.dot(p64.estimate((base + h * vt).contiguous()), wt))
    lm = float(torch.dot(p64.estimate((base - h * vt).contiguous()), wt))
    fd = (lp - lm) / (2 * h)
    assert abs(fd - dirderiv) <= 1e-4 * abs(fd), (fd, dirderiv)


def test_autograd_function_uses_the_adjoint():
    N, e = 32, fieldgen.unit_edges(8)
    plan = ps.Plan(N, 500.0, 3, e, "fp32")
    d = torch.from_numpy(fieldgen.field("lognormal", N, 9, np.float32)).cuda().requires_grad_(True)
    w = torch.from_numpy(np.random.default_rng(3).standard_normal(plan.nbins)).cuda()
    B = ps.polyspectrum(d, plan)
    (B * w).sum().backward()
    g_direct = plan.backward(d.detach(), w)
    assert torch.equal(d.grad, g_direct)
