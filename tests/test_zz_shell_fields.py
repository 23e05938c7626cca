"""The shell fields themselves, not only the estimates built from them.

poly_diag_fields runs the library's forward transform and shell-field stage
(Sec. 2, Eq. Bkfast, App. A: D_s(x) = sum over the modes q of shell s of
delta_hat(q) e^{+i q.x}, no 1/N^3) exactly as poly_estimate
does, and hands the fields back in natural [slot][x][y][z] order.  They are
compared point by point with the oracle's fields and with cuFFT (torch.fft,
FP64) applied to the same masked spectrum.  A shell fed with the wrong modes,
a sign flip of the exponent or a mis-tiled slot shows up here as an O(1)
error; the tolerances are the transforms' rounding (single-precision FFTs of
this size reach a few 1e-7 of each shell's peak).
This file is collected last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

import fieldgen
import oracle

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_11055_gb300 import build

    build.build()


def library_fields(plan, d):
    lib = ps.load_library()
    lib.poly_diag_fields.argtypes = [ctypes.c_void_p] * 4
    lib.poly_diag_fields.restype = ctypes.c_int
    nf = (2 if plan.ell else 1) * (len(plan.edges) - 1)
    out = np.empty((nf, plan.N, plan.N, plan.N), dtype=np.float64 if plan.prec == ps.POLY_FP64 else np.float32)
    rc = lib.poly_diag_fields(plan.handle, d.data_ptr(), out.ctypes.data, torch.cuda.current_stream().cuda_stream)
    assert rc == 0, f"poly_diag_fields returned {rc}"
    return out.astype(np.float64)


def grid_q2(N):
    f = torch.fft.fftfreq(N, d=1.0 / N, device="cuda", dtype=torch.float64)
    return f, f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2


def shell_mask(q2, edges, s):
    """Modes of shell s: edges[s]^2 <= |q|^2 < edges[s+1]^2, q = 0 excluded (Sec. 2)."""
    return (q2 >= float(edges[s]) ** 2) & (q2 < float(edges[s + 1]) ** 2) & (q2 > 0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_shell_fields_match_the_oracle_and_cufft(prec, tol):
    """48^3 lognormal field, 12 unit shells: every field against the oracle, three against cuFFT."""
    N, e = 48, fieldgen.unit_edges(12)
    d64 = fieldgen.field("lognormal", N, 23, np.float32).astype(np.float64)
    plan = ps.Plan(N, 1000.0, 3, e, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    got = library_fields(plan, torch.from_numpy(d64).to("cuda", dt))
    assert got.shape == (12, N, N, N)
    ref, _ = oracle.shell_fields(N, e, np.arange(12), oracle.forward(d64))
    peak = np.abs(ref).max(axis=(1, 2, 3))
    err = np.abs(got - ref).max(axis=(1, 2, 3))
    assert np.all(err <= tol * peak), f"worst field error / peak {np.max(err / peak):.3e}"
    F = torch.fft.fftn(torch.from_numpy(d64).cuda())
    _, q2 = grid_q2(N)
    for s in (0, 5, 11):
        cu = torch.fft.ifftn(F * shell_mask(q2, e, s), norm="forward").real.cpu().numpy()
        assert np.abs(got[s] - cu).max() <= tol * peak[s]


def test_multipole_fields_are_the_legendre_weighted_transforms():
    """A quadrupole plan (ell = 2, line of sight along the last axis): slots 0..5 hold the plain fields and
    slots 6..11 the transforms of L_2(q_z/|q|) delta_hat(q), both against cuFFT in FP64."""
    N, e = 32, fieldgen.unit_edges(6)
    d64 = fieldgen.field("lognormal", N, 24, np.float32).astype(np.float64)
    plan = ps.Plan(N, 1000.0, 3, e, "fp64", ell=2)
    got = library_fields(plan, torch.from_numpy(d64).cuda())
    assert got.shape[0] == 12
    F = torch.fft.fftn(torch.from_numpy(d64).cuda())
    f, q2 = grid_q2(N)
    mu2 = f[None, None, :] ** 2 / torch.clamp(q2, min=1.0)
    L2 = 1.5 * mu2 - 0.5
    for s in range(6):
        m = shell_mask(q2, e, s)
        plain = torch.fft.ifftn(F * m, norm="forward").real.cpu().numpy()
        weighted = torch.fft.ifftn(F * L2 * m, norm="forward").real.cpu().numpy()
        assert np.abs(got[s] - plain).max() <= 1e-10 * np.abs(plain).max()
        assert np.abs(got[6 + s] - weighted).max() <= 1e-10 * np.abs(weighted).max()
