"""The tcgen05 building block of the split-BF16 contraction, checked exactly.

poly_diag_tc_gemm runs one MMA step the way the contraction does (A in tensor
memory via tcgen05.st, B in shared memory in the K-major core-matrix layout,
FP32 accumulation).  With small integer inputs every product and partial sum is
exact in FP32, so the result must equal numpy's integer matrix product bit for
bit.  On failure the message names the first of a few plausible layout
mistakes that would explain the output.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu


def bf16_bits(x):
    """bf16 bit patterns of float32 values that bf16 represents exactly."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32)
    assert np.all((u & 0xFFFF) == 0)
    return (u >> 16).astype(np.uint16)


def run_gemm(A, B):
    from paper_1904_11055_gb300 import build

    build.build()
    lib = ps.load_library()
    lib.poly_diag_tc_gemm.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.poly_diag_tc_gemm.restype = ctypes.c_int
    N = B.shape[0]
    a = np.ascontiguousarray(bf16_bits(A))
    b = np.ascontiguousarray(bf16_bits(B))
    D = np.zeros((128, N), dtype=np.float32)
    rc = lib.poly_diag_tc_gemm(a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p), N,
                               D.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0, f"poly_diag_tc_gemm returned {rc}"
    return D


def explain(D, A, B):
    cands = {
        "A pairs swapped within a 32-bit column": A.reshape(128, 16, 2)[:, :, ::-1].reshape(128, 32),
        "B core matrices transposed (LBO/SBO swapped)": None,
        "only the first K16 step accumulated": np.concatenate([A[:, :16], np.zeros((128, 16), np.float32)], 1),
    }
    for name, Ax in cands.items():
        if Ax is not None and np.array_equal(D, Ax @ B.T):
            return name
    return "no candidate matches"


@pytest.mark.parametrize("N", [16, 48, 64, 256])
def test_tcgen05_gemm_layout_exact(N):
    rng = np.random.default_rng(N)
    A = rng.integers(-8, 9, size=(128, 32)).astype(np.float32)
    B = rng.integers(-8, 9, size=(N, 32)).astype(np.float32)
    D = run_gemm(A, B)
    ref = A @ B.T
    if not np.array_equal(D, ref):
        pytest.fail(f"tcgen05 GEMM differs from A @ B^T ({explain(D, A, B)}); "
                    f"max |diff| = {np.abs(D - ref).max()}")


def test_tcgen05_gemm_distinguishes_every_element():
    """Powers of two place each (row, k) and (col, k) contribution in its own bit."""
    A = np.zeros((128, 32), np.float32)
    B = np.zeros((64, 32), np.float32)
    A[np.arange(128), np.arange(128) % 32] = 1.0
    B[np.arange(64), np.arange(64) % 32] = 2.0 ** (np.arange(64) % 8)
    D = run_gemm(A, B)
    assert np.array_equal(D, A @ B.T)


def test_bounded_wait_gives_up_on_a_stalled_producer():
    """A wait on a barrier that nothing arrives on (a stalled producer) ends with POLY_ERR_TIMEOUT after the
    clock budget, through the pipelines' own bounded wait, and leaves the context usable."""
    from paper_1904_11055_gb300 import build

    build.build()
    import fieldgen

    lib = ps.load_library()
    lib.poly_diag_stalled_wait.argtypes = [ctypes.c_void_p]
    lib.poly_diag_stalled_wait.restype = ctypes.c_int
    ms = ctypes.c_double()
    assert lib.poly_diag_stalled_wait(ctypes.byref(ms)) == 5  # POLY_ERR_TIMEOUT
    assert 300.0 < ms.value < 30000.0, ms.value
    plan = ps.Plan(16, 100.0, 3, fieldgen.unit_edges(4), "split_bf16")
    d = torch.from_numpy(fieldgen.field("lognormal", 16, 1, np.float32)).cuda()
    B = plan.estimate(d)
    torch.cuda.synchronize()
    assert torch.isfinite(B).all()
