"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every entry point include/polyspec.h declares, and validates arguments
before it touches the device."""
import os
import re

import numpy as np
import pytest

import paper_1904_11055_gb300 as ps
from paper_1904_11055_gb300 import build as psbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    psbuild.build()
    return ps.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "polyspec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(poly_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_symbols() == sorted(ps.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    diag = open(os.path.join(ROOT, "include", "polyspec_diag.h")).read()
    diag = re.sub(r"/\*.*?\*/", "", diag, flags=re.S)
    for name in set(re.findall(r"\b(poly_diag_[a-z_0-9]+)\s*\(", diag)):
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(8):
        assert ps.poly_status_string(code) != "unknown status"
    assert ps.poly_status_string(99) == "unknown status"


@pytest.mark.parametrize("kwargs,status", [
    (dict(N=64, order=7), 6),                                          # order outside [2, 6]
    (dict(N=64, order=6, edges=np.arange(12) + 0.5), 2),                # 6 * 11 >= 64: aliasing
    (dict(N=50), 6),                                                   # N not supported
    (dict(N=64, edges=[0.5, 1.5, 1.5]), 1),                            # edges not increasing
    (dict(N=64, edges=[-1.0, 1.5]), 1),                                # negative edge
    (dict(N=32, edges=np.arange(18) + 0.5), 1),                        # beyond Nyquist (2K+1 > N)
    (dict(N=64, edges=np.arange(23) + 0.5), 2),                        # 3 * 22 >= 64: aliasing
    (dict(N=64, L=-1.0), 1),                                           # bad box size
    (dict(N=64, prec=2), 6),                                           # TF32x3 not implemented
    (dict(N=256, order=5, edges=np.arange(121) + 0.5, flags=2), 6),    # C(124, 5) > 2^26 sorted tuples
    (dict(N=256, order=6, edges=np.arange(61) + 0.5, flags=2), 6),     # C(65, 6) > 2^26 sorted tuples
])
def test_argument_validation_before_device(lib, kwargs, status):
    args = dict(N=64, L=1000.0, order=3, edges=np.arange(17) + 0.5, prec=0, flags=0)
    args.update(kwargs)
    with pytest.raises(ps.PolyError) as ei:
        ps.poly_plan_create(args["N"], args["L"], args["order"], args["edges"], args["prec"], args["flags"])
    assert ei.value.status == status


@pytest.mark.parametrize("ell,prec,order,status", [(1, 0, 3, 1), (10, 0, 3, 1), (-2, 3, 3, 1), (3, 1, 3, 1)])
def test_multipole_plans_validate_ell_and_precision(lib, ell, prec, order, status):
    """Bad ell is an argument error, in every precision."""
    with pytest.raises(ps.PolyError) as ei:
        ps.poly_plan_create_multipole(64, 1000.0, order, np.arange(17) + 0.5, prec, 0, ell)
    assert ei.value.status == status


def test_plan_create_without_device_fails_cleanly(lib):
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(ps.PolyError) as ei:
        ps.poly_plan_create(32, 100.0, 3, np.arange(9) + 0.5)
    assert ei.value.status == 4  # POLY_ERR_CUDA


def test_null_plan_is_rejected(lib):
    import ctypes

    n = ctypes.c_int64()
    assert lib.poly_plan_nbins(None, ctypes.byref(n)) == 1
    assert lib.poly_estimate(None, None, None, None, None) == 1
    lib.poly_plan_destroy(None)


def test_tuning_and_batched_entries_reject_null_arguments(lib):
    import ctypes

    cfg, ms = ctypes.c_int(), ctypes.c_double()
    assert lib.poly_plan_tune(None, None, ctypes.byref(cfg), ctypes.byref(ms), None) == 1
    assert lib.poly_plan_set_config(None, 0) == 1
    assert lib.poly_estimate_batched(None, None, None, 0, None) == 0  # an empty batch is a no-op
    assert lib.poly_estimate_batched(None, None, None, 2, None) == 1
    assert lib.poly_estimate_batched(None, None, None, -1, None) == 1


def test_every_abi_symbol_declares_its_argument_types(lib):
    """Without argtypes ctypes passes Python ints as 32-bit C ints, which truncates pointers."""
    for name in ps.ABI_SYMBOLS:
        assert getattr(lib, name).argtypes is not None, name


def test_binding_wrappers_marshal_without_a_device(lib):
    """Every ABI-named wrapper reaches the library and maps a NULL plan to POLY_ERR_ARG."""
    calls = [
        lambda: ps.poly_plan_nbins(None),
        lambda: ps.poly_plan_counts(None),
        lambda: ps.poly_plan_stats(None),
        lambda: ps.poly_plan_set_timing(None, True),
        lambda: ps.poly_plan_sync(None),
        lambda: ps.poly_estimate(None, None, None, None, None),
        lambda: ps.poly_backward(None, None, None, None, None),
        lambda: ps.poly_trispectrum_disconnected(None, None, None, None, None),
        lambda: ps.poly_plan_bin_wraps(None),
        lambda: ps.poly_plan_device_bytes(None),
    ]
    for call in calls:
        with pytest.raises(ps.PolyError) as ei:
            call()
        assert ei.value.status == 1
    assert lib.poly_plan_bin_wraps(None, None) == 1


def test_autotune_cache_tunes_once_per_signature(tmp_path):
    """autotune() times the shapes once per plan signature and restores the recorded choice afterwards
    (host logic only: a stand-in plan records the calls)."""
    class FakePlan:
        def __init__(self, sig):
            self.sig, self.calls = sig, []

        def signature(self):
            return self.sig

        def tune(self, delta):
            self.calls.append("tune")
            return 0x24, 7.5

        def set_config(self, cfg):
            self.calls.append(("set", cfg))

    cache = str(tmp_path / "tune.json")
    a = FakePlan("256/64/3/split")
    assert ps.autotune(a, None, cache) == 0x24 and a.calls == ["tune"]
    b = FakePlan("256/64/3/split")
    assert ps.autotune(b, None, cache) == 0x24 and b.calls == [("set", 0x24)]
    c = FakePlan("128/40/3/split")
    assert ps.autotune(c, None, cache) == 0x24 and c.calls == ["tune"]
    d = FakePlan("256/64/3/split")
    assert ps.autotune(d, None, None) == 0x24 and d.calls == ["tune"]  # no cache file: always tunes


C_CLIENT = r"""
#include <stdio.h>
#include <stdlib.h>
#include "polyspec.h"
#include "polyspec_diag.h"

int main(void) {
    /* argument errors come back before any device call */
    poly_plan plan = (poly_plan)1;
    const double edges[7] = {0.5, 1.5, 2.5, 3.5, 4.5, 5.5, 6.5};
    if (poly_plan_create(&plan, 32, 1000.0, 3, 6, NULL, POLY_FP32, 0) != POLY_ERR_ARG || plan != NULL) return 2;
    printf("status %s\n", poly_status_string(POLY_ERR_ALIAS));
    /* host tables through the diagnostic header */
    int64_t sizes[7];
    if (poly_diag_host_tables(32, 3, edges, 6, 0, 0, sizes, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL)) return 3;
    int32_t* bins = malloc(sizeof(int32_t) * 3 * (size_t)sizes[0]);
    if (poly_diag_host_tables(32, 3, edges, 6, 0, 0, sizes, bins, NULL, NULL, NULL, NULL, NULL, NULL, NULL)) return 4;
    printf("nbins %lld\n", (long long)sizes[0]);
    for (int64_t b = 0; b < sizes[0]; b++) printf("bin %d %d %d\n", bins[3 * b], bins[3 * b + 1], bins[3 * b + 2]);
    free(bins);
    int64_t ncell = 0;
    if (poly_diag_count_wedge(16, &ncell, NULL, NULL)) return 5;
    double* w = malloc(sizeof(double) * (size_t)ncell);
    if (poly_diag_count_wedge(16, &ncell, NULL, w)) return 6;
    double sum = 0.0;
    for (int64_t i = 0; i < ncell; i++) sum += w[i];
    printf("wedge %lld %.0f\n", (long long)ncell, sum);
    free(w);
    return 0;
}
"""


def test_plain_c_client_links_and_calls_the_host_entry_points(lib, tmp_path):
    """The boundary is a C ABI: a C99 program compiles against both headers (-Wall -Werror), links
    libpolyspec.so and calls the entry points that need no device."""
    import shutil
    import subprocess

    import oracle

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src, exe = tmp_path / "client.c", tmp_path / "client"
    src.write_text(C_CLIENT)
    libdir = os.path.dirname(ps.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", libdir, "-lpolyspec", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    assert out[0] == "status " + ps.poly_status_string(2)
    bins = np.array([[int(v) for v in line.split()[1:]] for line in out if line.startswith("bin ")])
    assert out[1] == f"nbins {len(bins)}"
    assert np.array_equal(bins, oracle.enumerate_bins(np.arange(7) + 0.5, 3))
    assert out[-1].split()[2] == str(16 ** 3)


def test_tensor_checks_run_before_any_library_call():
    """The binding refuses a tensor it cannot hand over as a pointer: host memory, another dtype, a strided
    view, a wrong size or another device (each reported by name), so no kernel reads past a buffer."""
    torch = pytest.importorskip("torch")

    class T:  # stand-in for a CUDA tensor (no device here)
        def __init__(self, dtype=torch.float32, n=512, contiguous=True, device="cuda:0"):
            self.is_cuda, self.dtype, self._n, self._c, self.device = True, dtype, n, contiguous, device

        def is_contiguous(self):
            return self._c

        def numel(self):
            return self._n

    ps._require(T(), torch.float32, 512, "delta", "cuda:0")
    for t, msg in [(torch.zeros(8, 8, 8), "CUDA tensor"), (T(dtype=torch.float64), "float32"),
                   (T(contiguous=False), "contiguous"), (T(n=511), "512 elements"),
                   (T(device="cuda:1"), "cuda:0")]:
        with pytest.raises(ValueError, match=msg):
            ps._require(t, torch.float32, 512, "delta", "cuda:0")
    plan = ps.Plan.__new__(ps.Plan)  # no library handle: every check below fires before a call
    plan.N, plan.nbins, plan.prec, plan.handle, plan.ell = 8, 5, ps.POLY_FP32, None, 0
    plan.edges = np.arange(4) + 0.5
    for call in (lambda: plan.estimate(torch.zeros(8, 8, 8)), lambda: plan.backward(torch.zeros(8, 8, 8), None),
                 lambda: plan.disconnected(torch.zeros(8, 8, 8)), lambda: plan.tune(torch.zeros(8, 8, 8))):
        with pytest.raises(ValueError, match="delta must be a CUDA tensor"):
            call()
    with pytest.raises(ValueError, match="512 elements"):
        plan.estimate_host(np.zeros(500, np.float32))
