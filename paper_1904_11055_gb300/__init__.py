"""Thin Python binding of libpolyspec.so (the C ABI in include/polyspec.h).

The functions below carry the ABI's names and only marshal arguments; every step
of the estimator runs in the CUDA library.  There is no CPU fallback: importing
works without a GPU, but any call that needs the library raises if it was not
built (``paper_1904_11055_gb300.build.build()``) or if CUDA is unavailable.

``Plan`` wraps a plan handle for torch tensors (device memory and streams only),
and ``PolyspectrumFunction`` is the torch.autograd.Function whose backward is the
library's hand-written adjoint (``poly_backward``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolyspec.so")

POLY_OK = 0
STATUS = {0: "POLY_OK", 1: "POLY_ERR_ARG", 2: "POLY_ERR_ALIAS", 3: "POLY_ERR_ALLOC", 4: "POLY_ERR_CUDA",
          5: "POLY_ERR_TIMEOUT", 6: "POLY_ERR_UNSUPPORTED", 7: "POLY_ERR_COUNT"}
POLY_FP32, POLY_SPLIT_BF16, POLY_TF32X3, POLY_FP64 = 0, 1, 2, 3
PRECISIONS = {"fp32": POLY_FP32, "split_bf16": POLY_SPLIT_BF16, "tf32x3": POLY_TF32X3, "fp64": POLY_FP64}
POLY_BINS_ALL_SORTED = 0x1
POLY_ALLOW_ALIAS = 0x2

# every symbol include/polyspec.h declares
ABI_SYMBOLS = ("poly_plan_create", "poly_plan_nbins", "poly_plan_bins", "poly_plan_counts", "poly_estimate",
               "poly_estimate_host", "poly_backward", "poly_estimate_batched", "poly_plan_sync", "poly_plan_destroy",
               "poly_status_string", "poly_last_error", "poly_debug_fail_alloc_after", "poly_plan_set_timing",
               "poly_plan_stats", "poly_estimate_noalloc", "poly_plan_tune", "poly_plan_set_config",
               "poly_trispectrum_disconnected", "poly_plan_create_multipole", "poly_plan_bin_wraps",
               "poly_plan_device_bytes", "poly_trispectrum_full")


class poly_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms_forward", ctypes.c_float), ("ms_fields", ctypes.c_float),
                ("ms_contract", ctypes.c_float), ("ms_reduce", ctypes.c_float), ("contract_flops", ctypes.c_double)]

_lib = None


class PolyError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({msg})" if msg else ""))


def load_library():
    """Load libpolyspec.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1904_11055_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, f64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint
    L.poly_plan_create.argtypes = [ctypes.POINTER(P), i32, f64, i32, i32, P, i32, u32]
    L.poly_plan_create_multipole.argtypes = [ctypes.POINTER(P), i32, f64, i32, i32, P, i32, u32, i32]
    L.poly_plan_nbins.argtypes = [P, ctypes.POINTER(i64)]
    L.poly_plan_bins.argtypes = [P, P]
    L.poly_plan_counts.argtypes = [P, P]
    L.poly_plan_bin_wraps.argtypes = [P, P]
    L.poly_plan_device_bytes.argtypes = [P, ctypes.POINTER(i64)]
    L.poly_estimate.argtypes = [P, P, P, P, P]
    L.poly_estimate_host.argtypes = [P, P, P, P]
    L.poly_backward.argtypes = [P, P, P, P, P]
    L.poly_estimate_batched.argtypes = [P, P, P, i32, P]
    L.poly_plan_sync.argtypes = [P, P]
    L.poly_plan_destroy.argtypes = [P]
    L.poly_plan_destroy.restype = None
    L.poly_status_string.argtypes = [i32]
    L.poly_status_string.restype = ctypes.c_char_p
    L.poly_last_error.restype = ctypes.c_char_p
    L.poly_plan_set_timing.argtypes = [P, i32]
    L.poly_plan_stats.argtypes = [P, ctypes.POINTER(poly_stats)]
    L.poly_estimate_noalloc.argtypes = [i32, f64, i32, P, P, P, P, P]
    L.poly_plan_tune.argtypes = [P, P, ctypes.POINTER(i32), ctypes.POINTER(f64), P]
    L.poly_plan_set_config.argtypes = [P, i32]
    L.poly_trispectrum_disconnected.argtypes = [P, P, P, P, P]
    L.poly_trispectrum_full.argtypes = [P, P, P, i32, P, P, P, P, P]
    L.poly_last_error.argtypes = []
    L.poly_debug_fail_alloc_after.argtypes = [i32]
    L.poly_debug_fail_alloc_after.restype = None
    for name in ABI_SYMBOLS:
        if name not in ("poly_plan_destroy", "poly_status_string", "poly_last_error", "poly_debug_fail_alloc_after"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def _check(status: int, where: str):
    if status != POLY_OK:
        raise PolyError(status, where, load_library().poly_last_error().decode())


# ---------------------------------------------------------------- ABI-named calls
def poly_plan_create(N: int, L: float, order: int, edges, prec: int = POLY_FP32, flags: int = 0) -> int:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load_library().poly_plan_create(ctypes.byref(h), int(N), float(L), int(order), e.size - 1,
                                           e.ctypes.data_as(ctypes.c_void_p), int(prec), int(flags)),
           "poly_plan_create")
    return h.value


def poly_plan_create_multipole(N: int, L: float, order: int, edges, prec: int = POLY_FP32, flags: int = 0,
                               ell: int = 0) -> int:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load_library().poly_plan_create_multipole(ctypes.byref(h), int(N), float(L), int(order), e.size - 1,
                                                     e.ctypes.data_as(ctypes.c_void_p), int(prec), int(flags),
                                                     int(ell)),
           "poly_plan_create_multipole")
    return h.value


def poly_plan_nbins(plan: int) -> int:
    n = ctypes.c_int64()
    _check(load_library().poly_plan_nbins(plan, ctypes.byref(n)), "poly_plan_nbins")
    return n.value


def poly_plan_bins(plan: int, order: int) -> np.ndarray:
    out = np.empty((poly_plan_nbins(plan), order), dtype=np.int32)
    _check(load_library().poly_plan_bins(plan, out.ctypes.data_as(ctypes.c_void_p)), "poly_plan_bins")
    return out


def poly_plan_counts(plan: int) -> np.ndarray:
    out = np.empty(poly_plan_nbins(plan), dtype=np.int64)
    _check(load_library().poly_plan_counts(plan, out.ctypes.data_as(ctypes.c_void_p)), "poly_plan_counts")
    return out


def poly_plan_bin_wraps(plan: int) -> np.ndarray:
    """Per bin, True where closures that wrap around the grid may add to the count (see the header)."""
    out = np.empty(poly_plan_nbins(plan), dtype=np.uint8)
    _check(load_library().poly_plan_bin_wraps(plan, out.ctypes.data_as(ctypes.c_void_p)), "poly_plan_bin_wraps")
    return out.astype(bool)


def poly_plan_device_bytes(plan: int) -> int:
    """Device memory the plan holds, in bytes."""
    v = ctypes.c_int64(0)
    _check(load_library().poly_plan_device_bytes(plan, ctypes.byref(v)), "poly_plan_device_bytes")
    return v.value


def poly_estimate(plan: int, delta_ptr: int, out_ptr: int, scale_ptr: int | None, stream: int | None) -> None:
    _check(load_library().poly_estimate(plan, delta_ptr, out_ptr, scale_ptr, stream), "poly_estimate")


def poly_estimate_host(plan: int, delta_host: np.ndarray, out_host: np.ndarray, stream: int | None = None) -> None:
    _check(load_library().poly_estimate_host(plan, delta_host.ctypes.data_as(ctypes.c_void_p),
                                             out_host.ctypes.data_as(ctypes.c_void_p), stream),
           "poly_estimate_host")


def poly_backward(plan: int, delta_ptr: int, dLdB_ptr: int, grad_ptr: int, stream: int | None) -> None:
    _check(load_library().poly_backward(plan, delta_ptr, dLdB_ptr, grad_ptr, stream), "poly_backward")


def poly_trispectrum_disconnected(plan: int, delta_ptr: int, out_ptr: int, power_ptr: int | None,
                                  stream: int | None) -> None:
    _check(load_library().poly_trispectrum_disconnected(plan, delta_ptr, out_ptr, power_ptr, stream),
           "poly_trispectrum_disconnected")


def poly_trispectrum_full(plan: int, delta_ptr: int | None, k, dedges, T_ptr: int | None, counts_ptr: int | None,
                          scale_ptr: int | None, stream: int | None) -> None:
    kk = np.ascontiguousarray(k, dtype=np.int32)
    de = np.ascontiguousarray(dedges, dtype=np.float64)
    if kk.shape != (4,) or de.ndim != 1 or de.size < 2:
        raise ValueError("k must hold 4 shell numbers and dedges at least 2 edges")
    _check(load_library().poly_trispectrum_full(plan, delta_ptr, kk.ctypes.data_as(ctypes.c_void_p), de.size - 1,
                                                de.ctypes.data_as(ctypes.c_void_p), T_ptr, counts_ptr, scale_ptr,
                                                stream), "poly_trispectrum_full")


def poly_estimate_batched(plans, field_ptrs, out_ptrs, stream: int | None) -> None:
    n = len(plans)
    P = ctypes.c_void_p * n
    _check(load_library().poly_estimate_batched(P(*plans), P(*field_ptrs), P(*out_ptrs), n, stream),
           "poly_estimate_batched")


def poly_plan_sync(plan: int, stream: int | None = None) -> None:
    _check(load_library().poly_plan_sync(plan, stream), "poly_plan_sync")


def poly_plan_tune(plan: int, delta_ptr: int, stream: int | None = None) -> tuple[int, float]:
    cfg, ms = ctypes.c_int(), ctypes.c_double()
    _check(load_library().poly_plan_tune(plan, delta_ptr, ctypes.byref(cfg), ctypes.byref(ms), stream),
           "poly_plan_tune")
    return cfg.value, ms.value


def poly_plan_set_config(plan: int, config: int) -> None:
    _check(load_library().poly_plan_set_config(plan, int(config)), "poly_plan_set_config")


def poly_plan_destroy(plan: int) -> None:
    load_library().poly_plan_destroy(plan)


def poly_plan_set_timing(plan: int, enable: bool) -> None:
    _check(load_library().poly_plan_set_timing(plan, int(bool(enable))), "poly_plan_set_timing")


def poly_plan_stats(plan: int) -> dict:
    st = poly_stats()
    _check(load_library().poly_plan_stats(plan, ctypes.byref(st)), "poly_plan_stats")
    return {k: getattr(st, k) for k, _ in poly_stats._fields_}


def poly_estimate_noalloc(N: int, L: float, edges, delta_ptr: int, counts: np.ndarray, out_ptr: int,
                          stream: int | None) -> None:
    """B_b of a small order-3 FP32 problem with no device allocation (see include/polyspec.h).

    counts must hold one exact count per bin of these shells (the library copies nbins of them from host
    memory): its length is checked against the bin count first."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    lib = load_library()
    nb = ctypes.c_int64(0)
    lib.poly_diag_bin_wraps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    lib.poly_diag_bin_wraps.restype = ctypes.c_int
    if (lib.poly_diag_bin_wraps(int(N), 3, e.ctypes.data_as(ctypes.c_void_p), e.size - 1, 0, ctypes.byref(nb), None)
            == POLY_OK and c.ndim == 1 and c.size != nb.value):
        raise ValueError(f"counts holds {c.size} values; the bispectrum of these shells has {nb.value} bins")
    if c.ndim != 1:
        raise ValueError("counts must be one-dimensional")
    _check(load_library().poly_estimate_noalloc(int(N), float(L), e.size - 1, e.ctypes.data_as(ctypes.c_void_p),
                                                delta_ptr, c.ctypes.data_as(ctypes.c_void_p), out_ptr, stream),
           "poly_estimate_noalloc")


def diag_fma_peak(is_double: bool = False, iters: int | None = None) -> dict:
    """Measured peak FMA rate of the CUDA cores (poly_diag_fma_peak in include/polyspec_diag.h)."""
    lib = load_library()
    lib.poly_diag_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.poly_diag_fma_peak.restype = ctypes.c_int
    it = iters if iters is not None else (4096 if is_double else 131072)
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.poly_diag_fma_peak(int(bool(is_double)), int(it), ctypes.byref(tf), ctypes.byref(ms)),
           "poly_diag_fma_peak")
    return {"tflops": tf.value, "ms": ms.value, "iters": it, "dtype": "f64" if is_double else "f32"}


def poly_status_string(status: int) -> str:
    return load_library().poly_status_string(int(status)).decode()


def poly_debug_fail_alloc_after(n: int) -> None:
    load_library().poly_debug_fail_alloc_after(int(n))


# ---------------------------------------------------------------- torch-facing wrapper
def _stream_handle(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _require(t, dtype, numel: int, name: str, device=None) -> None:
    """Check a tensor handed to the library before its pointer is: CUDA, dtype, contiguous, size, device."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, not {t.numel()}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} must be on {device}, not {t.device}")


class Plan:
    """A plan for one (N, L, n, edges, precision); owns the library handle."""

    def __init__(self, N: int, L: float, order: int, edges, precision: str | int = "fp32", flags: int = 0,
                 ell: int = 0):
        """ell > 0: redshift-space multipole plan (the first leg weighted by L_ell(q_z/|q|))."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.N, self.L, self.order, self.prec, self.flags = int(N), float(L), int(order), prec, int(flags)
        self.ell = int(ell)
        self.edges = np.ascontiguousarray(edges, dtype=np.float64)
        self.handle = (poly_plan_create(N, L, order, self.edges, prec, flags) if self.ell == 0 else
                       poly_plan_create_multipole(N, L, order, self.edges, prec, flags, self.ell))
        self.nbins = poly_plan_nbins(self.handle)
        self.bins = poly_plan_bins(self.handle, order)
        self.counts = poly_plan_counts(self.handle)

    @property
    def real_dtype(self):
        import torch

        return torch.float64 if self.prec == POLY_FP64 else torch.float32

    def estimate(self, delta, out=None, scale: bool = False, stream=None):
        """delta: CUDA tensor [N,N,N] of the plan's real dtype.  Returns B (float64) [and scale]."""
        import torch

        _require(delta, self.real_dtype, self.N ** 3, "delta")
        out = torch.empty(self.nbins, dtype=torch.float64, device=delta.device) if out is None else out
        _require(out, torch.float64, self.nbins, "out", delta.device)
        sc = torch.empty(self.nbins, dtype=torch.float64, device=delta.device) if scale else None
        poly_estimate(self.handle, delta.data_ptr(), out.data_ptr(), sc.data_ptr() if scale else None,
                      _stream_handle(stream))
        return (out, sc) if scale else out

    def estimate_host(self, delta: np.ndarray) -> np.ndarray:
        d = np.ascontiguousarray(delta, dtype=np.float64 if self.prec == POLY_FP64 else np.float32)
        if d.size != self.N ** 3:
            raise ValueError(f"delta must have {self.N ** 3} elements, not {d.size}")
        out = np.empty(self.nbins, dtype=np.float64)
        poly_estimate_host(self.handle, d, out, None)
        return out

    def backward(self, delta, dLdB, grad=None, stream=None):
        import torch

        _require(delta, self.real_dtype, self.N ** 3, "delta")
        g = dLdB.to(device=delta.device, dtype=torch.float64).contiguous()
        _require(g, torch.float64, self.nbins, "dLdB")
        grad = torch.empty_like(delta) if grad is None else grad
        _require(grad, self.real_dtype, self.N ** 3, "grad", delta.device)
        poly_backward(self.handle, delta.data_ptr(), g.data_ptr(), grad.data_ptr(), _stream_handle(stream))
        return grad

    def disconnected(self, delta, out=None, power: bool = False, stream=None):
        """Order-4 plans: the disconnected (Wick-paired) part B_disc of the trispectrum estimate of delta
        (subtract it from estimate() for the connected part).  Returns B_disc [and the shell powers]."""
        import torch

        _require(delta, self.real_dtype, self.N ** 3, "delta")
        out = torch.empty(self.nbins, dtype=torch.float64, device=delta.device) if out is None else out
        _require(out, torch.float64, self.nbins, "out", delta.device)
        pw = torch.empty(len(self.edges) - 1, dtype=torch.float64, device=delta.device) if power else None
        poly_trispectrum_disconnected(self.handle, delta.data_ptr(), out.data_ptr(), pw.data_ptr() if power else None,
                                      _stream_handle(stream))
        return (out, pw) if power else out

    def trispectrum_full(self, delta, k, dedges, scale: bool = False, stream=None):
        """Full-shape trispectrum of the shell quadruple k (1-based) split by the diagonals |q1 - q2| and
        |q1 - q3| into the bins of dedges (Eq. Tkfull).  Returns (T, counts) [and scale], each
        [ndiag, ndiag] on the device; delta=None gives the counts alone."""
        import torch

        nd = len(dedges) - 1
        dev = delta.device if delta is not None else torch.device("cuda", torch.cuda.current_device())
        if delta is not None:
            _require(delta, self.real_dtype, self.N ** 3, "delta")
        T = torch.empty((nd, nd), dtype=torch.float64, device=dev) if delta is not None else None
        C = torch.empty((nd, nd), dtype=torch.int64, device=dev)
        sc = torch.empty((nd, nd), dtype=torch.float64, device=dev) if scale else None
        poly_trispectrum_full(self.handle, delta.data_ptr() if delta is not None else None, k, dedges,
                              T.data_ptr() if T is not None else None, C.data_ptr(),
                              sc.data_ptr() if scale else None, _stream_handle(stream))
        if delta is None:
            return C
        return (T, C, sc) if scale else (T, C)

    def sync(self, stream=None):
        poly_plan_sync(self.handle, _stream_handle(stream))

    def tune(self, delta, stream=None) -> tuple[int, float]:
        """Time the contraction shapes on this field's shells; keep the fastest (returns code, ms)."""
        _require(delta, self.real_dtype, self.N ** 3, "delta")
        return poly_plan_tune(self.handle, delta.data_ptr(), _stream_handle(stream))

    def set_config(self, config: int) -> None:
        poly_plan_set_config(self.handle, config)

    def device_bytes(self) -> int:
        """Device memory the plan holds, in bytes (its workspace; the adjoint's once backward has run)."""
        return poly_plan_device_bytes(self.handle)

    def bin_wraps(self) -> np.ndarray:
        """Per bin, True where closures that wrap around the grid may add to it (POLY_ALLOW_ALIAS plans)."""
        return poly_plan_bin_wraps(self.handle)

    def signature(self) -> str:
        """Key for a tuning cache: everything the contraction shape depends on, plus the GPU model."""
        import torch

        e = ",".join(f"{v:.17g}" for v in self.edges)
        return f"{torch.cuda.get_device_name()}|N={self.N}|n={self.order}|p={self.prec}|f={self.flags}|e={e}"

    def close(self):
        if getattr(self, "handle", None):
            poly_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_batched(plans, fields, outs=None, stream=None):
    """Estimate many fields (of possibly different plans) in one call; returns the output tensors."""
    import torch

    if outs is None:
        outs = [torch.empty(p.nbins, dtype=torch.float64, device=f.device) for p, f in zip(plans, fields)]
    poly_estimate_batched([p.handle for p in plans], [f.data_ptr() for f in fields], [o.data_ptr() for o in outs],
                          _stream_handle(stream))
    return outs


def autotune(plan: Plan, delta, cache_path: str | None = None) -> int:
    """Tune plan on delta, or restore the choice recorded for the same signature in cache_path (JSON)."""
    import json

    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    key = plan.signature()
    if key in cache:
        plan.set_config(int(cache[key]["config"]))
        return int(cache[key]["config"])
    cfg, ms = plan.tune(delta)
    if cache_path:
        cache[key] = {"config": cfg, "contract_ms": ms}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return cfg


def _make_function():
    import torch

    class PolyspectrumFunction(torch.autograd.Function):
        """B = estimate(delta); backward returns the library's adjoint dL/d delta."""

        @staticmethod
        def forward(ctx, delta, plan):
            ctx.plan = plan
            ctx.save_for_backward(delta)
            return plan.estimate(delta.contiguous())

        @staticmethod
        def backward(ctx, gB):
            (delta,) = ctx.saved_tensors
            return ctx.plan.backward(delta.contiguous(), gB), None

    return PolyspectrumFunction


def polyspectrum(delta, plan: Plan):
    """Differentiable estimate: torch.autograd sees dL/d delta from poly_backward."""
    global PolyspectrumFunction
    if "PolyspectrumFunction" not in globals():
        PolyspectrumFunction = _make_function()
    return PolyspectrumFunction.apply(delta, plan)
