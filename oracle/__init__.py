"""FP64 CPU oracle for the FFT-based polyspectrum estimator (arXiv:1904.11055).

TEST INFRASTRUCTURE ONLY.  The product path never imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline``
leg and its ``--impl reference`` arm) may load it.  It shares no code with the
CUDA path; the two meet only through the seeded inputs of ``fieldgen``.

The arithmetic lives in ``oracle.c`` (plain C, FP64, its own mixed-radix FFT);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Conventions (paper Sec. 1, App. A): unnormalised forward DFT with e^{-i q.x},
unnormalised inverse with e^{+i q.x}; shell s holds the modes with
edges[s]^2 <= |q|^2 < edges[s+1]^2 (the half-width binning of Sec. 2); bins are
1-based sorted tuples k_1 >= ... >= k_n in the row-major order of Sec. 4.2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt copy of the library (used by the mutation test, which plants
# mistakes in a copy of oracle.c and checks that the pins catch them).
_LIB_OVERRIDE = os.environ.get("ORACLE_LIB_OVERRIDE")
_lib = None

RULE_POLYGON = 0   # k_1 <= k_2 + ... + k_n on shell centres (App. B, Eq. polygon)
RULE_ALL_SORTED = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            L = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.orc_last_error.restype = ctypes.c_char_p
        L.orc_set_threads.argtypes = [i32]
        L.orc_get_threads.restype = i32
        L.orc_fft1d.argtypes = [P, i32, i32]
        L.orc_fft3d.argtypes = [P, i32, i32, i32, i32]
        L.orc_shell_map.argtypes = [i32, i32, P, P]
        L.orc_enumerate_bins.argtypes = [i32, P, i32, i32, P]
        L.orc_enumerate_bins.restype = i64
        L.orc_forward.argtypes = [i32, P, P]
        L.orc_shell_fields.argtypes = [i32, P, P, i32, P, P, P]
        L.orc_product_sums.argtypes = [i32, P, P, i32, i64, P, P, P]
        L.orc_estimate.argtypes = [i32, f64, P, i32, P, i32, i64, P, P, P, P, P, P, P]
        L.orc_direct_sample.argtypes = [i32, P, i32, P, i32, i64, P, P, P]
        L.orc_counts_exact.argtypes = [i32, i32, P, i32, i64, P, P]
        L.orc_counts_triangles.argtypes = [i32, i32, P, i64, P, P]
        L.orc_gradient.argtypes = [i32, f64, P, i32, P, i32, i64, P, P, P, P]
        L.orc_disconnected.argtypes = [i32, f64, P, i32, P, i64, P, P, P, P]
        L.orc_estimate_ell.argtypes = [i32, f64, P, i32, P, i32, i32, i64, P, P, P, P]
        L.orc_trispectrum_full.argtypes = [i32, P, i32, P, P, i32, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}: {_load().orc_last_error().decode()}")


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def fft1d(x, sign: int = -1) -> np.ndarray:
    """Own mixed-radix DFT of a 1-D complex array (unnormalised, e^{sign 2 pi i jk/n})."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _check(_load().orc_fft1d(_p(a), a.size, sign))
    return a


def fft3d(x, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    n0, n1, n2 = a.shape
    _check(_load().orc_fft3d(_p(a), n0, n1, n2, sign))
    return a


def shell_map(N: int, edges) -> np.ndarray:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    out = np.empty((N, N, N), dtype=np.int32)
    _check(_load().orc_shell_map(N, e.size - 1, _p(e), _p(out)))
    return out


def enumerate_bins(edges, order: int, rule: int = RULE_POLYGON) -> np.ndarray:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    L = _load()
    nb = L.orc_enumerate_bins(e.size - 1, _p(e), order, rule, None)
    if nb < 0:
        _check(nb)
    out = np.empty((nb, order), dtype=np.int32)
    L.orc_enumerate_bins(e.size - 1, _p(e), order, rule, _p(out))
    return out


def forward(delta) -> np.ndarray:
    d = np.ascontiguousarray(delta, dtype=np.float64)
    N = d.shape[0]
    out = np.empty((N, N, N), dtype=np.complex128)
    _check(_load().orc_forward(N, _p(d), _p(out)))
    return out


def shell_fields(N: int, edges, shells, dhat=None):
    """D_s(x) for the given 0-based shells (dhat=None gives the counting fields iota_s)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    smap = shell_map(N, e)
    sel = np.ascontiguousarray(shells, dtype=np.int32)
    out = np.empty((sel.size, N, N, N), dtype=np.float64)
    im = ctypes.c_double(0.0)
    dh = None if dhat is None else np.ascontiguousarray(dhat, dtype=np.complex128)
    _check(_load().orc_shell_fields(N, _p(dh), _p(smap), sel.size, _p(sel), _p(out), ctypes.byref(im)))
    return out, im.value


def estimate(delta, L: float, edges, order: int, bins=None, rule: int = RULE_POLYGON) -> dict:
    """Whole estimator on a real N^3 field: B, R = S/(N^3 count), scale, counts, S."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    N = d.shape[0]
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = enumerate_bins(e, order, rule) if bins is None else np.ascontiguousarray(bins, dtype=np.int32)
    nb = b.shape[0]
    B = np.empty(nb)
    R = np.empty(nb)
    sc = np.empty(nb)
    S = np.empty(nb)
    cnt = np.empty(nb, dtype=np.int64)
    im = ctypes.c_double(0.0)
    _check(_load().orc_estimate(N, float(L), _p(d), e.size - 1, _p(e), order, nb, _p(b), _p(B), _p(R), _p(sc),
                                _p(cnt), _p(S), ctypes.byref(im)))
    return {"bins": b, "B": B, "R": R, "scale": sc, "counts": cnt, "S": S, "imag_max": im.value}


def direct_sample(delta, edges, order: int, bins, N: int | None = None):
    """Brute-force sum over all closed n-gons of grid modes (Eq. estimateBk). delta=None: counts only."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    nb = b.shape[0]
    S = np.zeros(nb)
    cnt = np.empty(nb, dtype=np.int64)
    if delta is None:
        assert N is not None
        _check(_load().orc_direct_sample(N, None, e.size - 1, _p(e), order, nb, _p(b), None, _p(cnt)))
        return None, cnt
    d = np.ascontiguousarray(delta, dtype=np.float64)
    _check(_load().orc_direct_sample(d.shape[0], _p(d), e.size - 1, _p(e), order, nb, _p(b), _p(S), _p(cnt)))
    return S, cnt


def counts_exact(N: int, edges, order: int, bins) -> np.ndarray:
    """Exact polygon counts (n = 2..6) by integer convolutions of the shell indicators (pairs; for n = 5, 6
    a group of n - 3 shells against a group of three)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    cnt = np.empty(b.shape[0], dtype=np.int64)
    _check(_load().orc_counts_exact(int(N), e.size - 1, _p(e), int(order), b.shape[0], _p(b), _p(cnt)))
    return cnt


def counts_triangles(N: int, edges, bins) -> np.ndarray:
    """Exact triangle counts (n = 3) for many bins at once: the pair convolutions of counts_exact, with the
    sum over the third shell taken for every third shell in one pass per pair (one convolution per pair)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    assert b.ndim == 2 and b.shape[1] == 3
    cnt = np.empty(b.shape[0], dtype=np.int64)
    _check(_load().orc_counts_triangles(int(N), e.size - 1, _p(e), b.shape[0], _p(b), _p(cnt)))
    return cnt


def estimate_ell(delta, L: float, edges, order: int, ell: int, bins) -> dict:
    """Multipole estimator: the first leg of each bin weighted by L_ell(q_z/|q|); B (with the 2 ell + 1
    factor), scale = sum_x |prod| / (N^3 count) with the weighted first leg, counts."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    nb = b.shape[0]
    B, sc, cnt = np.empty(nb), np.empty(nb), np.empty(nb, dtype=np.int64)
    _check(_load().orc_estimate_ell(d.shape[0], float(L), _p(d), e.size - 1, _p(e), int(order), int(ell), nb, _p(b),
                                    _p(B), _p(sc), _p(cnt)))
    return {"B": B, "scale": sc, "counts": cnt}


def trispectrum_full(delta, L: float, edges, k, dedges, N: int | None = None) -> dict:
    """Full-shape trispectrum of one bin k = (k1, k2, k3, k4) (Eq. Tkfull): the closed quadrilaterals split
    by their diagonals |q1 - q2| and |q1 - q3| into the bins of `dedges`.  Returns S and counts
    [ndiag, ndiag], T = (V^3/N^12) S / (N^3 count) (0 where count = 0) and `scale`, the same
    normalisation of A = N^3 sum prod_t |dhat(q_t)| (the size rounding errors in T are measured
    against).  delta=None: counts only."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    de = np.ascontiguousarray(dedges, dtype=np.float64)
    kk = np.ascontiguousarray(k, dtype=np.int32)
    nd = de.size - 1
    S = np.zeros((nd, nd))
    A = np.zeros((nd, nd))
    C = np.zeros((nd, nd), dtype=np.int64)
    if delta is None:
        assert N is not None
        _check(_load().orc_trispectrum_full(int(N), None, e.size - 1, _p(e), _p(kk), nd, _p(de), None, None, _p(C)))
    else:
        d = np.ascontiguousarray(delta, dtype=np.float64)
        N = d.shape[0]
        _check(_load().orc_trispectrum_full(N, _p(d), e.size - 1, _p(e), _p(kk), nd, _p(de), _p(S), _p(A), _p(C)))
    n3 = float(N) ** 3
    norm = (L ** 3) ** 3 / n3 ** 4
    T = np.where(C > 0, norm * S / (n3 * np.maximum(C, 1)), 0.0)
    scale = np.where(C > 0, norm * A / (n3 * np.maximum(C, 1)), 0.0)
    return {"S": S, "counts": C, "T": T, "scale": scale}


def disconnected(delta, L: float, edges, bins, counts):
    """Disconnected (Wick-paired) part of the trispectrum estimator per bin, and the shell powers
    P(k) = sum_{q in S_k} |dhat(q)|^2.  Returns (B_disc, P)."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    out = np.empty(b.shape[0])
    P = np.empty(e.size - 1)
    _check(_load().orc_disconnected(d.shape[0], float(L), _p(d), e.size - 1, _p(e), b.shape[0], _p(b), _p(c),
                                    _p(out), _p(P)))
    return out, P


def gradient(delta, L: float, edges, order: int, bins, counts, dLdB) -> np.ndarray:
    """dL/d delta(x) for L = sum_b dLdB_b B_b (analytic adjoint, FP64)."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    N = d.shape[0]
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    w = np.ascontiguousarray(dLdB, dtype=np.float64)
    out = np.empty((N, N, N))
    _check(_load().orc_gradient(N, float(L), _p(d), e.size - 1, _p(e), order, b.shape[0], _p(b), _p(c), _p(w),
                                _p(out)))
    return out
