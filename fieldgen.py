"""Seeded synthetic density fields: the only inputs shared by the oracle and the CUDA path.

This module holds none of the estimator's arithmetic; it only synthesises inputs.
The paper measures on no public dataset (its experiments are polygon counts on a
grid of unity and timings), so every workload is a seeded random field of the
shapes below.

Recipe (one real N^3 field, box side L, fundamental k_F = 2 pi / L):
  1. white noise w(x) ~ N(0, 1) from numpy.random.default_rng(seed);
  2. ghat(q) = FFT(w)(q) * sqrt(P(|q| k_F)), P(0) = 0;
  3. g = IFFT(ghat) (real), rescaled to unit sample variance;
  4. gaussian: delta = g;  lognormal: delta = exp(g - s^2/2) - 1, s^2 = var(g) = 1.
Power spectra (|q| in units of k_F):
  "cut":   P ~ k^-1.5 for k <= kcut, 0 above  (64^3 Gaussian workload, kcut = 16)
  "gauss": P ~ k^-1.5 exp(-(k / (0.5 k_Nyq))^2), k_Nyq = pi N / L, i.e. 0.5 k_Nyq = N/4 k_F
"""
from __future__ import annotations

import numpy as np


def _kmag(N: int) -> np.ndarray:
    m = np.fft.fftfreq(N) * N
    qx, qy, qz = np.meshgrid(m, m, m, indexing="ij")
    return np.sqrt(qx * qx + qy * qy + qz * qz)


def power_shape(N: int, spectrum: str, kcut: float | None = None) -> np.ndarray:
    k = _kmag(N)
    with np.errstate(divide="ignore"):
        p = np.where(k > 0, k ** -1.5, 0.0)
    if spectrum == "cut":
        p = np.where(k <= (16.0 if kcut is None else kcut), p, 0.0)
    elif spectrum == "gauss":
        p = p * np.exp(-(k / (N / 4.0)) ** 2)
    elif spectrum == "white":
        p = np.where(k > 0, 1.0, 0.0)
    else:
        raise ValueError(spectrum)
    return p


def gaussian_field(N: int, seed: int, spectrum: str = "gauss", kcut: float | None = None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((N, N, N))
    ghat = np.fft.fftn(w) * np.sqrt(power_shape(N, spectrum, kcut))
    g = np.fft.ifftn(ghat).real
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_field(N: int, seed: int, spectrum: str = "gauss") -> np.ndarray:
    g = gaussian_field(N, seed, spectrum)
    s2 = g.var()
    return np.exp(g - 0.5 * s2) - 1.0


def field(kind: str, N: int, seed: int, dtype=np.float32) -> np.ndarray:
    """kind: 'gaussian_cut16' | 'gaussian' | 'lognormal' | 'white'. Returned C-contiguous."""
    if kind == "gaussian_cut16":
        f = gaussian_field(N, seed, "cut", 16.0)
    elif kind == "gaussian":
        f = gaussian_field(N, seed, "gauss")
    elif kind == "lognormal":
        f = lognormal_field(N, seed, "gauss")
    elif kind == "white":
        f = np.random.default_rng(seed).standard_normal((N, N, N))
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(f.astype(dtype))


def plane_waves(N: int, waves) -> np.ndarray:
    """delta(x) = sum_a A_a cos(2 pi q_a . x / N + phi_a) for waves = [(q_a, A_a, phi_a), ...]."""
    i = np.arange(N)
    x, y, z = np.meshgrid(i, i, i, indexing="ij")
    out = np.zeros((N, N, N))
    for q, A, phi in waves:
        out += A * np.cos(2.0 * np.pi * (q[0] * x + q[1] * y + q[2] * z) / N + phi)
    return out


def unit_edges(nshell: int, width: float = 1.0) -> np.ndarray:
    """Edges c_i -/+ width/2 of shells centred on c_i = width * i, i = 1..nshell (units of k_F)."""
    return width * (np.arange(nshell + 1) + 0.5)
