"""Pins for the oracle's own FFT: the O(n^2) DFT written out, a library DFT (numpy.fft) and Parseval's identity."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n", list(range(1, 21)) + [27, 49, 96, 128, 160, 256])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_matches_numpy(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle.fft1d(x, sign)
    ref = np.fft.fft(x) if sign == -1 else np.fft.ifft(x) * n
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [8, 12, 15, 16])
def test_fft1d_matches_the_dft_definition(n):
    """X[k] = sum_j x[j] exp(sign 2 pi i j k / n), summed term by term."""
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    jk = np.outer(np.arange(n), np.arange(n))
    for sign in (-1, 1):
        ref = np.exp(sign * 2j * np.pi * jk / n) @ x
        assert np.abs(oracle.fft1d(x, sign) - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_fft3d_matches_the_dft_definition():
    """The 8^3 transform against the separable sum over all 8^3 points, term by term."""
    rng = np.random.default_rng(8)
    a = rng.standard_normal((8, 8, 8)) + 1j * rng.standard_normal((8, 8, 8))
    W = np.exp(-2j * np.pi * np.outer(np.arange(8), np.arange(8)) / 8)
    ref = np.einsum("ax,by,cz,xyz->abc", W, W, W, a)
    assert np.abs(oracle.fft3d(a, -1) - ref).max() < 1e-11


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 12), (16, 5, 9), (3, 1, 4)])
def test_fft3d_matches_numpy(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert np.abs(oracle.fft3d(a, -1) - np.fft.fftn(a)).max() < 1e-12
    assert np.abs(oracle.fft3d(a, +1) - np.fft.ifftn(a) * a.size).max() < 1e-12


def test_parseval_and_roundtrip():
    rng = np.random.default_rng(7)
    a = rng.standard_normal((12, 12, 12))
    f = oracle.fft3d(a, -1)
    assert abs(np.sum(np.abs(f) ** 2) / a.size - np.sum(a * a)) < 1e-10 * np.sum(a * a)
    back = oracle.fft3d(f, +1) / a.size
    assert np.abs(back.real - a).max() < 1e-13 and np.abs(back.imag).max() < 1e-13


def test_threads_do_not_change_results():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((16, 16, 16)) + 0j
    oracle.set_threads(1)
    one = oracle.fft3d(a)
    oracle.set_threads(4)
    four = oracle.fft3d(a)
    oracle.set_threads(1)
    assert np.array_equal(one, four)
