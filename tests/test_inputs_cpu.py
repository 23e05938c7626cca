"""The seeded input generator follows its stated recipe (no estimator arithmetic is involved):
unit-variance Gaussian fields with P(k) ~ k^-1.5 (cut above 16 k_F, or damped by exp(-(k / (N/4))^2)),
the lognormal map delta = exp(g - s^2/2) - 1, and the same field for the same seed."""
import numpy as np

import fieldgen


def shell_power(f, kmax):
    N = f.shape[0]
    F = np.fft.fftn(f)
    k = np.rint(fieldgen._kmag(N)).astype(int)
    p = np.bincount(k.ravel(), weights=(np.abs(F) ** 2).ravel(), minlength=kmax + 1)
    n = np.bincount(k.ravel(), minlength=kmax + 1)
    return p[: kmax + 1] / np.maximum(n[: kmax + 1], 1)


def test_gaussian_fields_have_unit_variance_and_zero_mean():
    for kind in ("gaussian", "gaussian_cut16"):
        g = fieldgen.field(kind, 32, 7, np.float64)
        assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12


def test_cut_spectrum_has_no_power_above_16_kF_and_falls_as_k_to_the_minus_1_5():
    g = fieldgen.field("gaussian_cut16", 64, 1, np.float64)
    F = np.fft.fftn(g)
    k = fieldgen._kmag(64)
    assert np.abs(F[k > 16.0]).max() < 1e-9 * np.abs(F).max()
    P = shell_power(g, 16)
    ks = np.arange(4, 16)
    slope = np.polyfit(np.log(ks), np.log(P[ks]), 1)[0]
    assert abs(slope + 1.5) < 0.15, slope


def test_damped_spectrum_follows_the_gaussian_damping():
    N = 64
    g = fieldgen.field("gaussian", N, 3, np.float64)
    P = shell_power(g, 30)
    ks = np.arange(4, 30)
    model = ks ** -1.5 * np.exp(-(ks / (N / 4.0)) ** 2)
    r = P[ks] / model
    assert np.std(np.log(r)) < 0.15  # one amplitude fits every shell, within the shells' sampling noise


def test_lognormal_map():
    g = fieldgen.gaussian_field(32, 5, "gauss")
    d = fieldgen.lognormal_field(32, 5, "gauss")
    assert np.allclose(d, np.exp(g - 0.5 * g.var()) - 1.0)
    assert d.min() > -1.0 and abs(d.mean()) < 0.05


def test_fields_are_determined_by_the_seed():
    a, b, c = (fieldgen.field("lognormal", 24, s, np.float32) for s in (11, 11, 12))
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.flags.c_contiguous and a.dtype == np.float32
