"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself:
  * shell membership and bin enumeration: independent numpy / itertools code;
  * polygon counts: direct enumeration of closed n-gons (Sec. 4, Eq. Ncalc) and
    the golden file written from that enumeration;
  * product sums: brute-force direct sampling of all triangles / quadrilaterals
    (Eq. estimateBk and its n-gon form);
  * n = 2: the textbook shell-averaged power spectrum from numpy.fft;
  * plane waves: closed forms for the connected and the disconnected case;
  * iid skewed noise: E[B] = kappa_3 (V/N^3)^2 for every bin (normalisation);
  * Gaussian fields: near-zero mean bispectrum;
  * analytic triangle counts (Eq. Ntri) within the paper's stated accuracy;
  * the adjoint: central finite differences of the estimator.
"""
import itertools
import os

import numpy as np
import pytest

import fieldgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def np_shell_map(N, edges):
    m = np.fft.fftfreq(N) * N
    qx, qy, qz = np.meshgrid(m, m, m, indexing="ij")
    q2 = qx * qx + qy * qy + qz * qz
    out = -np.ones((N, N, N), dtype=np.int32)
    for s in range(len(edges) - 1):
        sel = (q2 >= edges[s] ** 2) & (q2 < edges[s + 1] ** 2) & (q2 > 0)
        out[sel] = s
    return out


def itertools_bins(nshell, order, centres=None, all_sorted=False):
    c = np.arange(1, nshell + 1, dtype=float) if centres is None else np.asarray(centres)
    out = []
    for k in itertools.product(range(nshell, 0, -1), repeat=order):
        if any(k[t] < k[t + 1] for t in range(order - 1)):
            continue
        if all_sorted or c[k[0] - 1] <= sum(c[v - 1] for v in k[1:]) + 1e-9:
            out.append(k)
    out.sort()  # row-major order, k_n fastest, ascending
    return np.array(out, dtype=np.int32).reshape(-1, order)


# --------------------------------------------------------------------------- shells and bins
@pytest.mark.parametrize("N,width,nshell,first", [(16, 1.0, 7, 0), (20, 1.0, 9, 0), (24, 1.5, 7, 0), (15, 1.0, 7, 0),
                                                  (16, 1.0, 4, 2)])
def test_shell_map_matches_numpy(N, width, nshell, first):
    e = fieldgen.unit_edges(nshell + first, width)[first:]
    assert np.array_equal(oracle.shell_map(N, e), np_shell_map(N, e))


@pytest.mark.parametrize("nshell,order,width,expected", [(16, 3, 1.0, 508), (64, 3, 1.0, 24432),
                                                         (32, 4, 1.5, 45135), (32, 3, 1.0, 3384)])
def test_bin_enumeration(nshell, order, width, expected):
    e = fieldgen.unit_edges(nshell, width)
    got = oracle.enumerate_bins(e, order)
    assert got.shape == (expected, order)
    if nshell <= 32:
        ref = itertools_bins(nshell, order, centres=width * np.arange(1, nshell + 1))
        assert np.array_equal(got, ref)
    # paper order: k_1 >= ... >= k_n, row-major with k_n fastest
    assert np.all(np.diff(got, axis=1) <= 0)
    keys = [tuple(r) for r in got]
    assert keys == sorted(keys)


def test_all_sorted_rule():
    e = fieldgen.unit_edges(6)
    got = oracle.enumerate_bins(e, 3, oracle.RULE_ALL_SORTED)
    assert np.array_equal(got, itertools_bins(6, 3, all_sorted=True))


# --------------------------------------------------------------------------- counts
def _golden_counts(name):
    path = os.path.join(GOLDEN, name)
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return np.array([[int(v) for v in r] for r in rows], dtype=np.int64)


def test_counts_match_golden_enumeration():
    g = _golden_counts("counts_n3_N16_unit6.txt")
    e = fieldgen.unit_edges(6)
    r = oracle.estimate(np.zeros((16, 16, 16)), 1.0, e, 3, bins=g[:, :3].astype(np.int32))
    assert np.array_equal(r["counts"], g[:, 3])


@pytest.mark.parametrize("N,order,width,nshell", [(16, 3, 1.0, 6), (20, 3, 1.0, 5), (16, 3, 1.5, 4),
                                                  (12, 4, 1.0, 4), (15, 3, 1.0, 4)])
def test_counts_match_direct_enumeration(N, order, width, nshell):
    e = fieldgen.unit_edges(nshell, width)
    bins = oracle.enumerate_bins(e, order, oracle.RULE_ALL_SORTED)
    r = oracle.estimate(np.zeros((N, N, N)), 1.0, e, order, bins=bins)
    _, cnt = oracle.direct_sample(None, e, order, bins, N=N)
    assert np.array_equal(r["counts"], cnt)


@pytest.mark.parametrize("N,order,width,nshell", [(16, 3, 1.0, 6), (16, 2, 1.0, 6), (12, 4, 1.0, 4),
                                                  (12, 4, 1.5, 3), (15, 3, 1.0, 4), (16, 3, 1.5, 5)])
def test_exact_pair_convolution_counts_match_direct_enumeration(N, order, width, nshell):
    """The integer pair-convolution counts (used where the FP64 counting-field sum is not within
    1e-6 of an integer) against brute-force enumeration of the tuples and the counting fields."""
    e = fieldgen.unit_edges(nshell, width)
    bins = oracle.enumerate_bins(e, order, oracle.RULE_ALL_SORTED)
    exact = oracle.counts_exact(N, e, order, bins)
    _, cnt = oracle.direct_sample(None, e, order, bins, N=N)
    assert np.array_equal(exact, cnt)
    r = oracle.estimate(np.zeros((N, N, N)), 1.0, e, order, bins=bins)
    assert np.array_equal(exact, r["counts"])


@pytest.mark.parametrize("N,width,nshell,rule", [(16, 1.0, 6, "all"), (15, 1.0, 4, "all"), (20, 1.5, 6, "all"),
                                                 (24, 1.0, 10, "polygon")])
def test_batched_triangle_counts_equal_the_pair_convolution_counts(N, width, nshell, rule):
    """counts_triangles (one convolution and one histogram pass per pair) against direct enumeration
    of the closed triangles and against counts_exact, bit for bit, including zero-count bins and
    grids where closures wrap (16^3 with shells up to 6.5)."""
    e = fieldgen.unit_edges(nshell, width)
    bins = oracle.enumerate_bins(e, 3, oracle.RULE_ALL_SORTED if rule == "all" else oracle.RULE_POLYGON)
    tri = oracle.counts_triangles(N, e, bins)
    assert np.array_equal(tri, oracle.counts_exact(N, e, 3, bins))
    if N <= 16:
        _, cnt = oracle.direct_sample(None, e, 3, bins, N=N)
        assert np.array_equal(tri, cnt)
    if rule == "all":
        assert (tri == 0).any() and (tri > 0).any()


def test_golden_benchmark_counts_hold_on_the_256cube_grid():
    """tests/golden/counts_n3_64shells.txt was computed on a 200^3 grid (no closure of shells up to
    64.5 wraps on any grid above 192); re-derive the bins of two pairs on the 256^3 grid itself with
    counts_exact."""
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "counts_n3_64shells.txt"),
                      dtype=np.int64, comments="#")
    sel = rows[((rows[:, 0] == 64) & (rows[:, 1] == 63)) | ((rows[:, 0] == 41) & (rows[:, 1] == 23))]
    assert len(sel) > 60
    e = fieldgen.unit_edges(64)
    got = oracle.counts_exact(256, e, 3, sel[:, :3].astype(np.int32))
    assert np.array_equal(got, sel[:, 3])


def dp_counts(N, edges, bins):
    """Closed n-gon counts by dynamic programming over partial sums of grid modes (no FFT): the
    histogram of q_1 + ... + q_t (mod N) grows one shell at a time; the count is its value at 0."""
    smap = np_shell_map(N, edges)
    modes = [np.argwhere(smap == s) for s in range(len(edges) - 1)]
    out = []
    for b in bins:
        h = np.zeros((N, N, N), dtype=np.int64)
        h[0, 0, 0] = 1
        for k in b:
            nh = np.zeros_like(h)
            for q in modes[k - 1]:
                nh += np.roll(h, shift=tuple(int(v) for v in q), axis=(0, 1, 2))
            h = nh
        out.append(int(h[0, 0, 0]))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("N,order,width,nshell", [(13, 5, 1.0, 2), (16, 6, 1.0, 2), (12, 5, 1.5, 1)])
def test_exact_group_convolution_counts_n5_n6(N, order, width, nshell):
    """n = 5, 6: the group-convolution counts against dynamic programming over the tuples, the brute-force
    sampler, and the counting-field sums of the estimator (which fall back to the exact counts)."""
    e = fieldgen.unit_edges(nshell, width)
    bins = oracle.enumerate_bins(e, order, oracle.RULE_ALL_SORTED)
    exact = oracle.counts_exact(N, e, order, bins)
    assert np.array_equal(exact, dp_counts(N, e, bins))
    assert exact.max() > 0
    if order == 5:
        _, cnt = oracle.direct_sample(None, e, order, bins, N=N)
        assert np.array_equal(exact, cnt)
    r = oracle.estimate(np.zeros((N, N, N)), 1.0, e, order, bins=bins)
    assert np.array_equal(exact, r["counts"])


def wick_brute_force(delta, edges, bins):
    """N^3 x the Wick-paired sum over every closed quadrilateral of grid modes, tuple by tuple:
    sum over (q1, q2, q3) with q4 = -(q1 + q2 + q3) in its shell of
    [q1+q2=0][q3+q4=0]|d(q1)|^2|d(q3)|^2 + [q1+q3=0][q2+q4=0]|d(q1)|^2|d(q2)|^2 + [q1+q4=0][q2+q3=0]|d(q1)|^2|d(q2)|^2."""
    N = delta.shape[0]
    dh = np.fft.fftn(delta)
    pw = np.abs(dh) ** 2
    smap = np_shell_map(N, edges)
    modes = [np.argwhere(smap == s) for s in range(len(edges) - 1)]
    out = []
    for b in bins:
        q1, q2, q3 = (modes[k - 1] for k in b[:3])
        A = q1[:, None, None, :]
        B = q2[None, :, None, :]
        C = q3[None, None, :, :]
        D = (-(A + B + C)) % N
        inb = smap[D[..., 0], D[..., 1], D[..., 2]] == b[3] - 1
        zero = lambda u, v: np.all((u + v) % N == 0, axis=-1)
        p1 = pw[A[..., 0], A[..., 1], A[..., 2]]
        p2 = pw[B[..., 0], B[..., 1], B[..., 2]]
        p3 = pw[C[..., 0], C[..., 1], C[..., 2]]
        w = zero(A, B) & zero(C, D), zero(A, C) & zero(B, D), zero(A, D) & zero(B, C)
        tot = (w[0] * p1 * p3 + w[1] * p1 * p2 + w[2] * p1 * p2) * inb
        out.append(N ** 3 * tot.sum())
    return np.array(out)


def test_disconnected_trispectrum_matches_wick_enumeration():
    N, L, e = 10, 50.0, fieldgen.unit_edges(3)
    d = fieldgen.field("lognormal", N, 5, np.float64)
    bins = oracle.enumerate_bins(e, 4, oracle.RULE_ALL_SORTED)
    r = oracle.estimate(d, L, e, 4, bins=bins)
    Bd, P = oracle.disconnected(d, L, e, bins, r["counts"])
    Sd = wick_brute_force(d, e, bins)
    c4 = (L ** 3) ** 3 / float(N ** 3) ** 4
    ok = r["counts"] > 0
    ref = np.where(ok, c4 * Sd / (N ** 3 * np.maximum(r["counts"], 1)), 0.0)
    assert np.count_nonzero(ref) >= 3
    assert np.allclose(Bd, ref, rtol=1e-12, atol=0.0)
    # the shell powers are the per-mode power summed over each shell
    smap = np_shell_map(N, e)
    pw = np.abs(np.fft.fftn(d)) ** 2
    assert np.allclose(P, [pw[smap == s].sum() for s in range(3)], rtol=1e-12)
    # bins (k, k, k, k) pair under all three pairings: a positive disconnected part
    kk = np.all(bins == bins[:, :1], axis=1)
    assert np.all(Bd[kk & ok] > 0)


def multipole_brute_force(delta, L, edges, ell, bins, counts):
    """B^ell of triangles by enumeration of the closed triples, numpy's FFT and numpy's Legendre series:
    (2 ell + 1) c_3 N^3 Re sum L_ell(q1_z / |q1|) d(q1) d(q2) d(q3) / (N^3 count)."""
    N = delta.shape[0]
    dh = np.fft.fftn(delta)
    smap = np_shell_map(N, edges)
    f = np.fft.fftfreq(N) * N
    modes = [np.argwhere(smap == s) for s in range(len(edges) - 1)]
    coef = np.zeros(ell + 1)
    coef[ell] = 1.0
    out = []
    for (k1, k2, k3), c in zip(bins, counts):
        a, b = modes[k1 - 1][:, None, :], modes[k2 - 1][None, :, :]
        q3 = (-(a + b)) % N
        ok = smap[q3[..., 0], q3[..., 1], q3[..., 2]] == k3 - 1
        qa = f[modes[k1 - 1]]
        mu = qa[:, 2] / np.sqrt((qa ** 2).sum(axis=1))
        w = np.polynomial.legendre.legval(mu, coef)[:, None]
        prod = (w * dh[a[..., 0], a[..., 1], a[..., 2]] * dh[b[..., 0], b[..., 1], b[..., 2]]
                * dh[q3[..., 0], q3[..., 1], q3[..., 2]])
        S = N ** 3 * np.real(prod[ok].sum())
        out.append((2 * ell + 1) * (L ** 3) ** 2 / float(N ** 3) ** 3 * S / (N ** 3 * c) if c > 0 else 0.0)
    return np.array(out)


@pytest.mark.parametrize("N,nshell,ell,kind", [(12, 3, 2, "lognormal"), (14, 4, 4, "white"), (12, 3, 0, "gaussian")])
def test_multipole_bispectrum_matches_enumeration(N, nshell, ell, kind):
    """The Legendre-weighted first leg (redshift-space multipoles) against enumeration of the triangles."""
    L, e = 100.0, fieldgen.unit_edges(nshell)
    d = fieldgen.field(kind, N, 3, np.float64)
    bins = oracle.enumerate_bins(e, 3)
    r = oracle.estimate_ell(d, L, e, 3, ell, bins)
    ref = multipole_brute_force(d, L, e, ell, bins, r["counts"])
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.max(np.abs(r["B"] - ref)) <= 1e-10 * scale
    if ell == 0:  # the monopole is the plain estimator
        m = oracle.estimate(d, L, e, 3, bins=bins)
        assert np.allclose(r["B"], m["B"], rtol=1e-12, atol=1e-12 * np.abs(m["B"]).max())


def test_multipole_estimator_rejects_odd_ell():
    with pytest.raises(RuntimeError):
        oracle.estimate_ell(np.zeros((12, 12, 12)), 1.0, fieldgen.unit_edges(3), 3, 1, [[1, 1, 1]])


def test_full_shape_trispectrum_reduces_to_the_angle_average():
    """Eq. Tkfull: summed over diagonal bins that cover every |q1 - q2| and |q1 - q3|, the full-shape sums
    and counts of each bin are the angle-averaged trispectrum's S_b and count_b."""
    N, L, e = 14, 100.0, fieldgen.unit_edges(3)
    d = fieldgen.field("lognormal", N, 8, np.float64)
    bins = oracle.enumerate_bins(e, 4, oracle.RULE_ALL_SORTED)
    ref = oracle.estimate(d, L, e, 4, bins=bins)
    de = np.concatenate([[0.0], np.arange(8) + 0.5])  # diagonals 0, then unit bins up to 7.5 > 2 * 3.5
    for b, S_b, c_b in zip(bins, ref["S"], ref["counts"]):
        r = oracle.trispectrum_full(d, L, e, b, de)
        assert r["counts"].sum() == c_b
        assert abs(r["S"].sum() - S_b) <= 1e-9 * max(1.0, np.abs(r["S"]).sum())
    assert ref["counts"].max() > 0


def test_full_shape_trispectrum_matches_enumeration():
    """The diagonal binning against an independent enumeration of the quadrilaterals with numpy."""
    N, L, e = 10, 100.0, fieldgen.unit_edges(2)
    d = fieldgen.field("lognormal", N, 9, np.float64)
    de = np.array([0.0, 0.5, 1.5, 2.5, 3.5, 5.0])
    k = (2, 2, 1, 1)
    dh = np.fft.fftn(d)
    smap = np_shell_map(N, e)
    f = np.fft.fftfreq(N) * N
    modes = [np.argwhere(smap == s) for s in range(2)]
    S = np.zeros((5, 5))
    A = np.zeros((5, 5))
    C = np.zeros((5, 5), dtype=np.int64)
    for q1 in modes[k[0] - 1]:
        for q2 in modes[k[1] - 1]:
            p1 = f[q1] - f[q2]
            j1 = np.searchsorted(de ** 2, p1 @ p1, side="right") - 1
            for q3 in modes[k[2] - 1]:
                q4 = (-(q1 + q2 + q3)) % N
                if smap[tuple(q4)] != k[3] - 1:
                    continue
                p2 = f[q1] - f[q3]
                j2 = np.searchsorted(de ** 2, p2 @ p2, side="right") - 1
                if not (0 <= j1 < 5 and 0 <= j2 < 5):
                    continue
                C[j1, j2] += 1
                S[j1, j2] += np.real(dh[tuple(q1)] * dh[tuple(q2)] * dh[tuple(q3)] * dh[tuple(q4)])
                A[j1, j2] += np.abs(dh[tuple(q1)] * dh[tuple(q2)] * dh[tuple(q3)] * dh[tuple(q4)])
    r = oracle.trispectrum_full(d, L, e, k, de)
    assert np.array_equal(r["counts"], C)
    assert np.allclose(r["S"], N ** 3 * S, rtol=1e-10, atol=1e-10 * np.abs(N ** 3 * S).max())
    norm = (L ** 3) ** 3 / float(N) ** 12
    assert np.allclose(r["scale"], np.where(C > 0, norm * A / np.maximum(C, 1), 0.0), rtol=1e-10, atol=0.0)
    assert np.all(np.abs(r["T"]) <= r["scale"] * (1 + 1e-12))
    assert C.sum() > 0 and np.count_nonzero(C) > 3


def test_counts_n2_are_mode_counts():
    N, e = 16, fieldgen.unit_edges(6)
    bins = oracle.enumerate_bins(e, 2, oracle.RULE_ALL_SORTED)
    r = oracle.estimate(np.zeros((N, N, N)), 1.0, e, 2, bins=bins)
    smap = np_shell_map(N, e)
    for (i, j), c in zip(bins, r["counts"]):
        assert c == (np.sum(smap == i - 1) if i == j else 0)


def test_triangle_counts_follow_eq_ntri():
    """Eq. Ntri (8 pi^2 k1 k2 k3 dk^3, 4 pi^2 when folded) is good to 10-20 % (Sec. 4.2)."""
    N, e = 48, fieldgen.unit_edges(12)
    r = oracle.estimate(np.zeros((N, N, N)), 1.0, e, 3)
    k = r["bins"].astype(float)
    ntri = np.where(k[:, 0] == k[:, 1] + k[:, 2], 4.0, 8.0) * np.pi ** 2 * k.prod(axis=1)
    ratio = r["counts"] / ntri
    big = k[:, 2] >= 5
    assert big.sum() > 20
    assert np.all((ratio[big] > 0.75) & (ratio[big] < 1.45))
    assert abs(np.median(ratio[big]) - 1.0) < 0.05


def test_quadrilateral_counts_follow_eq_nquad():
    """Eq. Nquad's clean form (8 pi^3 dk^4 k1 k2 k3 k4 (-k1 + k2 + k3 + 3 k4 - |k1 - k2 - k3 + k4|)) holds to
    about 40 % (Sec. 4.2); a loose band on the bins with k4 >= 3."""
    N, e = 32, fieldgen.unit_edges(7)
    r = oracle.estimate(np.zeros((N, N, N)), 1.0, e, 4)
    k = r["bins"].astype(float)
    nq = 8 * np.pi ** 3 * k.prod(axis=1) * (-k[:, 0] + k[:, 1] + k[:, 2] + 3 * k[:, 3]
                                            - np.abs(k[:, 0] - k[:, 1] - k[:, 2] + k[:, 3]))
    sel = (k[:, 3] >= 3) & (nq > 0)
    ratio = r["counts"][sel] / nq[sel]
    assert sel.sum() > 50
    assert np.all((ratio > 0.4) & (ratio < 1.6))
    assert abs(np.median(ratio) - 1.0) < 0.15


# --------------------------------------------------------------------------- product sums
@pytest.mark.parametrize("N,order,nshell,kind,seed", [(16, 3, 6, "white", 1), (18, 3, 5, "lognormal", 2),
                                                      (12, 4, 4, "white", 3), (16, 2, 6, "white", 4)])
def test_sums_match_direct_sampling(N, order, nshell, kind, seed):
    e = fieldgen.unit_edges(nshell)
    d = fieldgen.field(kind, N, seed, np.float64)
    r = oracle.estimate(d, 1.0, e, order)
    S, cnt = oracle.direct_sample(d, e, order, r["bins"])
    assert np.array_equal(cnt, r["counts"])
    tol = 1e-12 * r["scale"] * N ** 3 * r["counts"]
    assert np.all(np.abs(S - r["S"]) <= tol + 1e-300)
    assert r["imag_max"] < 1e-12


def test_power_spectrum_textbook():
    """n = 2 reduces to P(k) = V/N^6 <|dhat(q)|^2> over the shell (App. A with n = 2)."""
    N, L, e = 24, 300.0, fieldgen.unit_edges(9)
    d = fieldgen.field("gaussian", N, 11, np.float64)
    r = oracle.estimate(d, L, e, 2, bins=np.array([[i, i] for i in range(1, 10)], dtype=np.int32))
    dk = np.fft.fftn(d)
    smap = np_shell_map(N, e)
    for s in range(9):
        sel = smap == s
        pk = L ** 3 / N ** 6 * np.mean(np.abs(dk[sel]) ** 2)
        assert r["counts"][s] == sel.sum()
        assert abs(r["B"][s] - pk) <= 1e-12 * pk


def _wave_field(N, waves):
    return fieldgen.plane_waves(N, waves)


def test_plane_waves_bispectrum_closed_form():
    N, L = 16, 200.0
    e = fieldgen.unit_edges(6)
    q1, q2 = np.array([3, 0, 0]), np.array([0, 2, 0])
    q3 = -(q1 + q2)  # |q3|^2 = 13 -> shell 4
    A = [1.3, 0.7, 0.9]
    phi = [0.4, -1.1, 2.0]
    d = _wave_field(N, [(q1, A[0], phi[0]), (q2, A[1], phi[1]), (q3, A[2], phi[2])])
    r = oracle.estimate(d, L, e, 3, rule=oracle.RULE_ALL_SORTED)
    n3 = N ** 3
    S_closed = n3 * 2.0 * (n3 / 2.0) ** 3 * A[0] * A[1] * A[2] * np.cos(sum(phi))
    idx = [i for i, b in enumerate(r["bins"]) if tuple(b) == (4, 3, 2)][0]
    assert abs(r["S"][idx] - S_closed) < 1e-10 * abs(S_closed)
    _, cnt = oracle.direct_sample(None, e, 3, r["bins"][idx:idx + 1], N=N)
    B_closed = (L ** 3) ** 2 / n3 ** 3 * S_closed / (n3 * cnt[0])
    assert abs(r["B"][idx] - B_closed) < 1e-10 * abs(B_closed)
    others = np.delete(r["S"], idx)
    assert np.abs(others).max() < 1e-9 * abs(S_closed)


def test_plane_waves_trispectrum_closed_forms():
    N, L = 16, 200.0
    e = fieldgen.unit_edges(6)
    q1, q2, q3 = np.array([2, 0, 0]), np.array([0, 3, 0]), np.array([0, 0, 4])
    q4 = -(q1 + q2 + q3)  # |q4|^2 = 29 -> shell 5
    A = [1.1, 0.8, 1.4, 0.6]
    phi = [0.3, 1.2, -0.5, 0.9]
    d = _wave_field(N, [(q1, A[0], phi[0]), (q2, A[1], phi[1]), (q3, A[2], phi[2]), (q4, A[3], phi[3])])
    want = np.array([[5, 4, 3, 2], [3, 3, 2, 2]], dtype=np.int32)
    r = oracle.estimate(d, L, e, 4, bins=want)
    n3 = N ** 3
    connected = n3 * 2.0 * (n3 / 2.0) ** 4 * np.prod(A) * np.cos(sum(phi))
    paired = n3 * 4.0 * (n3 / 2.0) ** 4 * A[0] ** 2 * A[1] ** 2
    assert abs(r["S"][0] - connected) < 1e-10 * abs(connected)
    assert abs(r["S"][1] - paired) < 1e-10 * abs(paired)


def test_iid_skewed_noise_normalisation():
    """iid noise with third cumulant k3 has B(k1,k2,k3) = k3 (V/N^3)^2 in every bin (Sec. 1 convention)."""
    N, L, e = 32, 500.0, fieldgen.unit_edges(10)
    p = 0.2
    k3 = p * (1 - p) * (1 - 2 * p)
    vals = []
    for seed in range(6):
        d = (np.random.default_rng(100 + seed).random((N, N, N)) < p).astype(float) - p
        r = oracle.estimate(d, L, e, 3)
        vals.append(r["B"] / (L ** 3 / N ** 3) ** 2)
    vals = np.array(vals)
    mean, err = vals.mean(), vals.std() / np.sqrt(vals.size)
    assert abs(mean - k3) < 4 * err + 0.02 * k3
    assert err < 0.15 * k3


def test_gaussian_mean_bispectrum_near_zero():
    N, e = 24, fieldgen.unit_edges(8)
    ratios = []
    for seed in range(8):
        d = fieldgen.field("gaussian", N, 500 + seed, np.float64)
        r = oracle.estimate(d, 1.0, e, 3)
        ratios.append(r["R"] / r["scale"])
    ratios = np.array(ratios)
    mean, err = ratios.mean(), ratios.std() / np.sqrt(ratios.size)
    assert abs(mean) < 4 * err


def test_lognormal_bispectrum_is_positive_on_average():
    """A lognormal field is positively skewed: its mean bispectrum is positive (sanity of the sign)."""
    N, e = 24, fieldgen.unit_edges(8)
    d = fieldgen.field("lognormal", N, 9, np.float64)
    r = oracle.estimate(d, 1.0, e, 3)
    assert np.mean(r["B"]) > 0


# --------------------------------------------------------------------------- adjoint
@pytest.mark.parametrize("order,nshell", [(3, 4), (4, 3)])
def test_gradient_matches_central_differences(order, nshell):
    N, L = 12, 100.0
    e = fieldgen.unit_edges(nshell)
    rng = np.random.default_rng(42 + order)
    d = rng.standard_normal((N, N, N))
    r = oracle.estimate(d, L, e, order)
    w = rng.standard_normal(len(r["bins"]))
    g = oracle.gradient(d, L, e, order, r["bins"], r["counts"], w)

    def loss(x):
        return float(np.dot(w, oracle.estimate(x, L, e, order, bins=r["bins"])["B"]))

    h = 1e-3
    for v in rng.choice(N ** 3, size=6, replace=False):
        i = np.unravel_index(v, d.shape)
        dp, dm = d.copy(), d.copy()
        dp[i] += h
        dm[i] -= h
        fd = (loss(dp) - loss(dm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (abs(g[i]) + np.abs(g).max() * 1e-3)


def test_nonzero_counts_are_the_polygon_rule_widened_by_one_shell():
    """Unit-width shells centred on integers: a sorted triple has closed triangles exactly when
    k1 <= k2 + k3 + 1 (the polygon inequality of App. B on the centres, widened by the shells' width), so
    the nonzero-count set is that rule (25,424 triples at 64 shells) and every sorted triple outside it
    counts zero."""
    e = fieldgen.unit_edges(12)
    b = oracle.enumerate_bins(e, 3, oracle.RULE_ALL_SORTED)
    c = oracle.counts_exact(48, e, 3, b)
    assert np.array_equal(c > 0, b[:, 0] <= b[:, 1] + b[:, 2] + 1)
