"""The library's host tables against the oracle, with no GPU.

poly_diag_host_tables runs the host part of plan creation (argument checks,
bins, shell line tables, contraction tiles) without touching a device.  These
tests check, for orders 2 to 6, several shell layouts and the multipole plans:
- the bins equal the oracle's enumeration (the ordering used throughout, with
  the polygon rule of App. B on the shell centres, or every sorted tuple);
- every bin's slot names a tile cell whose row and column factors are exactly
  the bin's shells, first legs in the row and the rest in the column, the first
  leg on the Legendre-weighted slot for a multipole plan; no two bins share a
  slot; the cell lies inside the tile and inside a region its mask marks;
- the line tables of every shell cover exactly the oracle's modes of that shell
  in the half space kz >= 0 (Sec. 2: q in the shell, q = 0 excluded), and the
  extra slot covers their union.
"""
import ctypes

import numpy as np
import pytest

import fieldgen
import oracle
import paper_1904_11055_gb300 as ps
from paper_1904_11055_gb300 import build as psbuild

RA = {2: 1, 3: 2, 4: 2, 5: 2, 6: 3}  # first legs held by a tile row
STATUS = {v: k for k, v in ps.STATUS.items()}


@pytest.fixture(scope="module")
def lib():
    psbuild.build()
    L = ps.load_library()
    P = ctypes.c_void_p
    L.poly_diag_host_tables.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_uint, ctypes.c_int,
                                        P, P, P, P, P, P, P, P, P]
    L.poly_diag_host_tables.restype = ctypes.c_int
    return L


def host_tables(lib, N, order, edges, flags=0, ell=0):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    ns = e.size - 1
    sizes = np.zeros(7, dtype=np.int64)
    args = (N, order, e.ctypes.data, ns, flags, ell)
    rc = lib.poly_diag_host_tables(*args, sizes.ctypes.data, *([None] * 8))
    if rc:
        return rc, None
    nb, nt, nfid, nr, nc, nl, noff = (int(v) for v in sizes)
    t = dict(bins=np.zeros((nb, order), np.int32), tiles=np.zeros((nt, 8), np.int32),
             field_ids=np.zeros(nfid, np.int32), rowf=np.zeros((nr, 4), np.int16), colf=np.zeros((nc, 4), np.int16),
             slot=np.zeros(nb, np.int64), lines=np.zeros((nl, 4), np.int16), line_off=np.zeros(noff, np.int32))
    ptrs = [t[k].ctypes.data for k in ("bins", "tiles", "field_ids", "rowf", "colf", "slot", "lines", "line_off")]
    assert lib.poly_diag_host_tables(*args, sizes.ctypes.data, *ptrs) == 0
    return 0, t


def check_tiles(t, order, nshell, shift):
    ra = RA[order]
    tiles, fid, rowf, colf = t["tiles"], t["field_ids"], t["rowf"], t["colf"]
    assert np.all(tiles[:, 5] <= 128)  # fields one tile may reference
    assert np.unique(t["slot"]).size == t["slot"].size
    for b, legs in enumerate(t["bins"]):
        tile, cell = divmod(int(t["slot"][b]), 64 * 64)
        r, c = divmod(cell, 64)
        row_off, nrow, col_off, ncol, foff, nf, mask, _ = tiles[tile]
        assert r < nrow and c < ncol
        assert (int(mask) >> ((r // 32) * 4 + c // 16)) & 1
        rf = [int(v) for v in rowf[row_off + r] if v >= 0]
        cf = [int(v) for v in colf[col_off + c] if v >= 0]
        assert all(v < nf for v in rf + cf)
        want = [int(k) - 1 for k in legs]
        want[0] += shift
        assert [int(fid[foff + v]) for v in rf] == want[:ra]
        assert [int(fid[foff + v]) for v in cf] == want[ra:]
    assert t["field_ids"].max() < nshell + shift


def line_modes(lines, lo, hi):
    out = set()
    for ky, kz, a, b in lines[lo:hi]:
        for ax in range(int(a), int(b) + 1):
            out.update({(ax, int(ky), int(kz)), (-ax, int(ky), int(kz))})
    return out


def oracle_modes(N, edges):
    smap = oracle.shell_map(N, edges)
    f = np.where(np.arange(N) < (N + 1) // 2, np.arange(N), np.arange(N) - N)
    per = []
    for s in range(len(edges) - 1):
        a, b, c = np.nonzero(smap == s)
        keep = f[c] >= 0
        per.append(set(zip(f[a][keep].tolist(), f[b][keep].tolist(), f[c][keep].tolist())))
    return per


LAYOUTS = {
    "unit12": fieldgen.unit_edges(12),
    "wide1.5x8": fieldgen.unit_edges(8, 1.5),
    "log9": np.concatenate([[0.5], np.geomspace(1.5, 14.0, 9)]),
}


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("layout", sorted(LAYOUTS))
@pytest.mark.parametrize("flags,rule", [(0, oracle.RULE_POLYGON), (ps.POLY_BINS_ALL_SORTED, oracle.RULE_ALL_SORTED)])
def test_bins_and_tiles(lib, order, layout, flags, rule):
    e = LAYOUTS[layout]
    N = 96
    rc, t = host_tables(lib, N, order, e, flags | ps.POLY_ALLOW_ALIAS)
    assert rc == 0
    assert np.array_equal(t["bins"], oracle.enumerate_bins(e, order, rule))
    check_tiles(t, order, len(e) - 1, 0)


@pytest.mark.parametrize("order,ell", [(3, 2), (3, 4), (4, 2), (5, 2)])
def test_multipole_tiles_read_the_weighted_first_leg(lib, order, ell):
    e = fieldgen.unit_edges(7)
    rc, t = host_tables(lib, 64, order, e, 0, ell)
    assert rc == 0
    assert np.array_equal(t["bins"], oracle.enumerate_bins(e, order))
    check_tiles(t, order, 7, 7)


@pytest.mark.parametrize("N,layout", [(32, "unit12"), (48, "wide1.5x8"), (48, "log9")])
def test_line_tables_cover_each_shell_exactly(lib, N, layout):
    e = LAYOUTS[layout]
    rc, t = host_tables(lib, N, 2, e)
    assert rc == 0
    ns, off = len(e) - 1, t["line_off"]
    assert off.size == ns + 2 and off[0] == 0 and np.all(np.diff(off) >= 0)
    ref = oracle_modes(N, e)
    for s in range(ns):
        assert line_modes(t["lines"], off[s], off[s + 1]) == ref[s], f"shell {s}"
    assert line_modes(t["lines"], off[ns], off[ns + 1]) == set().union(*ref)


@pytest.mark.parametrize("kwargs,status", [
    (dict(N=64, order=7), STATUS["POLY_ERR_UNSUPPORTED"]),
    (dict(N=62, order=3), STATUS["POLY_ERR_UNSUPPORTED"]),
    (dict(N=16, order=3), STATUS["POLY_ERR_ALIAS"]),
    (dict(N=64, order=3, ell=3), STATUS["POLY_ERR_ARG"]),
    (dict(N=64, order=3, edges=[0.5, 2.5, 1.5]), STATUS["POLY_ERR_ARG"]),
])
def test_host_checks_match_plan_creation(lib, kwargs, status):
    kw = dict(edges=fieldgen.unit_edges(6), flags=0, ell=0) | kwargs
    rc, _ = host_tables(lib, kw["N"], kw["order"], kw["edges"], kw["flags"], kw["ell"])
    assert rc == status
