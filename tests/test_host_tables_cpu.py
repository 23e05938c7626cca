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
    return ps.load_library()


def host_tables(lib, N, order, edges, flags=0, ell=0):
    P = ctypes.c_void_p
    lib.poly_diag_host_tables.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_uint, ctypes.c_int,
                                          P, P, P, P, P, P, P, P, P]
    lib.poly_diag_host_tables.restype = ctypes.c_int
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
# edges whose squares land on (or a rounding away from) integers |q|^2: ties decided by the exact comparison
TIES = np.sqrt(np.array([1.0, 5.0, 9.0, 20.0, 33.0, 50.0, 51.0, 98.0]))


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


@pytest.mark.parametrize("N,layout", [(32, "unit12"), (48, "wide1.5x8"), (48, "log9"), (32, "ties"),
                                      (128, "unit40"), (96, "wide1.5x20"), (256, "unit64")])
def test_line_tables_cover_each_shell_exactly(lib, N, layout):
    e = {"ties": TIES, "unit40": fieldgen.unit_edges(40), "wide1.5x20": fieldgen.unit_edges(20, 1.5),
         "unit64": fieldgen.unit_edges(64)}.get(layout, None)
    e = LAYOUTS[layout] if e is None else e
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
    (dict(N=256, order=5, edges=fieldgen.unit_edges(120), flags=ps.POLY_ALLOW_ALIAS), STATUS["POLY_ERR_UNSUPPORTED"]),
])
def test_host_checks_match_plan_creation(lib, kwargs, status):
    kw = dict(edges=fieldgen.unit_edges(6), flags=0, ell=0) | kwargs
    rc, _ = host_tables(lib, kw["N"], kw["order"], kw["edges"], kw["flags"], kw["ell"])
    assert rc == status


# ------------------------------------------------------------------ tensor-core contraction tables

def tc_tables(lib, N, order, edges, sms=152, max_mt=4, cta_mult=4, flags=0, ell=0):
    fn = lib.poly_diag_tc_tables
    P = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int] + [P] * 8
    fn.restype = ctypes.c_int
    e = np.ascontiguousarray(edges, dtype=np.float64)
    sizes = np.zeros(9, dtype=np.int64)
    args = (N, order, e.ctypes.data, e.size - 1, flags, ell, sms, max_mt, cta_mult)
    rc = fn(*args, sizes.ctypes.data, *([None] * 7))
    if rc:
        return rc, None
    nb, nc, ng, nm, nr, nrow, ncol, teams, slot_cap = (int(v) for v in sizes)
    t = dict(ctas=np.zeros((nc, 3), np.int64), groups=np.zeros((ng, 5), np.int32), mtiles=np.zeros((nm, 3), np.int32),
             runs=np.zeros((nr, 4), np.int32), rowf=np.zeros((nrow, 3), np.int16), colf=np.zeros((ncol, 3), np.int16),
             binmap=np.zeros((nb, 3), np.int32))
    ptrs = [t[k].ctypes.data for k in ("ctas", "groups", "mtiles", "runs", "rowf", "colf", "binmap")]
    assert fn(*args, sizes.ctypes.data, *ptrs) == 0
    t["teams"], t["slot_cap"] = teams, slot_cap
    return 0, t


def check_pipeline_teams(t):
    """Producer teams never outnumber a group's A/B slots: a team's parity wait on a slot's barrier is
    unambiguous only while the slot's previous use is known complete, which its own previous wait implies
    when teams <= slots (the kernel also caps its teams by the slots of its group)."""
    g = t["groups"]
    acc = (g[:, 4] + 31) // 32 * 32
    slots = np.minimum(t["slot_cap"], (512 - acc) // (g[:, 1] * 32))
    assert t["teams"] in (2, 3) and 2 <= t["slot_cap"] <= 4 and slots.min() >= 2
    assert t["teams"] == (3 if slots.min() >= 3 else 2)


def factor_wavefronts(t, which):
    """Shared-memory wavefronts of one 16-byte factor load (the row factor `which`: 0 first, 1 second)
    per producer warp, averaged over the M tiles' warps: a quarter warp reads 8 lanes in one wavefront
    unless two of its lanes read different staged rows equal modulo 8 (the 128-byte swizzle puts those
    in the same banks)."""
    rowf, total, n = t["rowf"], 0, 0
    for r0, _, _ in t["mtiles"]:
        for q in range(4):
            rows = rowf[r0 + 32 * q:r0 + 32 * q + 32, which]
            for qq in range(4):
                by = {}
                for r in set(rows[8 * qq:8 * qq + 8].tolist()):
                    by.setdefault(r & 7, set()).add(r)
                total += max(len(v) for v in by.values())
            n += 1
    return total / n


def check_tc_tables(t, bins, N, nshell, max_mt, shift=0):
    """shift: the first row factor's slot offset (nshell for a multipole plan's weighted fields)."""
    order = bins.shape[1]
    ra = 3 if order >= 6 else (2 if order >= 3 else 1)
    ctas, groups, mtiles, runs, rowf, colf, bm = (t[k] for k in ("ctas", "groups", "mtiles", "runs", "rowf", "colf",
                                                                "binmap"))
    ng, nchunks = len(groups), (N ** 3 + 31) // 32
    # blocks: each group's blocks are contiguous and their chunk ranges tile [0, nchunks)
    first, count = np.zeros(ng, np.int64), np.zeros(ng, np.int64)
    for g in range(ng):
        idx = np.nonzero(ctas[:, 0] == g)[0]
        assert idx.size >= 1 and np.all(np.diff(idx) == 1)
        first[g], count[g] = idx[0], idx.size
        c = ctas[idx]
        assert c[0, 1] == 0 and c[-1, 2] == nchunks and np.all(c[1:, 1] == c[:-1, 2]) and np.all(c[:, 2] > c[:, 1])
    # accumulator columns of each group: which M tile and local column each one holds (no column twice)
    owner = []
    for g, (mt_off, nmt, col_off, ncol, acc_cols) in enumerate(groups):
        assert 1 <= nmt <= max_mt and ncol % 16 == 0 and 0 < ncol <= 256 and 0 < acc_cols <= 256
        tab = -np.ones((256, 2), np.int64)
        for m in range(mt_off, mt_off + nmt):
            row_off, run_off, nrun = mtiles[m]
            assert 1 <= nrun <= 4
            rf = rowf[row_off:row_off + 128]
            assert np.all((rf[:, 0] >= shift) & (rf[:, 0] < nshell + shift))  # padding rows repeat a real row
            assert np.all(rf[:, 1] < nshell) and np.all((rf[:, 1] >= 0) == (ra >= 2))
            assert np.all(rf[:, 2] < nshell) and np.all((rf[:, 2] >= 0) == (ra == 3))
            for n0, nn, acc, mloc in runs[run_off:run_off + nrun]:
                assert mloc == m - mt_off and nn % 16 == 0 and n0 % 16 == 0 and n0 + nn <= ncol
                assert acc + nn <= acc_cols and np.all(tab[acc:acc + nn, 0] < 0)
                tab[acc:acc + nn, 0] = m
                tab[acc:acc + nn, 1] = col_off + n0 + np.arange(nn)
        owner.append(tab)
    owner = np.stack(owner)
    # every bin: one group's blocks, a slot inside it, the right row and column factors
    g = ctas[bm[:, 0], 0]
    assert np.all(bm[:, 0] == first[g]) and np.all(bm[:, 1] == count[g])
    acc_col, row = bm[:, 2] // 128, bm[:, 2] % 128
    assert np.all(acc_col < groups[g, 4])
    m, col = owner[g, acc_col, 0], owner[g, acc_col, 1]
    assert np.all(m >= 0)
    assert np.all(col < groups[g, 2] + groups[g, 3])
    rf = rowf[mtiles[m, 0] + row].astype(np.int64)
    cf = colf[col].astype(np.int64)
    legs = bins.astype(np.int64) - 1
    pad = -np.ones(len(bins), np.int64)
    want_row = np.stack([legs[:, 0] + shift, legs[:, 1] if ra >= 2 else pad, legs[:, 2] if ra == 3 else pad], 1)
    rest = legs[:, ra:]
    want_col = np.stack([rest[:, 0], rest[:, 1] if rest.shape[1] > 1 else pad,
                         rest[:, 2] if rest.shape[1] > 2 else pad], 1)
    assert np.array_equal(rf, want_row) and np.array_equal(cf, want_col)
    key = g * (256 * 128) + bm[:, 2]
    assert np.unique(key).size == key.size


@pytest.mark.parametrize("max_mt", [2, 3, 4])
@pytest.mark.parametrize("cta_mult", [1, 2, 4, 6, 8])
def test_tc_tables_bispectrum_256cube_64shells(lib, max_mt, cta_mult):
    """The benchmark's plan (256^3, 64 unit shells) in every contraction shape the tuner may choose."""
    e = fieldgen.unit_edges(64)
    rc, t = tc_tables(lib, 256, 3, e, 152, max_mt, cta_mult)
    assert rc == 0
    check_tc_tables(t, oracle.enumerate_bins(e, 3), 256, 64, max_mt)
    check_pipeline_teams(t)
    if max_mt >= 3:
        assert t["teams"] == 3  # groups of three M tiles: three slots beside at most 176 accumulator columns
    # every factor load of the producers is a conflict-free broadcast: four wavefronts per 16-byte load
    assert factor_wavefronts(t, 0) == 4.0 and factor_wavefronts(t, 1) == 4.0


@pytest.mark.parametrize("N,order,nshell,width", [(256, 4, 32, 1.5), (96, 4, 10, 2.0), (48, 3, 12, 1.0),
                                                  (64, 2, 30, 1.0), (128, 3, 40, 1.0), (128, 5, 16, 1.0),
                                                  (48, 5, 8, 1.0), (48, 6, 6, 1.0), (128, 6, 8, 1.0)])
@pytest.mark.parametrize("sms", [152, 20])
def test_tc_tables_other_plans(lib, N, order, nshell, width, sms):
    """The trispectrum (its pair columns split into several instances), the power spectrum, small grids."""
    e = fieldgen.unit_edges(nshell, width)
    rc, t = tc_tables(lib, N, order, e, sms)
    assert rc == 0
    check_tc_tables(t, oracle.enumerate_bins(e, order), N, nshell, 4)
    check_pipeline_teams(t)
    if (N, order, nshell) == (256, 4, 32):
        assert t["teams"] == 2  # the pair columns' B buffers leave shared memory for two slots


@pytest.mark.parametrize("N,order,nshell,ell", [(256, 3, 64, 2), (48, 3, 12, 4), (32, 4, 6, 2), (64, 2, 20, 2)])
@pytest.mark.parametrize("max_mt", [2, 4])
def test_tc_tables_multipole_plans(lib, N, order, nshell, ell, max_mt):
    """Multipole plans: each bin's row reads the weighted field of its first leg (slot k1 - 1 + nshell) and
    the plain field of its second; columns and every other invariant as for the monopole."""
    e = fieldgen.unit_edges(nshell)
    rc, t = tc_tables(lib, N, order, e, 152, max_mt, 4, 0, ell)
    assert rc == 0
    check_tc_tables(t, oracle.enumerate_bins(e, order), N, nshell, max_mt, shift=nshell)
    assert t["groups"][:, 4].max() <= 256
    check_pipeline_teams(t)


@pytest.mark.parametrize("kwargs,status", [
    (dict(order=7), STATUS["POLY_ERR_UNSUPPORTED"]),
    (dict(sms=0), STATUS["POLY_ERR_ARG"]),
    (dict(N=16), STATUS["POLY_ERR_ALIAS"]),
])
def test_tc_tables_refuse_what_plan_creation_refuses(lib, kwargs, status):
    kw = dict(N=64, order=3, sms=152) | kwargs
    rc, _ = tc_tables(lib, kw["N"], kw["order"], fieldgen.unit_edges(6), kw["sms"])
    assert rc == status


# ------------------------------------------------------------------ adjoint tables

def adj_tables(lib, N, order, edges, prec, sms=152):
    fn = lib.poly_diag_adj_tables
    P = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_int] + [P] * 8
    fn.restype = ctypes.c_int
    e = np.ascontiguousarray(edges, dtype=np.float64)
    ns = e.size - 1
    sizes = np.zeros(10, dtype=np.int64)
    args = (N, order, e.ctypes.data, ns, 0, ps.PRECISIONS[prec], sms)
    assert fn(*args, sizes.ctypes.data, *([None] * 7)) == 0
    nent, neb, ng, nch = (int(v) for v in sizes[:4])
    t = dict(moff=np.zeros(ns + 1, np.int32), ent=np.zeros((nent, 3), np.int16), eoff=np.zeros(nent + 1, np.int32),
             ebins=np.zeros(neb, np.int32), groups=np.zeros((ng, 6), np.int32), chunks=np.zeros(nch, np.int32),
             pos=np.zeros(nent if ng else 0, np.int32))
    ptrs = [t[k].ctypes.data for k in ("moff", "ent", "eoff", "ebins", "groups", "chunks", "pos")]
    assert fn(*args, sizes.ctypes.data, *ptrs) == 0
    t["kp"], t["acap"], t["b_total"] = int(sizes[4]), int(sizes[5]), int(sizes[6])
    return t


def check_entries(t, bins, nshell):
    """Every (bin, position of m) pair is listed exactly once, under the entry (m, other shells sorted)."""
    order = bins.shape[1]
    moff, ent, eoff, ebins = t["moff"], t["ent"], t["eoff"], t["ebins"]
    assert moff[0] == 0 and moff[-1] == len(ent) and np.all(np.diff(moff) >= 0)
    assert eoff[0] == 0 and eoff[-1] == len(ebins) and np.all(np.diff(eoff) >= 1)
    got = {}
    for m in range(nshell):
        for e in range(moff[m], moff[m + 1]):
            key = (m,) + tuple(int(v) for v in ent[e][:order - 1])
            assert key not in got and np.all(ent[e][order - 1:] == -1)
            got[key] = sorted(ebins[eoff[e]:eoff[e + 1]].tolist())
    want = {}
    for b, legs in enumerate(bins.astype(int) - 1):
        for tpos in range(order):
            rest = sorted(np.delete(legs, tpos).tolist())
            want.setdefault((int(legs[tpos]),) + tuple(rest), []).append(b)
    assert got == {k: sorted(v) for k, v in want.items()}


def check_at_tables(t, nshell):
    """Tensor-core adjoint: each group's chunks run over its m's in order, one chunk per (m, j block) that
    holds an entry; every entry's weight sits at its own place of its group's B (K-major, 8 x 8 core
    matrices), inside a K block that the group's mask marks."""
    ent, moff, groups, chunks, pos, kp = t["ent"], t["moff"], t["groups"], t["chunks"], t["pos"], t["kp"]
    assert kp % 32 == 0 and nshell <= kp and t["acap"] % 32 == 0
    where = {}
    next_off, ms_seen = 0, []
    for g, (coff, nch, hsplit, boff, km0, km1) in enumerate(groups):
        assert coff == (groups[g - 1, 0] + groups[g - 1, 1] if g else 0) and 0 < nch <= t["acap"] // 16
        assert boff == next_off
        next_off += nch * 16 * kp * 2
        c = chunks[coff:coff + nch]
        jb, m, last = c & 0xFF, (c >> 8) & 0xFF, (c >> 16) & 1
        assert np.all(np.diff(m) >= 0)
        assert np.array_equal(last.astype(bool), np.append(m[1:] != m[:-1], True))
        assert 0 <= hsplit <= nch and (hsplit in (0, nch) or m[hsplit - 1] != m[hsplit])
        ms_seen += sorted(set(m.tolist()))
        for q in range(nch):
            assert (int(m[q]), int(jb[q])) not in where
            where[(int(m[q]), int(jb[q]))] = (g, q)
    assert next_off == t["b_total"] and ms_seen == sorted(set(ms_seen))
    m_of = np.repeat(np.arange(nshell), np.diff(moff))
    need = {(int(m_of[e]), int(ent[e, 1]) // 16) for e in range(len(ent))}
    assert set(where) == need  # a chunk for every (m, j block) with an entry, and no other
    assert np.unique(pos).size == pos.size and np.all(pos % 2 == 0)
    for e in range(len(ent)):
        k, j = int(ent[e, 0]), int(ent[e, 1])
        assert k <= j
        g, q = where[(int(m_of[e]), j // 16)]
        off = int(pos[e]) - int(groups[g, 3])
        n = (off // (kp * 16)) * 8 + (off % 128) // 16
        kk = ((off % (kp * 16)) // 128) * 8 + (off % 16) // 2
        assert (n, kk) == (q * 16 + j % 16, k)
        assert (int(groups[g, 4 + n // 256]) >> (k // 16)) & 1


@pytest.mark.parametrize("N,order,nshell,width,prec", [
    (256, 3, 64, 1.0, "split_bf16"), (96, 3, 30, 1.0, "split_bf16"), (48, 3, 14, 1.0, "split_bf16"),
    (128, 3, 40, 1.0, "fp32"), (64, 2, 16, 1.0, "fp64"), (256, 4, 32, 1.5, "fp32"), (64, 4, 10, 1.5, "split_bf16"),
])
def test_adjoint_tables(lib, N, order, nshell, width, prec):
    e = fieldgen.unit_edges(nshell, width)
    t = adj_tables(lib, N, order, e, prec)
    check_entries(t, oracle.enumerate_bins(e, order), nshell)
    if order == 3 and prec == "split_bf16":
        assert len(t["groups"]) > 0
        check_at_tables(t, nshell)
    else:
        assert len(t["groups"]) == 0


# ------------------------------------------------------------------ the count wedge

def count_wedge(lib, N):
    fn = lib.poly_diag_count_wedge
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    n = ctypes.c_int64(0)
    assert fn(N, ctypes.byref(n), None, None) == 0
    cells, w = np.zeros(n.value, np.int32), np.zeros(n.value, np.float64)
    assert fn(N, ctypes.byref(n), cells.ctypes.data, w.ctypes.data) == 0
    return cells, w


@pytest.mark.parametrize("N", [6, 16, 24, 32])
def test_count_wedge_weights_are_orbit_sizes(lib, N):
    """Each cell of the wedge stands for its orbit under the cube's 48 symmetries (per-axis x -> -x mod N,
    axis permutations): the orbits partition the grid and the weights are their sizes."""
    cells, w = count_wedge(lib, N)
    g = np.indices((N, N, N)).reshape(3, -1)
    rep = np.sort(np.minimum(g, N - g), axis=0)  # fold each axis, then order the axes
    lin = (rep[0] * N + rep[1]) * N + rep[2]
    u, cnt = np.unique(lin, return_counts=True)
    order = np.argsort(cells)
    assert np.array_equal(cells[order], u) and np.array_equal(w[order], cnt.astype(np.float64))
    assert w.sum() == N ** 3


def test_count_wedge_reproduces_the_full_count_sum(lib):
    """The oracle's counting fields (16^3, 5 shells) summed over the wedge with its weights give the
    same products as the sum over every cell, for every bin (the symmetry the wedge relies on)."""
    N, e = 16, fieldgen.unit_edges(5)
    iota, _ = oracle.shell_fields(N, e, np.arange(5))
    cells, w = count_wedge(lib, N)
    flat = iota.reshape(5, -1)
    for b in oracle.enumerate_bins(e, 3, oracle.RULE_ALL_SORTED) - 1:
        full = np.prod(flat[b], axis=0).sum()
        wedge = (np.prod(flat[b][:, cells], axis=0) * w).sum()
        assert abs(full - wedge) <= 1e-9 * max(1.0, abs(full))


# ------------------------------------------------------------------ bins whose closures may wrap around the grid

def bin_wraps(lib, N, order, edges, flags=ps.POLY_ALLOW_ALIAS):
    fn = lib.poly_diag_bin_wraps
    P = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_uint, P, P]
    fn.restype = ctypes.c_int
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nb = ctypes.c_int64(0)
    assert fn(N, order, e.ctypes.data, e.size - 1, flags, ctypes.byref(nb), None) == 0
    out = np.zeros(nb.value, np.uint8)
    assert fn(N, order, e.ctypes.data, e.size - 1, flags, ctypes.byref(nb), out.ctypes.data) == 0
    return out.astype(bool)


@pytest.mark.parametrize("N,order,nshell,big", [(16, 3, 6, 32), (16, 4, 4, 32), (24, 3, 9, 48)])
def test_bin_wraps_cover_every_bin_whose_periodic_count_differs(lib, N, order, nshell, big):
    """The oracle's counts on the N grid (closures mod N) against those on a grid too large to wrap (exact
    closures): they differ only in flagged bins, and the flag is not vacuous (some flagged bin differs)."""
    e = fieldgen.unit_edges(nshell)
    bins = oracle.enumerate_bins(e, order)
    wraps = bin_wraps(lib, N, order, e)
    periodic, exact = oracle.counts_exact(N, e, order, bins), oracle.counts_exact(big, e, order, bins)
    differ = periodic != exact
    assert not np.any(differ & ~wraps)
    assert np.any(differ & wraps)


def test_bin_wraps_of_the_96cube_mocks(lib):
    """The 96^3 realisations of the mock workload (32 unit shells, n = 3 = N / 32): only (32, 32, 32) may
    wrap, and it does (its periodic count exceeds the exact one)."""
    e = fieldgen.unit_edges(32)
    bins = oracle.enumerate_bins(e, 3)
    wraps = bin_wraps(lib, 96, 3, e)
    assert [tuple(b) for b in bins[wraps]] == [(32, 32, 32)]
    b = bins[wraps]
    assert oracle.counts_exact(96, e, 3, b)[0] > oracle.counts_exact(128, e, 3, b)[0]


def test_no_wraps_without_the_alias_flag(lib):
    e = fieldgen.unit_edges(20)
    assert not bin_wraps(lib, 64, 3, e, 0).any()


def scanned_lines(edges, s, K):
    """Shell s's line table by testing every |kx| of every (ky, kz >= 0) line (numpy, exact integer |q|^2)."""
    ky, kz, kx = np.meshgrid(np.arange(-K, K + 1), np.arange(K + 1), np.arange(K + 1), indexing="ij")
    q2 = (ky * ky + kz * kz + kx * kx).astype(np.float64)
    m = (edges[s] * edges[s] <= q2) & (q2 < edges[s + 1] * edges[s + 1]) & (q2 != 0)
    hit = m.any(axis=2)
    a, b = m.argmax(axis=2), K - m[:, :, ::-1].argmax(axis=2)
    sel = np.nonzero(hit.reshape(-1))[0]
    return np.stack([ky[:, :, 0].reshape(-1)[sel], kz[:, :, 0].reshape(-1)[sel], a.reshape(-1)[sel],
                     b.reshape(-1)[sel]], axis=1)


def test_line_runs_equal_a_scan_of_every_kx_on_random_edges(lib):
    """Each line's |kx| run is computed from its ends, not by testing every |kx|: the tables equal, line for
    line, a scan of every |kx| on 60 random edge sets (unit shells at random offsets, squared edges on
    integers, random widths, edges from 0)."""
    rng = np.random.default_rng(2024)
    for trial in range(60):
        kind, ns = trial % 4, int(rng.integers(1, 8))
        if kind == 0:
            e = rng.uniform(0, 2) + np.arange(ns + 1)
        elif kind == 1:
            e = np.sqrt(np.cumsum(rng.integers(1, 40, ns + 1)).astype(np.float64))
        elif kind == 2:
            e = rng.uniform(0, 2) + np.cumsum(rng.uniform(0.05, 6.0, ns + 1))
        else:
            e = 0.5 * np.arange(ns + 1)
        K = 0
        while (K + 1) ** 2 < e[-1] ** 2:
            K += 1
        N = next(n for n in (16, 24, 32, 48, 64, 96, 128) if 2 * K + 1 <= n)
        rc, t = host_tables(lib, N, 2, e, ps.POLY_ALLOW_ALIAS)
        assert rc == 0
        off = t["line_off"]
        for s in range(ns):
            got = t["lines"][off[s]:off[s + 1]].astype(np.int64)
            assert np.array_equal(got, scanned_lines(e, s, K)), (trial, s)
