"""Writes tests/golden/counts_n3_64shells.txt by calling only oracle/.

Exact triangle counts (Sec. 4, Eq. Ncalc; App. A: the number of closed triangles
q1 + q2 + q3 = 0 of grid modes with q_i in shell k_i) for every bin of the
benchmark plan: 64 unit-width shells centred on 1..64 k_F (edges 0.5 .. 64.5),
bins k1 >= k2 >= k3 with k1 <= k2 + k3 (24,432 triangles), from
oracle.counts_triangles (integer pair convolutions of the shell indicators).

The shells reach |q_c| <= 64, so a closure sums to at most 192 in each component:
on any grid N > 192 no closure wraps and every N gives the same counts.  The file
is computed on a 200^3 grid (half the work of 256^3); the GPU test compares it
with the library's counts for the 256^3 plan, and a CPU test re-derives a sample
of it on 256^3 with oracle.counts_exact.

Run:  python tests/golden/make_counts_256.py      (about 10 minutes on 8 cores)
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

N_GRID = 200
OUT = os.path.join(HERE, "counts_n3_64shells.txt")


def main():
    oracle.set_threads(os.cpu_count() or 1)
    edges = np.arange(65) + 0.5
    bins = oracle.enumerate_bins(edges, 3)
    t0 = time.perf_counter()
    counts = oracle.counts_triangles(N_GRID, edges, bins)
    with open(OUT, "w") as f:
        f.write("# exact triangle counts, 64 unit shells centred on 1..64 (edges 0.5..64.5), polygon-rule bins\n")
        f.write(f"# k1 >= k2 >= k3, k1 <= k2 + k3 ({len(bins)} bins), any grid N > 192 (computed on {N_GRID}^3)\n")
        f.write("# written by tests/golden/make_counts_256.py (oracle.counts_triangles)\n")
        f.write("# k1 k2 k3 count\n")
        for b, c in zip(bins, counts):
            f.write(f"{b[0]} {b[1]} {b[2]} {int(c)}\n")
    print(f"{len(bins)} counts in {time.perf_counter() - t0:.0f} s -> {OUT}")


if __name__ == "__main__":
    main()
