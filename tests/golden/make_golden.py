"""Writes the stored expected values under tests/golden/ by calling only oracle/.

counts_n3_N16_unit6.txt: exact polygon counts (Sec. 4, Eq. Ncalc: the number of
closed triangles of grid modes q1+q2+q3 = 0 mod N with q_i in shell k_i) on a
16^3 grid with unit-width shells centred on 1..6 (edges 0.5, 1.5, ..., 6.5), for
every sorted triple k1 >= k2 >= k3, by brute-force enumeration of all triangles
(oracle.direct_sample with no field), not by the FFT route.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402


def main():
    N = 16
    edges = np.arange(7) + 0.5
    bins = oracle.enumerate_bins(edges, 3, oracle.RULE_ALL_SORTED)
    _, counts = oracle.direct_sample(None, edges, 3, bins, N=N)
    with open(os.path.join(HERE, "counts_n3_N16_unit6.txt"), "w") as f:
        f.write("# exact triangle counts, N=16, shells centred on 1..6 (width 1 k_F), all sorted triples\n")
        f.write("# written by tests/golden/make_golden.py (brute-force enumeration, oracle.direct_sample)\n")
        f.write("# k1 k2 k3 count\n")
        for b, c in zip(bins, counts):
            f.write(f"{b[0]} {b[1]} {b[2]} {int(c)}\n")


if __name__ == "__main__":
    main()
