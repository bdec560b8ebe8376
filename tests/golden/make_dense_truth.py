"""Writes dense FP64 ground truth (ECC for every node, Kemeny's constant) for
the small Erdos-Renyi workload, computed only by oracle/dense.py.

    python tests/golden/make_dense_truth.py

Output: tests/golden/dense_truth_er1000.txt.  The graph fingerprint (n, arcs,
SHA-1 of the CSR bytes) lets readers check the file still matches the
generator."""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle.dense as D  # noqa: E402
from paper_2311_10290_gb300 import inputs  # noqa: E402


def fingerprint(g):
    h = hashlib.sha1()
    h.update(g.row_ptr.astype("<i4").tobytes())
    h.update(g.col.astype("<i4").tobytes())
    return h.hexdigest()


def main():
    g = inputs.er_1000()
    ecc = D.ecc(g.n, g.row_ptr, g.col)
    kc = D.kemeny(g.n, g.row_ptr, g.col)
    path = os.path.join(HERE, "dense_truth_er1000.txt")
    with open(path, "w") as f:
        f.write("# Dense FP64 truth for the Erdos-Renyi G(1000, 0.01) workload (largest component, seed 0).\n")
        f.write("# Written by tests/golden/make_dense_truth.py from oracle/dense.py:\n")
        f.write("# ECC c(u) = (n-1)/(n L+_uu + Tr L+), Kemeny = Tr(calL+) (Section 2 of the paper).\n")
        f.write("n %d\narcs %d\nsha1 %s\n" % (g.n, g.arcs, fingerprint(g)))
        f.write("kemeny %.17g\n" % kc)
        for x in ecc:
            f.write("ecc %.17g\n" % x)
    print(path)


if __name__ == "__main__":
    main()
