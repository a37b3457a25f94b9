"""Write exact rational fixtures for the ray-factor messages.

Calls only oracle.brute (literal enumeration of Eq. "factor_to_node" with the
potential of Eq. "depth_potential", in exact rational arithmetic).  Each line:
N | m1_1..m1_N | nu_1..nu_N | nu_bg | mu1_1,mu0_1 ; ... (fractions as p/q).
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys
from fractions import Fraction as F

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import brute  # noqa: E402

CASES = [
    ([F(1, 2), F(1, 3)], [F(2), F(1)], F(1, 2)),
    ([F(1, 10)], [F(5, 2)], F(1, 4)),
    ([F(1, 10), F(9, 10), F(1, 2)], [F(1, 3), F(7), F(2, 5)], F(1, 100)),
    ([F(1, 5), F(1, 5), F(1, 5), F(1, 5)], [F(3), F(3), F(3), F(3)], F(3)),
    ([F(1, 5), F(2, 5), F(3, 5), F(4, 5)], [F(1), F(2), F(3), F(4)], F(0)),
    ([F(1, 7), F(2, 7), F(3, 7), F(4, 7), F(5, 7)], [F(1, 2), F(9, 2), F(1, 9), F(2), F(5)], F(1, 50)),
]


def fmt(x):
    return f"{x.numerator}/{x.denominator}"


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ray_messages_exact.txt")
    with open(out, "w") as f:
        f.write("# Exact ray-factor -> occupancy messages by enumeration (Eq. factor_to_node with\n")
        f.write("# Eq. depth_potential; all-empty configuration weighted by nu_bg).  Generated by\n")
        f.write("# tests/golden/make_golden.py from oracle.brute; do not edit by hand.\n")
        f.write("# N | m1 | nu | nu_bg | mu(o_i=1),mu(o_i=0) per voxel\n")
        for m1, nu, bg in CASES:
            res = brute.factor_to_node_exact(m1, nu, bg)
            f.write("%d | %s | %s | %s | %s\n" % (
                len(m1), " ".join(map(fmt, m1)), " ".join(map(fmt, nu)), fmt(bg),
                " ; ".join(f"{fmt(a)},{fmt(b)}" for a, b in res)))
        f.write("# Exact tree marginals p(o_i=1) of one ray with Bernoulli(prior) voxel priors\n")
        f.write("# (Eq. 1 restricted to one ray, Eq. prior_potential).\n")
        f.write("# TREE | prior | nu | nu_bg | p_1 .. p_N\n")
        for prior, nu, bg in [(F(1, 2), [F(2), F(1), F(3)], F(1, 2)),
                              (F(1, 10), [F(1, 4), F(8), F(1, 2), F(1)], F(1, 20))]:
            ps = brute.tree_marginals_exact(prior, nu, bg)
            f.write("TREE | %s | %s | %s | %s\n" % (fmt(prior), " ".join(map(fmt, nu)), fmt(bg),
                                                   " ".join(map(fmt, ps))))
    print("wrote", out)


if __name__ == "__main__":
    main()
