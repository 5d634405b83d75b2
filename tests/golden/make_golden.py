"""Writes tests/golden/pedigree_exact.json: a tiny GWAS whose results are exact rationals.

Calls only oracle.exact (rational Gauss-Jordan on Eq. "GLS").  The kinship is the relationship
matrix of a small pedigree built from the coefficients of Supplementary Note Section 1 (1 on the
diagonal, 1/2 between a parent and its child and between full siblings, 0 between unrelated
individuals).  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys
from fractions import Fraction as F

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
from oracle.exact import grid_exact  # noqa: E402

H = F(1, 2)
# 0, 1: unrelated parents; 2, 3: their children (full siblings); 4: child of 2 and an outsider
# (1/2 to its parent 2, 1/4 to grandparents 0 and 1 and to its aunt/uncle 3); 5: unrelated.
PHI = [
    [1, 0, H, H, F(1, 4), 0],
    [0, 1, H, H, F(1, 4), 0],
    [H, H, 1, H, H, 0],
    [H, H, H, 1, F(1, 4), 0],
    [F(1, 4), F(1, 4), H, F(1, 4), 1, 0],
    [0, 0, 0, 0, 0, 1],
]
XL = [[1, F(3, 2)], [1, F(-1, 2)], [1, F(1, 4)], [1, 2], [1, F(-3, 4)], [1, 0]]
XR = [[0, 1, 2, 1, 0, 1], [2, 2, 1, 0, 1, 0], [1, 0, 0, 1, 2, 2], [0, 0, 1, 1, 1, 2]]
Y = [[F(5, 4), 3], [F(-1, 2), F(1, 3)], [2, F(-2, 5)], [F(7, 3), 1], [0, F(-3, 2)], [F(1, 5), 2]]
H2 = [F(2, 5), F(3, 4)]
S2 = [F(1), F(3, 2)]


def s(x):
    x = F(x)
    return f"{x.numerator}/{x.denominator}"


def main():
    B, V, W = grid_exact(PHI, XL, XR, Y, H2, S2)
    out = {
        "source": "Eq. GLS / Eq. probDef, Supplementary Note Section 1; pedigree relationship "
                  "coefficients as defined there; exact rational arithmetic (oracle.exact)",
        "n": len(PHI), "q": len(XL[0]), "m": len(XR), "t": len(Y[0]),
        "Phi": [[s(v) for v in row] for row in PHI],
        "XL": [[s(v) for v in row] for row in XL],
        "XR": XR,
        "Y": [[s(v) for v in row] for row in Y],
        "h2": [s(v) for v in H2], "s2": [s(v) for v in S2],
        "B": [[[s(v) for v in b] for b in Bi] for Bi in B],
        "Vdiag": [[[s(var[k][k]) for k in range(len(var))] for var in Vi] for Vi in V],
        "W": [[s(w) for w in Wi] for Wi in W],
    }
    path = os.path.join(os.path.dirname(__file__), "pedigree_exact.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
