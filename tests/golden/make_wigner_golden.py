"""Writes wigner_d_closed_forms.txt: textbook closed forms of the small Wigner
d-matrix for j = 1 and j = 2 (e.g. Varshalovich, Moskalev & Khersonskii 1988,
Table 4.3; the same table is reproduced in most quantum-mechanics texts), in the
convention d^j_{m'm}(beta) = <j m'| exp(-i beta J_y) |j m>.
Uses only the math module.  Run: python tests/golden/make_wigner_golden.py
"""
import math
import os

def table(b):
    c, s = math.cos(b), math.sin(b)
    r = {}
    r[(1, 1, 1)] = (1 + c) / 2
    r[(1, 1, 0)] = -s / math.sqrt(2)
    r[(1, 1, -1)] = (1 - c) / 2
    r[(1, 0, 0)] = c
    r[(2, 2, 2)] = ((1 + c) / 2) ** 2
    r[(2, 2, 1)] = -(1 + c) * s / 2
    r[(2, 2, 0)] = math.sqrt(3.0 / 8.0) * s * s
    r[(2, 2, -1)] = -(1 - c) * s / 2
    r[(2, 2, -2)] = ((1 - c) / 2) ** 2
    r[(2, 1, 1)] = (1 + c) * (2 * c - 1) / 2
    r[(2, 1, 0)] = -math.sqrt(3.0 / 2.0) * s * c
    r[(2, 1, -1)] = (1 - c) * (2 * c + 1) / 2
    r[(2, 0, 0)] = (3 * c * c - 1) / 2
    return r

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wigner_d_closed_forms.txt")
    with open(out, "w") as f:
        f.write("# j m' m beta d^j_{m'm}(beta); textbook closed forms, see make_wigner_golden.py\n")
        for b in (0.3, 1.1, 2.2, 2.9):
            for (j, mp, m), v in sorted(table(b).items()):
                f.write(f"{j} {mp} {m} {b!r} {v!r}\n")
