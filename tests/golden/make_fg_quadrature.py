"""Writes fg_quadrature.txt: F, G of eqs. int1/int2 by direct mpmath quadrature.

Calls only oracle.rpy.fg_integral (the integral definition, not the closed
form of Appendix A), so the stored values pin the closed form independently.
Run from the repository root:  python tests/golden/make_fg_quadrature.py
"""
import os
import sys

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))
from oracle import rpy  # noqa: E402

CASES = [  # (r, xi, a): both branches of Appendix A, two radii, three xi
    (0.5, 0.5, 1.0), (1.0, 0.5, 1.0), (1.5, 0.8, 1.0), (2.5, 0.5, 1.0), (3.0, 0.5, 1.0),
    (5.0, 0.5, 1.0), (2.0, 0.6, 1.3), (3.1, 0.6, 1.3), (0.9, 0.3, 1.0), (4.0, 0.3, 1.0),
]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(__file__), "fg_quadrature.txt")
    with open(out, "w") as f:
        f.write("# F, G (dimensionless, 6 pi eta a M^(r) = F (I - rr) + G rr) from eqs. int1/int2\n")
        f.write("# (arXiv:1611.09322 Sec. II A) by mpmath quadosc at 30 digits.  r xi a F G\n")
        for r, xi, a in CASES:
            F, G = rpy.fg_integral(r, xi, a)
            f.write(f"{r!r} {xi!r} {a!r} {F:.17e} {G:.17e}\n")
            print(r, xi, a, F, G, flush=True)
