"""Fits the odd polynomial used by the kernels' FP32 atan2 (k_recurse.cu, fast_atan2).

atan(r) on r in [0, 1] is approximated as r * P(r^2), P of degree DEG, by a
weighted least-squares fit on Chebyshev nodes followed by a few Lawson
(iteratively reweighted) passes that push the fit towards the minimax
polynomial of the absolute error. Prints the coefficients (highest degree
first, for Horner evaluation) and the FP64 maximum error of the fit.

  python paper_1505_00581_gb300/csrc/fit_atan.py [DEG]

DEG defaults to 6, the degree of the shipped coefficients (7 terms).
"""
import sys

import numpy as np


def fit(deg: int, n: int = 4000, passes: int = 60):
    k = np.arange(n)
    r = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / n))          # Chebyshev nodes on [0, 1]
    s = r * r
    target = np.arctan(r)
    V = np.stack([r * s ** j for j in range(deg + 1)], axis=1)   # columns r, r^3, r^5, ...
    w = np.ones(n)
    for _ in range(passes):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], target * sw, rcond=None)
        err = np.abs(V @ c - target)
        w = w * (err + 1e-30)
        w /= w.sum()
    rr = np.linspace(0, 1, 200001)
    Vd = np.stack([rr * (rr * rr) ** j for j in range(deg + 1)], axis=1)
    return c, float(np.max(np.abs(Vd @ c - np.arctan(rr))))


if __name__ == "__main__":
    deg = int(sys.argv[1]) if len(sys.argv) > 1 else 6
    c, e = fit(deg)
    print(f"degree {deg} in r^2, max |err| = {e:.3e} rad")
    for v in c[::-1]:
        print(f"    {v:+.9e}f,")
