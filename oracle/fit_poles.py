"""Write the rational-approximant tables used as inputs by every workload.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): this script calls only the
oracle's fitter.  Output: paper_2605_19951_gb300/data/rational_m{m}.json with
the poles xi_i (one per conjugate pair, Section 2.3), the coefficients
alpha_i^[j] for each stored set of log-spaced observation times in
[1e-5, 1e-2] s, and the measured max error of r_j against exp(-t_j z) on a
20k-point grid.

Run:  python -m oracle.fit_poles
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import rational

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2605_19951_gb300", "data")
TIME_COUNTS = (8, 16, 24, 32, 40)


def _key(t):
    return f"{len(t)}:{t[0]:.6e}:{t[-1]:.6e}"


def main():
    os.makedirs(OUT, exist_ok=True)
    for m in (8, 10):
        xi = rational.fit_poles(m)
        tab = {"m": m, "t_range": [1e-5, 1e-2],
               "xi_re": xi.real.tolist(), "xi_im": xi.imag.tolist(),
               "system": "A_i = K - xi_i M; each xi_i stands for the pair {xi_i, conj xi_i}",
               "alpha": {}}
        for K in TIME_COUNTS:
            t = np.logspace(-5, -2, K)
            al = rational.fit_alpha(xi, t)
            eps = rational.max_error(xi, al, t)
            tab["alpha"][_key(t)] = {"times": t.tolist(), "re": al.real.tolist(),
                                     "im": al.imag.tolist(), "max_abs_err": eps.tolist(),
                                     "cancellation": rational.cancellation(xi, al)}
            print(f"m={m} K={K} max |exp - r| = {eps.max():.3e}  "
                  f"cancellation {rational.cancellation(xi, al):.2e}")
        with open(os.path.join(OUT, f"rational_m{m}.json"), "w") as fh:
            json.dump(tab, fh, indent=1)


if __name__ == "__main__":
    main()
