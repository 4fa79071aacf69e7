"""Choose sinc-quadrature parameters (u0, du) for the Newton kernel, eq. (3.6).

The paper leaves the quadrature nodes open.  This script picks, for R nodes
t_q = exp(u0 + q du) with weights 2/sqrt(pi) du t_q (the geometric tail below u0 folded into
the first weight, as the oracle defines it), the pair (u0, du) that minimises the max
relative error of the exponential sum against 1/r over [r_min, r_max] (log-spaced samples),
using only the oracle's quadrature routine.  Its output is pasted into the input generator's
table as plain numbers.

Usage:  python -m oracle.sinc_fit
"""

from __future__ import annotations

import numpy as np
from scipy.optimize import minimize

import oracle

CLASSES = {
    # name: (R, r_min, r_max)
    "periodic_8": (24, 0.03125, 16.0),
    "tube_256": (32, 0.0109375, 362.0),
    "box_64": (32, 0.025, 186.0),
    "cubic_32": (32, 0.015625, 60.0),
    "small": (20, 0.04, 60.0),
    "hetero_24": (24, 0.025, 1500.0),
    "hetero_32": (32, 0.025, 1500.0),
}


def max_rel_error(R: int, u0: float, du: float, r: np.ndarray) -> float:
    approx = oracle.sinc_inverse_r(R, u0, du, r)
    return float(np.max(np.abs(approx * r - 1.0)))


def fit(R: int, r_min: float, r_max: float, samples: int = 600):
    r = np.geomspace(r_min, r_max, samples)
    best = None
    for du in np.linspace(0.15, 1.2, 43):
        for u0 in np.linspace(-16.0, 0.0, 81):
            e = max_rel_error(R, u0, du, r)
            if best is None or e < best[0]:
                best = (e, u0, du)
    res = minimize(lambda p: max_rel_error(R, p[0], p[1], r), x0=[best[1], best[2]],
                   method="Nelder-Mead", options={"xatol": 1e-6, "fatol": 1e-12, "maxiter": 4000})
    u0, du = float(res.x[0]), float(res.x[1])
    u0, du = round(u0, 4), round(du, 4)
    return u0, du, max_rel_error(R, u0, du, r)


def main():
    for name, (R, lo, hi) in CLASSES.items():
        u0, du, err = fit(R, lo, hi)
        print(f'    "{name}": ({R}, {u0}, {du}),   # max rel err {err:.2e} on [{lo}, {hi}]')


if __name__ == "__main__":
    main()
