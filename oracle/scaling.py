"""Closed-form relations of the paper used to pin the oracle and to parameterise
the synthetic workloads.  Test infrastructure (part of the oracle).

* Eq. 8 (Sec. 3.2): width scaling law of the arborescent distributor,
      (w_{k+1}/w_k)^4 (h + w_k)(3h + w_k) / ((h + w_{k+1})(3h + w_{k+1})) = 1/4,
  with channel depth h = 10 mm and the smallest width fixed at 2 mm.  Given the
  smaller width, the next larger one is the root of a monotone function, found
  here by plain bisection.
* Sec. 3.3: Re_in = W_in u_in / nu, u_in the cross-sectional mean velocity.
* Sec. 2.1 (text after Eq. 1): tau = 3 nu + dt/2, i.e. nu = (tau - 1/2)/3 with dt = 1.
"""


def eq8_residual(w_small: float, w_large: float, h: float) -> float:
    """Left-hand side of Eq. 8 minus 1/4, with w_k = w_large, w_{k+1} = w_small."""
    ratio4 = (w_small / w_large) ** 4
    return ratio4 * (h + w_large) * (3.0 * h + w_large) / ((h + w_small) * (3.0 * h + w_small)) - 0.25


def eq8_next_wider(w_small: float, h: float, tol: float = 1e-13) -> float:
    """Width w_k of the parent channel whose child has width w_{k+1} = w_small."""
    lo, hi = w_small, 64.0 * w_small + 64.0 * h
    # residual(lo) = 1 - 1/4 > 0 and residual decreases to -1/4 as w_large grows
    assert eq8_residual(w_small, lo, h) > 0 > eq8_residual(w_small, hi, h)
    while hi - lo > tol * hi:
        mid = 0.5 * (lo + hi)
        if eq8_residual(w_small, mid, h) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def eq8_widths(w_smallest: float = 2.0, h: float = 10.0, scales: int = 4) -> list:
    """Widths from the smallest channel upward: [w_4, w_3, w_2, w_1] for scales=4."""
    widths = [w_smallest]
    for _ in range(scales - 1):
        widths.append(eq8_next_wider(widths[-1], h))
    return widths


def reynolds(width: float, u_mean: float, nu: float) -> float:
    """Re = W u / nu (Sec. 3.3)."""
    return width * u_mean / nu


def viscosity(tau: float) -> float:
    """Kinematic viscosity in lattice units, nu = (tau - 1/2)/3 (Sec. 2.1)."""
    return (tau - 0.5) / 3.0
