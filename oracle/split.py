"""Force-split constants of the oracle, derived in FP64 from the paper.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2.4, Eq. (fitform): the residual filtered grid force between two unit
masses at separation r is fitted by

    F_grid(r) = tanh(b r)/r^2 - (b/r)/cosh^2(b r) + c r (1 + d r^2) exp(-d r^2)
                + e (1 + f r^2 + g r^4 + l r^6) exp(-h r^2)

with b=0.72, c=0.01, d=0.27, e=1e-4, f=360, g=100, h=0.67, l=17.

Sec. 3.1, Eq. (force): the short-range kernel is f_SR(s) = (s+eps)^(-3/2) - P5(s)
with s = r.r and P5 a fifth-order polynomial in s that stands in for the grid
force.  The paper prints neither P5's coefficients, nor r_cut, nor eps, so
these readings are taken (each is a parameter of the library, these are only
the defaults):

* P5(s) approximates F_grid(r)/r, because (s+eps)^(-3/2) r is the softened
  Newtonian force vector, so what is subtracted must be the grid force / r.
* r_cut is where the fitted grid force meets Newton, r^2 F_grid(r) = 1 near
  three grid cells (Sec. 2.3 puts the matching at three grid cells).
* P5 is the least-squares fit of F_grid(r)/r on (0, r_cut] weighted by r^3
  (so the residual is measured relative to the Newtonian force 1/r^2), under
  the equality constraint P5(r_cut^2) = F_grid(r_cut)/r_cut, which makes
  f_SR(r_cut^2) = 0 at eps = 0 (force continuous at the cutoff).
* eps = 2.5e-4 grid units^2 (a softening length of ~0.016 grid cells, the
  ratio of the quoted force resolutions to the mean particle spacing in
  Sec. 1's Outer Rim and Q Continuum runs).
"""
from __future__ import annotations

import numpy as np

FITFORM = dict(b=0.72, c=0.01, d=0.27, e=1e-4, f=360.0, g=100.0, h=0.67, l=17.0)
EPS_DEFAULT = 2.5e-4
G_DEFAULT = 1.0
FIT_POINTS = 40001
FIT_RMIN = 1e-3


def f_grid(r):
    """Eq. (fitform), FP64, vectorised over r > 0."""
    p = FITFORM
    r = np.asarray(r, dtype=np.float64)
    br = p["b"] * r
    return (np.tanh(br) / r**2 - (p["b"] / r) / np.cosh(br) ** 2
            + p["c"] * r * (1.0 + p["d"] * r**2) * np.exp(-p["d"] * r**2)
            + p["e"] * (1.0 + p["f"] * r**2 + p["g"] * r**4 + p["l"] * r**6)
            * np.exp(-p["h"] * r**2))


def r_cut_default(lo: float = 2.5, hi: float = 3.5) -> float:
    """Root of r^2 F_grid(r) = 1 between lo and hi, by bisection to FP64 rounding."""
    g = lambda r: float(r * r * f_grid(r)) - 1.0
    assert g(lo) < 0.0 < g(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def fit_poly5(r_cut: float, npts: int = FIT_POINTS, rmin: float = FIT_RMIN,
              constrained: bool = True) -> np.ndarray:
    """Coefficients c_0..c_5 of P5(s) (ascending powers of s), FP64.

    Weighted least squares of sum_k c_k s^k against F_grid(r)/r on a uniform r
    grid in [rmin, r_cut], residuals weighted by r^3.  With `constrained`, the
    constraint P5(r_cut^2) = F_grid(r_cut)/r_cut is imposed exactly by
    eliminating c_0.  The fit is done in u = s / r_cut^2 for conditioning and
    mapped back (c_k = d_k / r_cut^(2k)).
    """
    r = np.linspace(rmin, r_cut, npts)
    s = r * r
    u = s / (r_cut * r_cut)
    y = f_grid(r) / r
    w = r**3
    V = np.vander(u, 6, increasing=True)
    if constrained:
        y_c = float(f_grid(r_cut) / r_cut)          # value of P5 at u = 1
        # P5(u) = y_c + sum_{k>=1} d_k (u^k - 1)
        A = (V[:, 1:] - 1.0) * w[:, None]
        rhs = (y - y_c) * w
        d_rest, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        d = np.concatenate([[y_c - d_rest.sum()], d_rest])
    else:
        d, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
    return d / (r_cut * r_cut) ** np.arange(6)


def default_split() -> dict:
    """The default force-split parameters (r_cut, eps, poly c_0..c_5, G)."""
    rc = r_cut_default()
    return dict(r_cut=rc, eps=EPS_DEFAULT, poly=fit_poly5(rc), G=G_DEFAULT)


def p5(s, c):
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros_like(s)
    for k in range(5, -1, -1):
        out = out * s + c[k]
    return out
