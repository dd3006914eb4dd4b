"""Lagrange interpolation error bound of the AIM for lossy media (Sec. IV,
Eqs. (kdefs), (Lbounds), (LboundsD), (Ddef), (LboundsD2)).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With s = sigma/(omega eps), k = k_r sqrt(1 - j s) and theta = k_r d, the
(n+1)-th derivative of exp(-j theta sqrt(1 - j s)) / theta is D_n(theta, s)
(Eq. Ddef, product rule of the n-th derivative), and the interpolation error
of order n satisfies Delta G_n / k_r <= (theta_n - theta_0)^(n+1)/(n+1)! |D_n(theta_0, s)|
(Eq. LboundsD2).
"""
from math import comb, factorial

import numpy as np


def D(n, theta, s):
    """D_n(theta, s) of Eq. (Ddef)."""
    theta = np.asarray(theta, dtype=np.float64)
    q = np.sqrt(1.0 - 1j * np.asarray(s, dtype=np.float64))
    tot = 0.0
    for l in range(n + 2):
        tot = tot + comb(n + 1, l) * (-1.0) ** (n + 1 - l) * factorial(n + 1 - l) \
            * theta ** (-(n - l + 2)) * (-1j) ** l * q ** l
    return np.exp(-1j * theta * q) * tot


def bound(n, theta0, thetan, s):
    """Right-hand side of Eq. (LboundsD2) (error bound divided by k_r)."""
    return (thetan - theta0) ** (n + 1) / factorial(n + 1) * np.abs(D(n, theta0, s))


def lossy_ratio(n, theta0, s):
    """Delta G_n / Delta G_n,lossless for the same grid: |D_n(theta0, s)| / |D_n(theta0, 0)|."""
    return np.abs(D(n, theta0, s)) / np.abs(D(n, theta0, 0.0))


def max_lossy_ratio(n=2, theta=(0.05, 20.0), s=(1e-3, 1e3), num=400):
    """Maximum of lossy_ratio over a log grid of (theta0, s), refined locally by a
    Nelder-Mead polish (scipy).  Returns (max, theta0, s)."""
    from scipy.optimize import minimize
    th = np.geomspace(*theta, num)
    ss = np.geomspace(*s, num)
    TH, SS = np.meshgrid(th, ss, indexing="ij")
    R = lossy_ratio(n, TH, SS)
    i, j = np.unravel_index(np.argmax(R), R.shape)
    f = lambda p: -lossy_ratio(n, np.exp(p[0]), np.exp(p[1]))
    res = minimize(f, [np.log(th[i]), np.log(ss[j])], method="Nelder-Mead",
                   options=dict(xatol=1e-10, fatol=1e-14, maxiter=4000))
    return -res.fun, float(np.exp(res.x[0])), float(np.exp(res.x[1]))
