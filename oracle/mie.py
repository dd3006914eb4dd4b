"""Mie series of a homogeneous sphere (the paper's accuracy check, Sec. V-A:
monostatic RCS of the sphere compared with the Mie series).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Written from the published series (Bohren & Huffman form, time dependence
exp(-i w t)).  The paper's exp(+j w t) complex permittivity eps_r - j sigma/(w eps0)
maps to eps_r + i sigma/(w eps0) there; m = sqrt of it with Im m >= 0.
Logarithmic derivative D_n(mx) by downward recurrence (needed at large |m x|,
e.g. a copper sphere), Riccati-Bessel functions of the real argument from
scipy's spherical Bessel functions.
"""
import numpy as np
from scipy.special import spherical_jn, spherical_yn

EPS0 = 8.8541878128e-12
C0 = 299792458.0


def rel_index(eps_r, sigma, freq):
    w = 2 * np.pi * freq
    return np.sqrt(eps_r + 1j * sigma / (w * EPS0) + 0j)


def coefficients(x, m, nmax=None):
    """a_n, b_n for n = 1..nmax (size parameter x = k a, relative index m)."""
    if nmax is None:
        nmax = int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    z = m * x
    nmx = int(max(nmax, abs(z))) + 16
    Dn = np.zeros(nmx + 1, complex)
    for n in range(nmx, 0, -1):
        Dn[n - 1] = n / z - 1.0 / (Dn[n] + n / z)
    n = np.arange(0, nmax + 1)
    psi = x * spherical_jn(n, x)
    chi = -x * spherical_yn(n, x)
    xi = psi - 1j * chi
    a = np.zeros(nmax, complex)
    b = np.zeros(nmax, complex)
    for k in range(1, nmax + 1):
        ta = Dn[k] / m + k / x
        tb = m * Dn[k] + k / x
        a[k - 1] = (ta * psi[k] - psi[k - 1]) / (ta * xi[k] - xi[k - 1])
        b[k - 1] = (tb * psi[k] - psi[k - 1]) / (tb * xi[k] - xi[k - 1])
    return a, b


def pec_coefficients(x, nmax=None):
    """Perfect conductor limit (m -> infinity): a_n = psi_n' / xi_n', b_n = psi_n / xi_n."""
    if nmax is None:
        nmax = int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    n = np.arange(0, nmax + 1)
    psi = x * spherical_jn(n, x)
    chi = -x * spherical_yn(n, x)
    xi = psi - 1j * chi
    k = np.arange(1, nmax + 1)
    dpsi = psi[k - 1] - k * psi[k] / x
    dxi = xi[k - 1] - k * xi[k] / x
    return dpsi / dxi, psi[k] / xi[k]


def backscatter_rcs(radius, freq, eps_r=None, sigma=0.0, pec=False):
    """Monostatic RCS (m^2) of the sphere: pi a^2 / x^2 |sum (2n+1) (-1)^n (a_n - b_n)|^2."""
    k0 = 2 * np.pi * freq / C0
    x = k0 * radius
    a, b = pec_coefficients(x) if pec else coefficients(x, rel_index(eps_r, sigma, freq))
    n = np.arange(1, len(a) + 1)
    s = np.sum((2 * n + 1) * (-1.0) ** n * (a - b))
    return np.pi * radius ** 2 / x ** 2 * abs(s) ** 2


def amplitudes(theta, x, a, b):
    """S1(theta), S2(theta) (theta from the forward direction)."""
    mu = np.cos(np.atleast_1d(theta))
    nmax = len(a)
    pi_prev = np.zeros_like(mu)
    pi_cur = np.ones_like(mu)
    S1 = np.zeros(mu.shape, complex)
    S2 = np.zeros(mu.shape, complex)
    for n in range(1, nmax + 1):
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_cur + b[n - 1] * tau)
        S2 += f * (a[n - 1] * tau + b[n - 1] * pi_cur)
        pi_prev, pi_cur = pi_cur, ((2 * n + 1) * mu * pi_cur - (n + 1) * pi_prev) / n
    return S1, S2


def bistatic_rcs(theta, phi, radius, freq, eps_r=None, sigma=0.0, pec=False):
    """sigma(theta, phi) = 4 pi / k^2 (|S2|^2 cos^2 phi + |S1|^2 sin^2 phi) for an
    incident wave polarised along phi = 0 (theta from the propagation direction)."""
    k0 = 2 * np.pi * freq / C0
    x = k0 * radius
    a, b = pec_coefficients(x) if pec else coefficients(x, rel_index(eps_r, sigma, freq))
    S1, S2 = amplitudes(theta, x, a, b)
    return 4 * np.pi / k0 ** 2 * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)
