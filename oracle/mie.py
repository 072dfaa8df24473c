"""Mie series for homogeneous and coated spheres (oracle; test infrastructure only).

The paper validates its RCS against the exact Mie series (Sec. IV-A); the
series is textbook theory (Bohren & Huffman, ch. 4 and Sec. 8.1), written here
from the mathematics.  Convention map: the paper uses exp(+j w t), Bohren &
Huffman exp(-i w t), so the refractive index is m = conj(sqrt(eps_r)) on the
branch Im m >= 0.

Bistatic RCS for an x-polarized plane wave travelling along +z, observed at
polar angle theta from +z and azimuth phi:
  sigma = (4 pi / k^2) (|S2|^2 cos^2 phi + |S1|^2 sin^2 phi),  in lambda0^2.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def refractive_index(eps_r: complex) -> complex:
    m = np.sqrt(np.conj(complex(eps_r)))
    return m if m.imag >= 0 else -m


def _psi(n, z):
    return z * spherical_jn(n, z)


def _dpsi(n, z):
    return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)


def _chi(n, z):
    return -z * spherical_yn(n, z)


def _dchi(n, z):
    return -(spherical_yn(n, z) + z * spherical_yn(n, z, derivative=True))


def coefficients_homogeneous(x: float, m: complex, nmax: int | None = None):
    """a_n, b_n of a homogeneous sphere (size parameter x, relative index m).

    The logarithmic derivative D_n(mx) comes from the downward recurrence
    D_{n-1} = n/z - 1/(D_n + n/z) (Wiscombe), the Riccati-Bessel functions of
    the real argument from the spherical Bessel functions.
    """
    if nmax is None:
        nmax = int(round(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    z = m * x
    nstart = int(max(nmax, abs(z))) + 16
    D = np.zeros(nstart + 1, dtype=np.complex128)
    for n in range(nstart, 0, -1):
        D[n - 1] = n / z - 1.0 / (D[n] + n / z)
    n = np.arange(1, nmax + 1)
    psi = _psi(n, x)
    psim1 = _psi(n - 1, x)
    xi = x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))
    xim1 = x * (spherical_jn(n - 1, x) + 1j * spherical_yn(n - 1, x))
    Dn = D[1:nmax + 1]
    ta = Dn / m + n / x
    tb = m * Dn + n / x
    a = (ta * psi - psim1) / (ta * xi - xim1)
    b = (tb * psi - psim1) / (tb * xi - xim1)
    return a, b


def coefficients_coated(x: float, y: float, m1: complex, m2: complex, nmax: int | None = None):
    """a_n, b_n of a coated sphere: core size parameter x, index m1; outer y, shell index m2.

    Aden-Kerker coefficients (Bohren & Huffman Sec. 8.1) with chi_n(z) = -z y_n(z).
    """
    if nmax is None:
        nmax = int(round(y + 4.0 * y ** (1.0 / 3.0) + 2.0))
    n = np.arange(1, nmax + 1)
    u, v, w = m1 * x, m2 * x, m2 * y
    An = (m2 * _psi(n, v) * _dpsi(n, u) - m1 * _dpsi(n, v) * _psi(n, u)) / (
        m2 * _chi(n, v) * _dpsi(n, u) - m1 * _dchi(n, v) * _psi(n, u))
    Bn = (m2 * _psi(n, u) * _dpsi(n, v) - m1 * _psi(n, v) * _dpsi(n, u)) / (
        m2 * _dchi(n, v) * _psi(n, u) - m1 * _dpsi(n, u) * _chi(n, v))
    psy, dpsy = _psi(n, y), _dpsi(n, y)
    xi = y * (spherical_jn(n, y) + 1j * spherical_yn(n, y))
    dxi = _dpsi(n, y) + 1j * (spherical_yn(n, y) + y * spherical_yn(n, y, derivative=True))
    fa = _dpsi(n, w) - An * _dchi(n, w)
    ga = _psi(n, w) - An * _chi(n, w)
    fb = _dpsi(n, w) - Bn * _dchi(n, w)
    gb = _psi(n, w) - Bn * _chi(n, w)
    a = (psy * fa - m2 * dpsy * ga) / (xi * fa - m2 * dxi * ga)
    b = (m2 * psy * fb - dpsy * gb) / (m2 * xi * fb - dxi * gb)
    return a, b


def amplitudes(a, b, theta):
    """S1(theta), S2(theta) from the angular functions pi_n, tau_n."""
    mu = np.cos(np.atleast_1d(theta))
    nmax = len(a)
    S1 = np.zeros(mu.shape, dtype=np.complex128)
    S2 = np.zeros(mu.shape, dtype=np.complex128)
    pim1 = np.zeros_like(mu)
    pi = np.ones_like(mu)
    for n in range(1, nmax + 1):
        tau = n * mu * pi - (n + 1) * pim1
        c = (2 * n + 1) / (n * (n + 1))
        S1 += c * (a[n - 1] * pi + b[n - 1] * tau)
        S2 += c * (a[n - 1] * tau + b[n - 1] * pi)
        pi, pim1 = ((2 * n + 1) * mu * pi - (n + 1) * pim1) / n, pi
    return S1, S2


def efficiencies(a, b, x):
    n = np.arange(1, len(a) + 1)
    qext = 2.0 / x ** 2 * np.sum((2 * n + 1) * (a + b).real)
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return qext, qsca


def rcs_sphere(radius: float, eps_r: complex, theta, phi, k0: float = 2 * np.pi, core=None):
    """Bistatic RCS (lambda0^2) of a sphere, or of a shell when core = (r_in, eps_core)."""
    m2 = refractive_index(eps_r)
    y = k0 * radius
    if core is None:
        a, b = coefficients_homogeneous(y, m2)
    else:
        a, b = coefficients_coated(k0 * core[0], y, refractive_index(core[1]), m2)
    S1, S2 = amplitudes(a, b, theta)
    phi = np.asarray(phi, dtype=np.float64)
    return 4 * np.pi / k0 ** 2 * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)
