"""Mie series for homogeneous, coated and multilayer spheres (oracle; test infrastructure only).

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


def coefficients_multilayer(xs, ms, nmax: int | None = None):
    """a_n, b_n of a sphere of concentric layers.

    Layer j (0 = innermost) has relative index ms[j] and outer size parameter
    xs[j] (increasing).  Inside layer j the radial function of each mode is
    f(rho) = psi_n(rho) - A chi_n(rho), rho = ms[j] k r; the innermost is psi_n.
    At an interface the tangential fields are continuous, which for the
    logarithmic derivative D = f'/f gives D / m continuous for the electric (a)
    modes and m D continuous for the magnetic (b) modes; each layer's A follows
    from D at its inner radius, and D at its outer radius from A.  At the
    surface (size parameter y = xs[-1], index m = ms[-1]):
      a_n = (D_a/m psi_n(y) - psi_n'(y)) / (D_a/m xi_n(y) - xi_n'(y)),
      b_n = (m D_b psi_n(y) - psi_n'(y)) / (m D_b xi_n(y) - xi_n'(y)).
    """
    xs = np.asarray(xs, dtype=np.float64)
    ms = np.asarray(ms, dtype=np.complex128)
    y = float(xs[-1])
    if nmax is None:
        nmax = int(round(y + 4.0 * y ** (1.0 / 3.0) + 2.0))
    n = np.arange(1, nmax + 1)
    z0 = ms[0] * xs[0]
    Da = _dpsi(n, z0) / _psi(n, z0)
    Db = Da.copy()
    for j in range(1, len(xs)):
        Da = Da * ms[j] / ms[j - 1]
        Db = Db * ms[j - 1] / ms[j]
        r1, r2 = ms[j] * xs[j - 1], ms[j] * xs[j]
        p1, dp1, c1, dc1 = _psi(n, r1), _dpsi(n, r1), _chi(n, r1), _dchi(n, r1)
        p2, dp2, c2, dc2 = _psi(n, r2), _dpsi(n, r2), _chi(n, r2), _dchi(n, r2)
        Aa = (Da * p1 - dp1) / (Da * c1 - dc1)
        Ab = (Db * p1 - dp1) / (Db * c1 - dc1)
        Da = (dp2 - Aa * dc2) / (p2 - Aa * c2)
        Db = (dp2 - Ab * dc2) / (p2 - Ab * c2)
    m = ms[-1]
    psy, dpsy = _psi(n, y), _dpsi(n, y)
    xi = y * (spherical_jn(n, y) + 1j * spherical_yn(n, y))
    dxi = dpsy + 1j * (spherical_yn(n, y) + y * spherical_yn(n, y, derivative=True))
    ta, tb = Da / m, m * Db
    a = (ta * psy - dpsy) / (ta * xi - dxi)
    b = (tb * psy - dpsy) / (tb * xi - dxi)
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


def rcs_sphere(radius: float, eps_r: complex, theta, phi, k0: float = 2 * np.pi, core=None, layers=None):
    """Bistatic RCS (lambda0^2) of a sphere, of a shell when core = (r_in, eps_core), or of a
    multilayer sphere when layers = [(outer radius, eps_r), ...] from the innermost out (then
    radius and eps_r are ignored)."""
    if layers is not None:
        xs = [k0 * r for r, _ in layers]
        a, b = coefficients_multilayer(xs, [refractive_index(e) for _, e in layers])
        S1, S2 = amplitudes(a, b, theta)
        phi = np.asarray(phi, dtype=np.float64)
        return 4 * np.pi / k0 ** 2 * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)
    m2 = refractive_index(eps_r)
    y = k0 * radius
    if core is None:
        a, b = coefficients_homogeneous(y, m2)
    else:
        a, b = coefficients_coated(k0 * core[0], y, refractive_index(core[1]), m2)
    S1, S2 = amplitudes(a, b, theta)
    phi = np.asarray(phi, dtype=np.float64)
    return 4 * np.pi / k0 ** 2 * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)
