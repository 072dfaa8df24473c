"""Quadrature rules on the reference tetrahedron and triangle (oracle; test infrastructure only).

The paper does not state its quadrature (Sec. II is silent).  The reading used
by both implementations (a specification, implemented twice):
  * ``tet4``: the symmetric 4-point degree-2 rule, barycentric (a, b, b, b)
    with a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, equal weights;
  * ``tri3``: the symmetric 3-point degree-2 rule, barycentric (2/3, 1/6, 1/6);
  * ``tet_conical(n)`` / ``tri_conical(n)``: Stroud conical product rules from
    the collapsed-coordinate (Duffy) map x = u, y = (1-u) v, z = (1-u)(1-v) w
    with Gauss-Jacobi nodes in u (weight (1-u)^2 or (1-u)) and v (weight
    (1-v)) and Gauss-Legendre nodes in w, exact to degree 2n-1.
All rules return barycentric coordinates (q, 4) or (q, 3) and weights that sum
to 1 (multiply by the element's volume or area).
"""
from __future__ import annotations

import functools
import math

import numpy as np
from scipy.special import roots_jacobi, roots_legendre


def _unit(alpha: int, n: int):
    """Gauss-Jacobi rule on [0, 1] for the weight (1-u)^alpha."""
    if alpha == 0:
        x, w = roots_legendre(n)
    else:
        x, w = roots_jacobi(n, alpha, 0.0)
    return (1.0 + x) / 2.0, w / 2.0 ** (alpha + 1)


@functools.lru_cache(None)
def tet4():
    a = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    b = (5.0 - math.sqrt(5.0)) / 20.0
    lam = np.full((4, 4), b)
    np.fill_diagonal(lam, a)
    return lam, np.full(4, 0.25)


@functools.lru_cache(None)
def tri3():
    lam = np.full((3, 3), 1.0 / 6.0)
    np.fill_diagonal(lam, 2.0 / 3.0)
    return lam, np.full(3, 1.0 / 3.0)


@functools.lru_cache(None)
def tet_conical(n: int):
    u, wu = _unit(2, n)
    v, wv = _unit(1, n)
    s, ws = _unit(0, n)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                x = u[i]
                y = (1.0 - u[i]) * v[j]
                z = (1.0 - u[i]) * (1.0 - v[j]) * s[k]
                pts.append([1.0 - x - y - z, x, y, z])
                wts.append(6.0 * wu[i] * wv[j] * ws[k])
    return np.array(pts), np.array(wts)


@functools.lru_cache(None)
def tri_conical(n: int):
    u, wu = _unit(1, n)
    v, wv = _unit(0, n)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            x = u[i]
            y = (1.0 - u[i]) * v[j]
            pts.append([1.0 - x - y, x, y])
            wts.append(2.0 * wu[i] * wv[j])
    return np.array(pts), np.array(wts)
