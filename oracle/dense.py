"""Dense solve, far field and RCS (oracle; test infrastructure only).

Sec. II: Z I = V (Eq. 4) is solved here by a library LU factorization (the
plain definition of the exact discrete solution).  The scattered far field of
the polarization current J = j w kappa D is
  E_s ~ exp(-j k0 r)/r * k0^2/(4 pi) (I - rr) . F,  F = int kappa d(r') exp(j k0 rhat . r') dv',
so sigma = k0^4/(4 pi) |(I - rr) . F|^2 (lambda0^2, unit incident amplitude);
F uses tet_conical(3).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import quadrature as Q
from .mesh import swg_eval


def solve_dense(Z: np.ndarray, V: np.ndarray) -> np.ndarray:
    lu, piv = sla.lu_factor(Z, check_finite=False)
    return sla.lu_solve((lu, piv), V, check_finite=False)


def far_field(E, I: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """F(rhat) for each direction (ndir, 3) and each column of I: (ndir, nrhs, 3)."""
    mesh = E.mesh
    nt = len(mesh["tets"])
    t = np.arange(nt)
    r, w = E.tet_rule(t, Q.tet_conical(3))
    f = swg_eval(E.geo, t, r)                                  # (nt, q, 4, 3)
    I = np.atleast_2d(I.T).T
    coef = I[mesh["tet_faces"]]                                # (nt, 4, nrhs)
    d = np.einsum("tqad,tar->tqrd", f, coef)                   # d at quadrature points
    kd = E.kappa[:, None, None, None] * d * w[:, :, None, None]
    out = np.zeros((len(dirs), I.shape[1], 3), dtype=np.complex128)
    for i, u in enumerate(np.atleast_2d(dirs)):
        ph = np.exp(1j * E.k0 * (r @ u))                       # (nt, q)
        out[i] = np.einsum("tq,tqrd->rd", ph, kd)
    return out


def rcs(E, I: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """sigma(rhat) in lambda0^2, (ndir, nrhs)."""
    dirs = np.atleast_2d(dirs)
    F = far_field(E, I, dirs)
    Ft = F - np.einsum("id,ird->ir", dirs, F)[:, :, None] * dirs[:, None, :]
    return E.k0 ** 4 / (4 * np.pi) * (np.abs(Ft) ** 2).sum(-1)


def cut_directions(theta_deg, phi_deg):
    th = np.radians(np.asarray(theta_deg, dtype=np.float64))
    ph = np.radians(float(phi_deg))
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
