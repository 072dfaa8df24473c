"""Restarted, right-preconditioned GMRES (oracle; test infrastructure only).

The paper solves the preconditioned system (Eq. 6) with TFQMR and a stopping
tolerance chi_sol; reading: right preconditioning, so that the stopping test
is on the true residual ||b - A x|| / ||b||.  Textbook GMRES(m): modified
Gram-Schmidt Arnoldi on A M, Givens rotations for the small least-squares
problem, restart every m steps.
"""
from __future__ import annotations

import numpy as np


def gmres(apply_A, b: np.ndarray, apply_M=None, rtol: float = 1e-6, restart: int = 30,
          max_iter: int = 1000, x0=None):
    """Solve A x = b; returns (x, iterations, relative residual history)."""
    M = apply_M if apply_M is not None else (lambda v: v)
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while it < max_iter:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta / nb <= rtol:
            break
        m = min(restart, max_iter - it)
        Vb = np.zeros((len(b), m + 1), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Vb[:, 0] = r / beta
        k_used = 0
        for k in range(m):
            w = apply_A(M(Vb[:, k]))
            for i in range(k + 1):
                H[i, k] = np.vdot(Vb[:, i], w)
                w = w - H[i, k] * Vb[:, i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0:
                Vb[:, k + 1] = w / H[k + 1, k]
            for i in range(k):  # apply previous rotations [c, s; -conj(s), c], c real
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -np.conj(sn[i]) * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            a, c = H[k, k], H[k + 1, k]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            if abs(a) == 0.0:
                cs[k], sn[k] = 0.0, 1.0
            else:
                cs[k] = abs(a) / den
                sn[k] = (a / abs(a)) * np.conj(c) / den
            H[k, k] = cs[k] * a + sn[k] * c
            H[k + 1, k] = 0.0
            g[k + 1] = -np.conj(sn[k]) * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            hist.append(abs(g[k + 1]) / nb)
            if abs(g[k + 1]) / nb <= rtol:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + M(Vb[:, :k_used] @ y)
        if hist[-1] <= rtol:
            r = b - apply_A(x)
            hist.append(np.linalg.norm(r) / nb)
            if hist[-1] <= rtol:
                break
    return x, it, hist
