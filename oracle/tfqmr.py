"""Left-preconditioned TFQMR (oracle; test infrastructure only).

The paper solves the left-preconditioned system of Eq. (6),
Zinv Z I = Zinv V, with the transpose-free quasi-minimal residual method
(Freund 1993) and a stopping tolerance chi_sol.  This is that method written
out in its textbook form for the operator A = M Z and right-hand side M b:

* the CGS-like pair of search vectors y1, y2 = y1 - alpha v per iteration and
  two quasi-residual half-steps, one per y;
* after each half-step, the quasi-minimal residual update with
  theta = ||w|| / tau, c = 1 / sqrt(1 + theta^2), tau <- tau theta c,
  eta = c^2 alpha, d <- y + (theta_prev^2 eta_prev / alpha) d, x <- x + eta d;
* the stopping test uses the bound ||r_m|| <= tau_m sqrt(m + 1) on the
  preconditioned residual, then confirms with the true preconditioned residual
  and restarts from the current iterate if the bound was optimistic.

An "iteration" is one pass of the outer loop (two applications of A).
"""
from __future__ import annotations

import numpy as np


def tfqmr(apply_A, b: np.ndarray, apply_M=None, rtol: float = 1e-6, max_iter: int = 500, x0=None,
          trace=None):
    """Solve A x = b with left preconditioner M (a callable, default identity).

    Returns (x, iterations, final relative preconditioned residual
    ||M (b - A x)|| / ||M b||).  `trace`, when a list, receives
    (true preconditioned residual norm, tau * sqrt(m + 1)) after every half-step.
    """
    M = apply_M if apply_M is not None else (lambda v: v)
    op = lambda v: M(apply_A(v))  # noqa: E731
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    mb = M(b)
    nmb = np.linalg.norm(mb)
    if nmb == 0.0:
        return x, 0, 0.0
    it = 0
    rel = np.linalg.norm(mb - op(x)) / nmb
    while it < max_iter and rel > rtol:
        it_start = it
        r0 = mb - op(x)
        w = r0.copy()
        y1 = r0.copy()
        Ay1 = op(y1)
        v = Ay1.copy()
        d = np.zeros_like(b)
        tau = np.linalg.norm(r0)
        theta = 0.0
        eta = 0.0
        rt = r0  # shadow vector r~0
        rho = np.vdot(rt, r0)
        m = 0
        done = False
        while it < max_iter and not done:
            sigma = np.vdot(rt, v)
            if sigma == 0 or rho == 0:
                break  # breakdown: restart from the current iterate
            alpha = rho / sigma
            y2 = y1 - alpha * v
            Ay2 = op(y2)
            it += 1
            for y, Ay in ((y1, Ay1), (y2, Ay2)):
                m += 1
                w = w - alpha * Ay
                theta_prev, eta_prev = theta, eta
                theta = np.linalg.norm(w) / tau
                c = 1.0 / np.sqrt(1.0 + theta * theta)
                tau = tau * theta * c
                d = y + (theta_prev ** 2 * eta_prev / alpha) * d
                eta = c * c * alpha
                x = x + eta * d
                bound = tau * np.sqrt(m + 1)
                if trace is not None:
                    trace.append((np.linalg.norm(mb - op(x)), bound))
                if bound <= rtol * nmb:
                    done = True
                    break
            if done:
                break
            rho_new = np.vdot(rt, w)
            beta = rho_new / rho
            rho = rho_new
            y1 = w + beta * y2
            Ay1 = op(y1)
            v = Ay1 + beta * (Ay2 + beta * v)
        rel = np.linalg.norm(mb - op(x)) / nmb
        if it == it_start:
            break  # breakdown before any progress
    return x, it, rel
