"""Algorithm 2 (BF_SMW) and Algorithm 1 with it, from products only (oracle; test infrastructure only).

Sec. III-B inverts the HOD-BF matrix recursively (Algorithm 1): with the
children's inverses known, B'_taui = D_taui^-1 B_taui is recompressed from
products (BF_random_matvec), and D_tau^-1 = BF_SMW([I, B'_tau1; B'_tau2, I])
diag(D_tau1^-1, D_tau2^-1).  BF_SMW (Algorithm 2) inverts I + (a butterfly)
by splitting it into 2 x 2 quadrants, each I + (a butterfly of L - 2 levels):
  A22^-1      <- BF_SMW(A22)
  S - I       <- products of A11 - A12 A22^-1 A21 - I          (Schur complement)
  S^-1 - I    <- BF_SMW(S)
  A^-1 - I    <- products of [I, 0; -A22^-1 A21, I] diag(S^-1, A22^-1)
                 [I, -A12 A22^-1; 0, I] - I,
every "<- products of" being a butterfly built by RandomButterfly from
products with the operator and its adjoint.  Small operators (two levels or
fewer, or at most `dense_max` unknowns) are inverted densely from n products
with unit vectors.  Each butterfly of A^-1 - I is returned as a
RandomButterfly over the node's row and column tree.
"""
from __future__ import annotations

import numpy as np

from .bf_random import RandomButterfly
from .hodbf import sub_bounds


class _Op:
    """y = (X - I) x for an operator given by products with X - I (mv) and its adjoint (rmv)."""

    def __init__(self, mv, rmv, n):
        self.mv, self.rmv, self.n = mv, rmv, n


def _quadrant(op: _Op, n1: int, r: int, c: int) -> _Op:
    """Quadrant (r, c) in {0, 1}^2 of X - I as products (the identity lives on the diagonal quadrants)."""
    n = op.n
    rs = slice(0, n1) if r == 0 else slice(n1, n)
    cs = slice(0, n1) if c == 0 else slice(n1, n)
    nc = cs.stop - cs.start

    def mv(x):
        z = np.zeros((n,) + x.shape[1:], dtype=np.complex128)
        z[cs] = x
        return op.mv(z)[rs]

    def rmv(y):
        z = np.zeros((n,) + y.shape[1:], dtype=np.complex128)
        z[rs] = y
        return op.rmv(z)[cs]

    return _Op(mv, rmv, nc)


def bf_smw(op: _Op, bounds, level: int, node: int, L: int, tol: float, dense_max: int = 256, seed: int = 0):
    """A^-1 - I over the node (level, node) with L butterfly levels, from products with A - I."""
    ob = sub_bounds(bounds, level, node, L)
    n = op.n
    if L <= 2 or n <= dense_max:
        M = op.mv(np.eye(n, dtype=np.complex128))
        E = np.linalg.inv(np.eye(n) + M) - np.eye(n)
        return RandomButterfly(lambda X: E @ X, lambda Y: E.conj().T @ Y, ob, ob, L, tol, seed=seed)
    n1 = int(bounds[level + 1][2 * node + 1] - bounds[level + 1][2 * node])
    A11, A12 = _quadrant(op, n1, 0, 0), _quadrant(op, n1, 0, 1)
    A21, A22 = _quadrant(op, n1, 1, 0), _quadrant(op, n1, 1, 1)
    R22 = bf_smw(A22, bounds, level + 1, 2 * node + 1, L - 2, tol, dense_max, seed + 1)

    def inv22(y):
        return y + R22.apply(y)

    def inv22h(y):
        return y + R22.apply_adjoint(y)

    S = _Op(lambda x: A11.mv(x) - A12.mv(inv22(A21.mv(x))),
            lambda y: A11.rmv(y) - A21.rmv(inv22h(A12.rmv(y))), n1)
    ob1 = sub_bounds(bounds, level + 1, 2 * node, L - 2)
    Sb = RandomButterfly(S.mv, S.rmv, ob1, ob1, L - 2, tol, seed=seed + 2)
    R11 = bf_smw(_Op(Sb.apply, Sb.apply_adjoint, n1), bounds, level + 1, 2 * node, L - 2, tol, dense_max, seed + 3)

    def full(x):  # A^-1 x - x through the block LDU factors
        x1, x2 = x[:n1], x[n1:]
        u1 = x1 - A12.mv(inv22(x2))
        v1 = u1 + R11.apply(u1)
        v2 = inv22(x2)
        w2 = v2 - inv22(A21.mv(v1))
        return np.concatenate([v1, w2]) - x

    def full_h(y):
        y1, y2 = y[:n1], y[n1:]
        a1 = y1 - A21.rmv(inv22h(y2))
        b1 = a1 + R11.apply_adjoint(a1)
        b2 = inv22h(y2)
        c2 = b2 - inv22h(A12.rmv(b1))
        return np.concatenate([b1, c2]) - y

    return RandomButterfly(full, full_h, ob, ob, L, tol, seed=seed + 4)


class HODBFInverseSMW:
    """Algorithm 1 with BF_random_matvec (line 7) and BF_SMW (line 8), from products only.

    A: the operator in tree order as a dense matrix (products with its blocks and with the
    children's inverses are the only use made of it above the leaves)."""

    def __init__(self, A: np.ndarray, bounds, LH: int, tol: float, dense_max: int = 256):
        self.bounds, self.LH = bounds, LH
        lb = bounds[LH]
        self.Dinv = [np.linalg.inv(A[lb[i]:lb[i + 1], lb[i]:lb[i + 1]]) for i in range(2 ** LH)]
        self.E = {}
        for l in range(LH - 1, -1, -1):
            for i in range(2 ** l):
                a, m, b = bounds[l][i], bounds[l + 1][2 * i + 1], bounds[l][i + 1]
                L = LH - l
                # B'_tau1 = D_tau1^-1 B_tau1 and B'_tau2 = D_tau2^-1 B_tau2, applied through the
                # inverse already built for the children (Algorithm 1, line 7)
                B1, B2 = A[a:m, m:b], A[m:b, a:m]

                def inv_sub(y, lo, hi, adjoint=False):
                    return self._apply_range(y, lo, hi, adjoint)

                def mv(x, a=a, m=m, b=b, B1=B1, B2=B2):
                    x1, x2 = x[:m - a], x[m - a:]
                    return np.concatenate([inv_sub(B1 @ x2, a, m), inv_sub(B2 @ x1, m, b)])

                def rmv(y, a=a, m=m, b=b, B1=B1, B2=B2):
                    y1, y2 = y[:m - a], y[m - a:]
                    return np.concatenate([B2.conj().T @ inv_sub(y2, m, b, True),
                                           B1.conj().T @ inv_sub(y1, a, m, True)])

                self.E[(l, i)] = bf_smw(_Op(mv, rmv, b - a), bounds, l, i, L, tol, dense_max, seed=7 * l + i)

    def _apply_range(self, y, lo, hi, adjoint=False):
        """The inverse of the diagonal block over [lo, hi) (a node whose subtree is complete)."""
        b = self.bounds
        out = np.zeros((b[0][-1],) + y.shape[1:], dtype=np.complex128)
        out[lo:hi] = y
        out = self.apply(out, lo, hi, adjoint)
        return out[lo:hi]

    def apply(self, x: np.ndarray, lo: int = 0, hi: int | None = None, adjoint: bool = False) -> np.ndarray:
        """Zinv x (leaf inverses, then y_tau <- y_tau + E_tau y_tau upwards), restricted to the
        nodes inside [lo, hi) when given; the adjoint runs the factors in reverse order."""
        b = self.bounds
        hi = b[0][-1] if hi is None else hi
        y = np.array(x, dtype=np.complex128)
        lb = b[self.LH]
        nodes = [(l, i) for l in range(self.LH - 1, -1, -1) for i in range(2 ** l)
                 if (l, i) in self.E and b[l][i] >= lo and b[l][i + 1] <= hi]
        if not adjoint:
            for i in range(2 ** self.LH):
                if lb[i] >= lo and lb[i + 1] <= hi:
                    y[lb[i]:lb[i + 1]] = self.Dinv[i] @ y[lb[i]:lb[i + 1]]
            for (l, i) in nodes:
                s = slice(b[l][i], b[l][i + 1])
                y[s] = y[s] + self.E[(l, i)].apply(y[s])
        else:
            for (l, i) in reversed(nodes):
                s = slice(b[l][i], b[l][i + 1])
                y[s] = y[s] + self.E[(l, i)].apply_adjoint(y[s])
            for i in range(2 ** self.LH):
                if lb[i] >= lo and lb[i + 1] <= hi:
                    y[lb[i]:lb[i + 1]] = self.Dinv[i].conj().T @ y[lb[i]:lb[i + 1]]
        return y
