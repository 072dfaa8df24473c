"""Butterfly construction from matrix-vector products only (oracle; test infrastructure only).

Sec. III-B builds the blocks of the inverse with BF_random_matvec: a butterfly
is reconstructed from the products of the operator (and its adjoint) with
random vectors, at tolerance chi_fact, in O(n^1.5 log n) work.  The paper
gives the method by citation only; this is a plain construction written from
that description, in the two-sided form of a butterfly (the form Sec. III-A
calls equivalent):

* Column side, levels l = 0 .. h (h = floor(L / 2)): for each row group tau at
  level l of the row tree, a Gaussian block G supported on the rows of tau
  gives the row sketch G^H A(tau, :) = (A^H G)^H of every column at once; the
  column ID of the sketch restricted to the candidate columns (a leaf of the
  column tree at l = 0, else the two children's skeletons) gives the skeleton
  columns and the V^0 / W^l factors, exactly as the entry-based builder does
  with sampled rows.
* Row side, steps t = 0 .. L - h (row-tree level L - t, column-tree level t):
  a Gaussian block supported on the columns of nu gives A(:, nu) G for every
  row at once; the column ID of the transposed sketch restricted to the
  candidate rows (a leaf of the row tree at t = 0, else the two children's row
  skeletons) gives skeleton rows and the interpolation A(cand, nu) ~ U A(I, nu).
* Middle, at (row level h, column level L - h): with the column chain C and the
  row skeleton I of a pair, A(I, nu) G = M (C G) for the random block G of the
  last row step, solved for M by least squares.

Apply: the column chain up to level h, the middle blocks, then the row
interpolations from level h down to the row leaves (children receive the
sum over both column children of their parent).  Product count: about
(2^{h+1} + 2^{L-h+1}) (r + p) columns, r the largest rank.
"""
from __future__ import annotations

import numpy as np

from .hodbf import interp_decomp


def _gauss(rng, m, k):
    return (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))) / np.sqrt(2.0)


class RandomButterfly:
    """A(o, s) ~ R M C from products with A and A^H only.

    matvec(X): A @ X for X of shape (n_s, k); rmatvec(Y): A^H @ Y for Y (m_o, k).
    ob[l], sb[l]: offsets of the level-l nodes of the row and column trees.
    """

    def __init__(self, matvec, rmatvec, ob, sb, L: int, tol: float, p: int = 8, seed: int = 0):
        rng = np.random.default_rng(seed)
        o = [np.asarray(b) - ob[0][0] for b in ob]
        s = [np.asarray(b) - sb[0][0] for b in sb]
        self.o, self.s, self.L = o, s, L
        m, n = int(o[0][-1]), int(s[0][-1])
        self.m, self.n = m, n
        h = L // 2
        self.h = h
        self.products = 0  # columns multiplied by A or A^H
        # ---- column side: levels 0 .. h
        k = max(int(np.max(np.diff(s[L]))), 1) + p
        S = rmatvec(_gauss(rng, m, k)).conj().T  # (k, n) = G^H A
        self.products += k
        self.V = []
        row = []
        for j in range(2 ** L):
            cols = np.arange(s[L][j], s[L][j + 1])
            J, V = interp_decomp(S[:, cols], tol)
            self.V.append(V)
            row.append(cols[J])
        skel = [row]
        self.W = []
        for l in range(1, h + 1):
            lev, new = [], []
            for i in range(2 ** l):
                rows = np.arange(o[l][i], o[l][i + 1])
                prow = skel[i // 2]
                cands = [np.concatenate([prow[2 * j], prow[2 * j + 1]]) for j in range(2 ** (L - l))]
                k = max(len(c) for c in cands) + p
                G = np.zeros((m, k), dtype=np.complex128)
                G[rows] = _gauss(rng, len(rows), k)
                S = rmatvec(G).conj().T
                self.products += k
                Wi, si = [], []
                for c in cands:
                    J, W = interp_decomp(S[:, c], tol)
                    Wi.append(W)
                    si.append(c[J])
                lev.append(Wi)
                new.append(si)
            self.W.append(lev)
            skel = new
        self.cskel = skel  # [i at row level h][j at column level L - h]
        # ---- row side: steps t = 0 .. L - h
        k = max(int(np.max(np.diff(o[L]))), 1) + p
        G = _gauss(rng, n, k)
        X = matvec(G)
        self.products += k
        self.U = [[]]     # U[t][i][j]: (len(cand), len(I)) with A(cand, nu_j) ~ U A(I, nu_j)
        rsk = []          # rsk[i][j]: skeleton rows of (row node i at level L - t, column node j at level t)
        for i in range(2 ** L):
            rows = np.arange(o[L][i], o[L][i + 1])
            J, Vr = interp_decomp(X[rows].T, tol)
            self.U[0].append([Vr.T])
            rsk.append([rows[J]])
        last_G = [None]
        for t in range(1, L - h + 1):
            ni, nj = 2 ** (L - t), 2 ** t
            Ut = [[None] * nj for _ in range(ni)]
            new = [[None] * nj for _ in range(ni)]
            last_G = []
            for j in range(nj):
                cols = np.arange(s[t][j], s[t][j + 1])
                cands = [np.concatenate([rsk[2 * i][j // 2], rsk[2 * i + 1][j // 2]]) for i in range(ni)]
                k = max(len(c) for c in cands) + p
                G = np.zeros((n, k), dtype=np.complex128)
                G[cols] = _gauss(rng, len(cols), k)
                X = matvec(G)
                self.products += k
                last_G.append((G, X))
                for i, c in enumerate(cands):
                    J, Vr = interp_decomp(X[c].T, tol)
                    Ut[i][j] = Vr.T
                    new[i][j] = c[J]
            self.U.append(Ut)
            rsk = new
        self.rskel = rsk  # [i at row level h][j at column level L - h]
        # ---- middle: M_ij from A(I, nu_j) G_j = M_ij (C_ij G_j)
        self.M = [[None] * (2 ** (L - h)) for _ in range(2 ** h)]
        if L - h == 0:  # no row step beyond the leaves: use one block of the whole column range
            G = _gauss(rng, n, max(len(c) for c in skel[0]) + p)
            last_G = [(G, matvec(G))]
            self.products += G.shape[1]
        for j, (G, X) in enumerate(last_G):
            CG = self._column_chain(G)  # coefficients [i][j'] for the block G
            for i in range(2 ** h):
                I = self.rskel[i][j]
                cg = CG[i][j]
                if cg.shape[0] == 0 or len(I) == 0:
                    self.M[i][j] = np.zeros((len(I), cg.shape[0]), dtype=np.complex128)
                    continue
                self.M[i][j] = np.linalg.lstsq(cg.T, X[I].T, rcond=None)[0].T

    def _column_chain(self, xs):
        """Coefficients of the column chain up to level h: [i at row level h][j at column level L - h]."""
        L, h, s = self.L, self.h, self.s
        c = [[self.V[j] @ xs[s[L][j]:s[L][j + 1]] for j in range(2 ** L)]]
        for l in range(1, h + 1):
            new = []
            for i in range(2 ** l):
                p = c[i // 2]
                new.append([self.W[l - 1][i][j] @ np.concatenate([p[2 * j], p[2 * j + 1]])
                            for j in range(2 ** (L - l))])
            c = new
        return c

    def apply(self, xs: np.ndarray) -> np.ndarray:
        L, h, o = self.L, self.h, self.o
        c = self._column_chain(xs)
        d = [[self.M[i][j] @ c[i][j] for j in range(2 ** (L - h))] for i in range(2 ** h)]
        for t in range(L - h, 0, -1):  # row interpolation towards the leaves
            ni, nj = 2 ** (L - t), 2 ** t
            prev = [[None] * (nj // 2) for _ in range(2 * ni)]
            for i in range(ni):
                for j in range(nj):
                    e = self.U[t][i][j] @ d[i][j]
                    n1 = self.U[t - 1][2 * i][j // 2].shape[1]  # skeleton rows of the first child
                    for ch, part in ((2 * i, e[:n1]), (2 * i + 1, e[n1:])):
                        prev[ch][j // 2] = part if prev[ch][j // 2] is None else prev[ch][j // 2] + part
            d = prev
        y = np.zeros((self.m,) + xs.shape[1:], dtype=np.result_type(xs, np.complex128))
        for i in range(2 ** L):
            y[o[L][i]:o[L][i + 1]] = self.U[0][i][0] @ d[i][0]
        return y

    def apply_adjoint(self, ys: np.ndarray) -> np.ndarray:
        """x = A^H y: the adjoint of every factor, in reverse order."""
        L, h, o, s = self.L, self.h, self.o, self.s
        d = [[self.U[0][i][0].conj().T @ ys[o[L][i]:o[L][i + 1]]] for i in range(2 ** L)]
        for t in range(1, L - h + 1):  # row chain upwards
            ni, nj = 2 ** (L - t), 2 ** t
            d = [[self.U[t][i][j].conj().T @ np.concatenate([d[2 * i][j // 2], d[2 * i + 1][j // 2]])
                  for j in range(nj)] for i in range(ni)]
        g = [[self.M[i][j].conj().T @ d[i][j] for j in range(2 ** (L - h))] for i in range(2 ** h)]
        for l in range(h, 0, -1):  # column chain downwards
            prev = [[None] * (2 ** (L - l + 1)) for _ in range(2 ** (l - 1))]
            for i in range(2 ** l):
                for j in range(2 ** (L - l)):
                    e = self.W[l - 1][i][j].conj().T @ g[i][j]
                    n1 = (self.V[2 * j].shape[0] if l == 1 else self.W[l - 2][i // 2][2 * j].shape[0])
                    for jj, part in ((2 * j, e[:n1]), (2 * j + 1, e[n1:])):
                        cur = prev[i // 2][jj]
                        prev[i // 2][jj] = part if cur is None else cur + part
            g = prev
        x = np.zeros((self.n,) + ys.shape[1:], dtype=np.result_type(ys, np.complex128))
        for j in range(2 ** L):
            x[s[L][j]:s[L][j + 1]] = self.V[j].conj().T @ g[0][j]
        return x

    def entries(self) -> int:
        n = sum(v.size for v in self.V) + sum(w.size for lev in self.W for Wi in lev for w in Wi)
        n += sum(u.size for Ut in self.U for Ui in Ut for u in Ui)
        return n + sum(mm.size for Mi in self.M for mm in Mi)
