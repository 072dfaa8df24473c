"""Straightforward HOD-BF: cluster tree, ID, butterfly, apply, dense-defined inverse.

Oracle; test infrastructure only.  Follows Sec. III-A and III-B step by step:

* Cluster tree (Sec. III-A): recursive bisection into halves of nearly equal
  size until a complete binary tree of L_H levels whose leaves hold at most
  ``leaf`` unknowns.  Reading (KD clustering): split along the longest axis of
  the bounding box of the face centroids (ties: lowest axis), sort by that
  coordinate (ties: face id) and give the first ceil(n/2) to the left child.
  L_H = ceil(log2(N / leaf)) (0 when N <= leaf).
* HOD-BF layout (Sec. III-A, Fig. 1): dense leaf blocks D_tau = Z(tau, tau);
  for siblings tau1, tau2 at level l the blocks B_tau1 = Z(tau1, tau2) and
  B_tau2 = Z(tau2, tau1) are butterflies of L = L_H - l levels.
* Interpolative decomposition (Eq. 7): Z(tau, nu) ~ Z(tau, nu_bar) V, from a
  column-pivoted QR; the rank is the number of pivots with |R_kk| > tol |R_11|
  (reading of "O(chi_con)"), V = [I, R11^-1 R12] P^T.
* Nested bases (Eq. 8): W_{tau,nu} from the ID of [Z(tau, nu1_bar), Z(tau, nu2_bar)].
* Butterfly (Eqs. 9-10): Z(o, s) ~ B^L W^L ... W^1 V^0.
* The oracle uses all rows of each sub-block in its IDs (no row sampling).
* Inverse (Sec. III-B, Algorithm 1) from its plain definition:
  D_tau^-1 = (I + E_tau) diag(D_tau1^-1, D_tau2^-1) with
  E_tau = [I, B'_tau1; B'_tau2, I]^-1 - I and B'_taui = D_taui^-1 B_taui,
  all formed densely from the compressed operator, then each E_tau is
  compressed as a butterfly over tau x tau (L_H - l levels) at chi_fact with
  the same ID construction.  Applying the inverse: leaf inverses, then
  y_tau <- y_tau + E_tau y_tau level by level from the leaves to the root.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------------------------
# cluster tree
# ----------------------------------------------------------------------------------

def face_centroids(mesh: dict) -> np.ndarray:
    v = mesh["verts"][mesh["faces"]]
    return (v[:, 0] + v[:, 1] + v[:, 2]) / 3.0


def tree_depth(n: int, leaf: int) -> int:
    return 0 if n <= leaf else int(math.ceil(math.log2(n / leaf)))


def cluster_tree(points: np.ndarray, leaf: int = 64):
    """Returns (perm, L_H, bounds): perm[i] = original index at tree position i;
    bounds[l] = array of 2^l + 1 offsets of the level-l nodes in tree order."""
    n = len(points)
    LH = tree_depth(n, leaf)
    perm = np.arange(n)
    bounds = [np.array([0, n])]
    for l in range(LH):
        prev = bounds[-1]
        nxt = [0]
        for i in range(len(prev) - 1):
            a, b = prev[i], prev[i + 1]
            idx = perm[a:b]
            p = points[idx]
            ext = p.max(0) - p.min(0) if len(idx) else np.zeros(3)
            ax = int(np.argmax(ext))  # first maximum = lowest axis on ties
            order = np.lexsort((idx, p[:, ax]))  # by coordinate, then by face id
            perm[a:b] = idx[order]
            nxt += [a + (b - a + 1) // 2, b]
        bounds.append(np.array(nxt))
    return perm, LH, bounds


# ----------------------------------------------------------------------------------
# interpolative decomposition
# ----------------------------------------------------------------------------------

def interp_decomp(A: np.ndarray, tol: float):
    """Column ID A ~ A[:, J] V (Eq. 7).  Returns (J, V) with J local column indices."""
    m, n = A.shape
    if n == 0 or m == 0:
        return np.zeros(0, dtype=np.int64), np.zeros((0, n), dtype=A.dtype)
    R, piv = sla.qr(A, mode="r", pivoting=True)
    d = np.abs(np.diag(R))
    if d[0] == 0.0:
        return np.zeros(0, dtype=np.int64), np.zeros((0, n), dtype=A.dtype)
    k = int(np.sum(d > tol * d[0]))
    T = sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False) if k < n else np.zeros((k, 0), A.dtype)
    V = np.zeros((k, n), dtype=A.dtype)
    V[:, piv[:k]] = np.eye(k)
    V[:, piv[k:]] = T
    return piv[:k].copy(), V


# ----------------------------------------------------------------------------------
# butterfly (Eqs. 8-10)
# ----------------------------------------------------------------------------------

def sub_bounds(bounds, level0: int, node: int, L: int):
    """Offsets of the subtree of `node` (at level0) down L levels: list of arrays per level."""
    out = []
    for l in range(L + 1):
        k = 2 ** l
        lo = node * k
        out.append(bounds[level0 + l][lo:lo + k + 1])
    return out


class Butterfly:
    """Z(o, s) ~ B^L W^L ... W^1 V^0 (Eq. 9), built from full rows with the ID."""

    def __init__(self, block_fn, ob, sb, L: int, tol: float):
        # ob[l], sb[l]: offsets (tree order, global) of the level-l nodes of T_o, T_s
        self.ob, self.sb, self.L = ob, sb, L
        self.V = []      # V^0: per leaf nu of T_s, V_{o,nu}  (r x |nu|)
        self.W = []      # W[l-1][i][j] = W_{tau_i,nu_j} at level l (r x (r1 + r2))
        skel = []        # skel[i][j]: skeleton columns (global) of (tau_i, nu_j)
        o0, o1 = ob[0][0], ob[0][-1]
        row = []
        for j in range(2 ** L):
            cols = np.arange(sb[L][j], sb[L][j + 1])
            J, V = interp_decomp(block_fn(np.arange(o0, o1), cols), tol)
            self.V.append(V)
            row.append(cols[J])
        skel = [row]
        for l in range(1, L + 1):
            lev, new = [], []
            for i in range(2 ** l):
                rows = np.arange(ob[l][i], ob[l][i + 1])
                prow = skel[i // 2]
                Wi, si = [], []
                for j in range(2 ** (L - l)):
                    cand = np.concatenate([prow[2 * j], prow[2 * j + 1]])
                    J, W = interp_decomp(block_fn(rows, cand), tol)
                    Wi.append(W)
                    si.append(cand[J])
                lev.append(Wi)
                new.append(si)
            self.W.append(lev)
            skel = new
        self.B = []      # B^L: per leaf tau of T_o, Z(tau, s_bar_tau)  (|tau| x r)
        for i in range(2 ** L):
            rows = np.arange(ob[L][i], ob[L][i + 1])
            self.B.append(block_fn(rows, skel[i][0]))

    def apply(self, xs: np.ndarray) -> np.ndarray:
        """y_o = B^L W^L ... W^1 V^0 x_s; xs indexed locally over s."""
        L, sb, ob = self.L, self.sb, self.ob
        s0, o0 = sb[0][0], ob[0][0]
        c = [[self.V[j] @ xs[sb[L][j] - s0:sb[L][j + 1] - s0] for j in range(2 ** L)]]
        for l in range(1, L + 1):
            new = []
            for i in range(2 ** l):
                p = c[i // 2]
                new.append([self.W[l - 1][i][j] @ np.concatenate([p[2 * j], p[2 * j + 1]])
                            for j in range(2 ** (L - l))])
            c = new
        y = np.zeros((ob[0][-1] - o0,) + xs.shape[1:], dtype=np.result_type(xs, np.complex128))
        for i in range(2 ** L):
            y[ob[L][i] - o0:ob[L][i + 1] - o0] = self.B[i] @ c[i][0]
        return y

    def ranks(self):
        r = [[v.shape[0] for v in self.V]]
        for lev in self.W:
            r.append([w.shape[0] for Wi in lev for w in Wi])
        return r

    def entries(self) -> int:
        n = sum(v.size for v in self.V) + sum(b.size for b in self.B)
        return n + sum(w.size for lev in self.W for Wi in lev for w in Wi)


# ----------------------------------------------------------------------------------
# HOD-BF matrix
# ----------------------------------------------------------------------------------

class HODBF:
    """HOD-BF compression of a matrix given by ``block_fn(rows, cols)`` in tree order."""

    def __init__(self, block_fn, bounds, LH: int, tol: float):
        self.bounds, self.LH, self.tol = bounds, LH, tol
        lb = bounds[LH]
        self.D = [block_fn(np.arange(lb[i], lb[i + 1]), np.arange(lb[i], lb[i + 1])) for i in range(2 ** LH)]
        self.B = {}
        for l in range(1, LH + 1):
            L = LH - l
            for i in range(2 ** l):
                sib = i ^ 1
                ob = sub_bounds(bounds, l, i, L)
                sb = sub_bounds(bounds, l, sib, L)
                self.B[(l, i)] = Butterfly(block_fn, ob, sb, L, tol)

    def apply(self, x: np.ndarray) -> np.ndarray:
        """y = Z x in tree order (leaf blocks plus every butterfly, Sec. III-A)."""
        b = self.bounds
        y = np.zeros(x.shape, dtype=np.result_type(x, np.complex128))
        lb = b[self.LH]
        for i in range(2 ** self.LH):
            y[lb[i]:lb[i + 1]] = self.D[i] @ x[lb[i]:lb[i + 1]]
        for (l, i), bf in self.B.items():
            sib = i ^ 1
            y[b[l][i]:b[l][i + 1]] += bf.apply(x[b[l][sib]:b[l][sib + 1]])
        return y

    def dense(self) -> np.ndarray:
        n = self.bounds[0][-1]
        return self.apply(np.eye(n, dtype=np.complex128))

    def entries(self) -> int:
        return sum(d.size for d in self.D) + sum(bf.entries() for bf in self.B.values())

    def max_rank(self) -> int:
        return max((max(max(r) for r in bf.ranks() if len(r)) for bf in self.B.values()), default=0)


class HODBFInverse:
    """Algorithm 1 from its dense definition, each E_tau compressed as a butterfly."""

    def __init__(self, A: np.ndarray, bounds, LH: int, tol: float, construct: str = "id"):
        """A: dense matrix in tree order (e.g. the densified compressed operator).

        construct = "id": each E_tau is compressed by IDs of its entries (Eqs. 7-10);
        "random": by products with E_tau and E_tau^H only (BF_random_matvec of Sec. III-B),
        each product computed from the definition E_tau X = M^-1 X - X without forming E_tau."""
        self.bounds, self.LH = bounds, LH
        lb = bounds[LH]
        self.Dinv = [np.linalg.inv(A[lb[i]:lb[i + 1], lb[i]:lb[i + 1]]) for i in range(2 ** LH)]
        self.E = {}
        for l in range(LH - 1, -1, -1):
            for i in range(2 ** l):
                a, m, b = bounds[l][i], bounds[l + 1][2 * i + 1], bounds[l][i + 1]
                D1 = A[a:m, a:m]
                D2 = A[m:b, m:b]
                B1 = np.linalg.solve(D1, A[a:m, m:b])
                B2 = np.linalg.solve(D2, A[m:b, a:m])
                M = np.eye(b - a, dtype=np.complex128)
                M[:m - a, m - a:] = B1
                M[m - a:, :m - a] = B2
                L = LH - l
                ob = sub_bounds(bounds, l, i, L)
                if construct == "random":
                    from .bf_random import RandomButterfly

                    lu = sla.lu_factor(M)
                    mv = lambda X, lu=lu: sla.lu_solve(lu, X) - X  # noqa: E731
                    rmv = lambda Y, lu=lu: sla.lu_solve(lu, Y, trans=2) - Y  # noqa: E731
                    self.E[(l, i)] = RandomButterfly(mv, rmv, ob, ob, L, tol, seed=l * 1000 + i)
                else:
                    E = np.linalg.inv(M) - np.eye(b - a)
                    self.E[(l, i)] = Butterfly(lambda r, c, E=E, a=a: E[np.ix_(r - a, c - a)], ob, ob, L, tol)

    def apply(self, x: np.ndarray) -> np.ndarray:
        b = self.bounds
        y = np.zeros(x.shape, dtype=np.result_type(x, np.complex128))
        lb = b[self.LH]
        for i in range(2 ** self.LH):
            y[lb[i]:lb[i + 1]] = self.Dinv[i] @ x[lb[i]:lb[i + 1]]
        for l in range(self.LH - 1, -1, -1):
            for i in range(2 ** l):
                s = slice(b[l][i], b[l][i + 1])
                y[s] = y[s] + self.E[(l, i)].apply(y[s])
        return y

    def entries(self) -> int:
        return sum(d.size for d in self.Dinv) + sum(e.entries() for e in self.E.values())
