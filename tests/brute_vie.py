"""Brute-force Galerkin entries of the D-VIE for pinning the oracle (test helper).

Written independently of oracle/entries.py: it takes the mesh arrays only
(vertices, tets, faces, T+/T-, eps per tet), builds its own SWG data and
integrates every term of the entry formula (Eq. 5 in the normalized form, with
the distributional divergences of half-SWG faces and charge jumps) by nested
Gauss rules whose inner integral removes the 1/R singularity by construction:

* the source tetrahedron is split into the four cones from the observation
  point r to its faces (signed volumes, valid for r inside or outside), and in
  a cone r' = r + t (y - r) the volume element t^2 h dt dA_y cancels the 1/R
  of the kernel;
* every face (of a cone, or a source triangle) is split into the three
  triangles from the projection rho of r to its edges (signed areas), in polar
  form y = rho + s (z - rho); the remaining near-singular factor s / |y - r|
  is made smooth by s = a sinh(tau), a = dist(r, plane) / |z - rho|.

All rules are Gauss-Legendre in collapsed coordinates; nothing here shares a
formula with the closed-form potentials or the conical rules of the oracle.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial.legendre import leggauss

FOUR_PI = 4.0 * np.pi


def gl(n, a=0.0, b=1.0):
    x, w = leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def tet_points(P, n):
    """Collapsed Gauss rule on the tetrahedron P (4, 3): points (q, 3), weights (q,)."""
    u, wu = gl(n)
    U, V, W = np.meshgrid(u, u, u, indexing="ij")
    WW = (wu[:, None, None] * wu[None, :, None] * wu[None, None, :]).ravel()
    U, V, W = U.ravel(), V.ravel(), W.ravel()
    a, b, c, d = P
    x = a + U[:, None] * ((b - a) + V[:, None] * ((c - b) + W[:, None] * (d - c)))
    vol6 = abs(np.dot(np.cross(b - a, c - a), d - a))
    return x, WW * U * U * V * vol6


def tri_points(T, n):
    u, wu = gl(n)
    U, V = np.meshgrid(u, u, indexing="ij")
    WW = (wu[:, None] * wu[None, :]).ravel()
    U, V = U.ravel(), V.ravel()
    a, b, c = T
    x = a + U[:, None] * ((b - a) + V[:, None] * (c - b))
    ar2 = np.linalg.norm(np.cross(b - a, c - a))
    return x, WW * U * ar2


def _sinh_nodes(lo, hi, c, eps, n):
    """Gauss nodes and weights on [lo, hi] after w = c + eps sinh(sigma) (clusters at c; arrays (m,))."""
    x, wx = leggauss(n)
    a = np.arcsinh((lo - c) / eps)
    b = np.arcsinh((hi - c) / eps)
    sg = 0.5 * (b - a)[:, None] * x[None, :] + 0.5 * (b + a)[:, None]
    w = c[:, None] + eps[:, None] * np.sinh(sg)
    return w, 0.5 * (b - a)[:, None] * wx[None, :] * eps[:, None] * np.cosh(sg)


def _face_polar(r, F, n_s, n_w):
    """Polar decomposition of triangle F (3, 3) around the projections of the points r (m, 3).

    Yields (y, wt, hs) per sub-triangle: y (m, q, 3) the points, wt (m, q) the weights of
    int_F phi(y) / |y - r| dA (the 1/|y - r| included), hs (m,) the signed distance.  Along the
    edge the nodes cluster (sinh map) at the foot of rho, where |z - rho| is smallest."""
    a, b, c = F
    nrm = np.cross(b - a, c - a)
    nrm = nrm / np.linalg.norm(nrm)
    hs = (r - a) @ nrm                       # (m,)
    rho = r - hs[:, None] * nrm               # projections
    m = len(r)
    tau, wt_tau = gl(n_s)
    for p, q in ((a, b), (b, c), (c, a)):
        e = q - p
        le2 = e @ e
        w0 = ((rho - p) @ e) / le2                                   # foot of rho on the edge line
        de = np.linalg.norm(rho - p - w0[:, None] * e, axis=1) / np.sqrt(le2)
        eps = np.maximum(np.sqrt(de * de + (hs * hs) / le2), 1e-12)  # distance of r to the edge line / |e|
        wc = np.clip(w0, 0.0, 1.0)
        inside = (w0 > 0.0) & (w0 < 1.0)
        # two pieces [0, wc], [wc, 1] (one of them empty when the foot is outside the edge)
        W1, V1 = _sinh_nodes(np.zeros(m), wc, wc, eps, n_w)
        W2, V2 = _sinh_nodes(wc, np.ones(m), wc, eps, n_w)
        V1 = np.where(inside[:, None] | (w0[:, None] >= 1.0), V1, 0.0)
        V2 = np.where(inside[:, None] | (w0[:, None] <= 0.0), V2, 0.0)
        w = np.concatenate([W1, W2], 1)                               # (m, nw2)
        ww = np.concatenate([V1, V2], 1)
        z = p[None, None, :] + w[:, :, None] * e[None, None, :]        # (m, nw2, 3)
        zr = z - rho[:, None, :]
        L = np.linalg.norm(zr, axis=-1)                              # (m, nw2)
        sarea2 = np.cross(p - rho, q - rho) @ nrm                     # signed 2 x area, (m,)
        Ls = np.where(L > 0, L, 1.0)
        A = np.abs(hs)[:, None] / Ls                                  # (m, nw2)
        # s = A sinh(t'), t' in [0, asinh(1/A)]; s ds / |y - r| = A sinh(t') dt' / L
        tmax = np.arcsinh(1.0 / np.maximum(A, 1e-300))
        small = A < 1e-13
        tp = tau[None, None, :] * tmax[:, :, None]                    # (m, nw2, ns)
        s = np.where(small[:, :, None], tau[None, None, :], A[:, :, None] * np.sinh(tp))
        jac = np.where(small[:, :, None], 1.0 / Ls[:, :, None], A[:, :, None] * np.sinh(tp) * tmax[:, :, None] / Ls[:, :, None])
        wgt = jac * wt_tau[None, None, :] * ww[:, :, None] * sarea2[:, None, None]
        y = rho[:, None, None, :] + s[..., None] * zr[:, :, None, :]
        yield y.reshape(m, -1, 3), wgt.reshape(m, -1), hs


def inner_tri(r, F, dens, k0, n_s=16, n_w=12):
    """int_F dens(y) exp(-j k0 |y - r|) / (4 pi |y - r|) dA for points r (m, 3) -> (m, ...)."""
    out = 0.0
    for y, wt, _ in _face_polar(r, F, n_s, n_w):
        R = np.linalg.norm(y - r[:, None, :], axis=-1)
        val = dens(y) * (wt * np.exp(-1j * k0 * R) / FOUR_PI)[(...,) + (None,) * (dens(y).ndim - 2)]
        out = out + val.sum(1)
    return out


def inner_tet(r, P, dens, k0, n_s=16, n_w=12, n_t=8):
    """int_T dens(r') exp(-j k0 |r' - r|) / (4 pi |r' - r|) dv' over the tetrahedron P (4, 3)."""
    t, wt = gl(n_t)
    out = 0.0
    for f in ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)):
        F = P[list(f)]
        opp = P[[i for i in range(4) if i not in f][0]]
        # orient F so that its normal points out of the tetrahedron
        if np.dot(np.cross(F[1] - F[0], F[2] - F[0]), F[0] - opp) < 0:
            F = F[[0, 2, 1]]
        nrm = np.cross(F[1] - F[0], F[2] - F[0])
        nrm = nrm / np.linalg.norm(nrm)
        for y, wy, _ in _face_polar(r, F, n_s, n_w):
            hsig = (F[0] - r) @ nrm                                   # (m,) signed height of the cone
            d = y - r[:, None, :]                                      # (m, q, 3)
            rho = np.linalg.norm(d, axis=-1)                           # (m, q)
            # cone: dv' = t^2 h dt dA, kernel exp(-j k t rho) / (4 pi t rho): t h / (4 pi rho) ...
            acc = 0.0
            for ti, wti in zip(t, wt):
                x = r[:, None, :] + ti * d
                val = dens(x)
                fac = wti * ti * np.exp(-1j * k0 * ti * rho) / FOUR_PI
                acc = acc + val * fac[(...,) + (None,) * (val.ndim - 2)]
            # the polar weights carry 1/|y - r| = 1/rho already
            out = out + (acc * (wy * hsig[:, None])[(...,) + (None,) * (acc.ndim - 2)]).sum(1)
    return out


class Brute:
    """Z(m, n) of Eq. 5 for a voxel/Kuhn mesh given as arrays, by brute force."""

    def __init__(self, verts, tets, faces, face_tp, face_tm, eps_tet, k0):
        self.V, self.T, self.F = verts, tets, faces
        self.tp, self.tm = face_tp, face_tm
        self.eps = eps_tet
        self.kap = (eps_tet - 1.0) / eps_tet
        self.k0 = k0

    def _swg(self, f, t):
        """(c, p, div) of SWG f in tet t: f = c (r - p), div = 3 c."""
        P = self.V[self.T[t]]
        fv = set(self.F[f].tolist())
        p = self.V[[v for v in self.T[t] if v not in fv][0]]
        A, B, C = self.V[self.F[f]]
        area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
        vol = abs(np.dot(np.cross(P[1] - P[0], P[2] - P[0]), P[3] - P[0])) / 6.0
        sgn = 1.0 if t == self.tp[f] else -1.0
        c = sgn * area / (3.0 * vol)
        return c, p, 3.0 * c

    def _tets(self, f):
        return [t for t in (self.tp[f], self.tm[f]) if t >= 0]

    def entry(self, m, n, n_out=10):
        k0 = self.k0
        z = 0.0 + 0.0j
        jump_n = (self.kap[self.tm[n]] if self.tm[n] >= 0 else 0.0) - self.kap[self.tp[n]]
        bnd_m = self.tm[m] < 0
        for T in self._tets(m):
            cm, pm, dm = self._swg(m, T)
            PT = self.V[self.T[T]]
            ro, wo = tet_points(PT, n_out)
            for Tp in self._tets(n):
                cn, pn, dn = self._swg(n, Tp)
                Pp = self.V[self.T[Tp]]
                if T == Tp:  # Gram term, observation tet's 1 / eps_r
                    z += (wo * cm * cn * np.einsum("qi,qi->q", ro - pm, ro - pn)).sum() / self.eps[T]
                dens = lambda x, pn=pn: np.concatenate([x - pn, np.ones(x.shape[:-1] + (1,))], -1)
                I = inner_tet(ro, Pp, dens, k0)                     # (q, 4): vector part, scalar part
                vec = cn * I[:, :3]
                sca = I[:, 3]
                z += -k0 * k0 * self.kap[Tp] * (wo * cm * np.einsum("qi,qi->q", ro - pm, vec)).sum()
                z += self.kap[Tp] * dm * dn * (wo * sca).sum()
            if jump_n != 0.0:
                Fn = self.V[self.F[n]]
                one = lambda x: np.ones(x.shape[:-1])
                z += jump_n * dm * (wo * inner_tri(ro, Fn, one, k0)).sum()
        if bnd_m:
            Fm = self.V[self.F[m]]
            rs, ws = tri_points(Fm, n_out + 4)
            for Tp in self._tets(n):
                cn, pn, dn = self._swg(n, Tp)
                one = lambda x: np.ones(x.shape[:-1])
                z += -1.0 * self.kap[Tp] * dn * (ws * inner_tet(rs, self.V[self.T[Tp]], one, k0)).sum()
            if jump_n != 0.0:
                one = lambda x: np.ones(x.shape[:-1])
                z += -1.0 * jump_n * (ws * inner_tri(rs, self.V[self.F[n]], one, k0)).sum()
        return z


def _entry_task(args):
    br, m, n, n_out = args
    return br.entry(m, n, n_out=n_out)


def entries(br: Brute, pairs, n_out=10, procs=None) -> np.ndarray:
    """br.entry for every (m, n) in pairs, one pair per worker process (started with spawn)."""
    import multiprocessing as mp
    import os

    pairs = list(pairs)
    procs = min(len(pairs), procs or max(1, os.cpu_count() or 1))
    if procs <= 1:
        return np.array([br.entry(m, n, n_out=n_out) for m, n in pairs])
    with mp.get_context("spawn").Pool(procs) as pool:
        return np.array(pool.map(_entry_task, [(br, m, n, n_out) for m, n in pairs]))
