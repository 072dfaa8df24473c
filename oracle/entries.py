"""Galerkin SWG entries of the D-VIE (oracle; test infrastructure only).

Eqs. (1)-(5), Sec. II.  With lambda0 = 1, k0 = 2 pi, d = D / eps0, eps_r and
kappa = (eps_r - 1)/eps_r per tetrahedron, -j omega eta0 (-j k0) = -k0^2/eps0
(Eq. 1 with Eq. 2), and after multiplying the tested equation by eps0 the
entries read (Eq. 5; reading Q1: the integrand of L acts on X(r'), reading
Q2: eta = eta0):

  Z(m, n) =   int f_m . f_n / eps_r dv                              (Gram)
            - k0^2 int int f_m(r) . kappa(r') f_n(r') g(r, r') dv' dv  (vector potential)
            + int int (div f_m)(r) (div' kappa f_n)(r') g(r, r') dv' dv (scalar potential)

  g = exp(-j k0 R) / (4 pi R)  (exp(+j omega t) convention, Sec. II)

Both divergences are distributional: div f_m has the volume part +-a_m/V+- and,
for a boundary (half-SWG) face, the surface density -1 on face m;
div'(kappa f_n) has the volume part +-kappa a_n/V+- and the surface density
kappa(T-) - kappa(T+) on face n (kappa(T-) = 0 outside the body).

  V(m) = int f_m . E_inc dv,  E_inc = pol exp(-j k0 khat . r).

Quadrature (the paper is silent; reading shared as a specification by both
implementations).  The tier of an element pair is the Chebyshev distance D of
the voxels holding them (a surface element lives in the voxel of its T+):
  D >= 3  far:  tet4 x tet4, tri3 x tri3 on the full kernel;
  D == 2  mid:  tet_conical(2) x tet_conical(2), tri_conical(2) on the full kernel;
  D <= 1  near: singularity subtraction g = 1/(4 pi R) + g_s.  The 1/R part is
        integrated over the source element in closed form (the potential of a
        uniform triangle, Wilton et al. 1984 / Graglia 1993; for a tetrahedron
        reduced to its faces by div'((r'-r)/R) = 2/R and int grad' R = sum_f n_f
        int_f R), then over the observation element with tet_conical(3) /
        tri_conical(3); the smooth remainder g_s = (exp(-j k0 R) - 1)/(4 pi R)
        uses tet_conical(2) / tri_conical(2) on both sides.
  Gram term: tet4 (exact for the quadratic integrand).
On a general tet mesh (mesh.build_mesh_general) the voxels are replaced by the
tier cells of mesh.tier_cells, and a pair of elements whose tets share a vertex is
near (D <= 1) whatever its cells, so touching elements always take the singular
treatment; on a voxel mesh tets that share a vertex lie in voxels at distance <= 1,
so the voxel rule is unchanged.
"""
from __future__ import annotations

import numpy as np

from . import quadrature as Q
from .mesh import swg_div, swg_eval, tet_geometry

FOUR_PI = 4.0 * np.pi

# The quadrature specification (see the module docstring).  Tests may swap in
# higher orders to check that the specification has converged.
RULES = {
    "far_tet": lambda: Q.tet4(), "far_tri": lambda: Q.tri3(),
    "mid_tet": lambda: Q.tet_conical(2), "mid_tri": lambda: Q.tri_conical(2),
    "near_tet": lambda: Q.tet_conical(3), "near_tri": lambda: Q.tri_conical(3),
    "smooth_tet": lambda: Q.tet_conical(2), "smooth_tri": lambda: Q.tri_conical(2),
}
_LOCAL_FACE = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])


# ----------------------------------------------------------------------------------
# kernels
# ----------------------------------------------------------------------------------

def green(R, k0):
    return np.exp(-1j * k0 * R) / (FOUR_PI * R)


def green_smooth(R, k0):
    """(exp(-j k0 R) - 1) / (4 pi R), written without cancellation; limit -j k0/(4 pi) at R = 0."""
    x = k0 * R
    safe = np.where(R > 0, R, 1.0)
    val = (-2.0 * np.sin(0.5 * x) ** 2 - 1j * np.sin(x)) / (FOUR_PI * safe)
    return np.where(R > 0, val, -1j * k0 / FOUR_PI)


# ----------------------------------------------------------------------------------
# closed-form potentials of a flat triangle (Wilton et al. 1984; Graglia 1993)
# ----------------------------------------------------------------------------------

def tri_potentials(r, A, B, C):
    """I_m1 = int_T 1/|r - r'| ds' and I_1 = int_T |r - r'| ds' for points r.

    r, A, B, C broadcast to (..., 3).  With d the signed height of r over the
    plane, rho its projection and, per edge i, t0 the in-plane distance from
    rho to the edge line (positive inside), l+- the edge-end coordinates
    along the edge and R+- the distances to the edge ends:
      I_m1 = sum_i t0_i f_i - |d| sum_i beta_i,
      f_i  = ln((R+ + l+)/(R- + l-)),
      beta_i = atan(t0 l+/(R0^2 + |d| R+)) - atan(t0 l-/(R0^2 + |d| R-)),
      I_1  = (d^2 I_m1 + 1/2 sum_i t0_i (R0_i^2 f_i + l+ R+ - l- R-)) / 3,
    the last from div_s((rho' - rho) R) = 3R - d^2/R and the edge integral of R.
    """
    r, A, B, C = np.broadcast_arrays(r, A, B, C)
    n = np.cross(B - A, C - A)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    d = np.einsum("...i,...i->...", r - A, n)
    ad = np.abs(d)
    rho = r - d[..., None] * n
    Im1 = np.zeros(d.shape)
    S1 = np.zeros(d.shape)
    for P1, P2 in ((A, B), (B, C), (C, A)):
        e = P2 - P1
        le = np.linalg.norm(e, axis=-1, keepdims=True)
        lh = e / le
        uh = np.cross(lh, n)
        t0 = np.einsum("...i,...i->...", P1 - rho, uh)
        lp = np.einsum("...i,...i->...", P2 - rho, lh)
        lm = np.einsum("...i,...i->...", P1 - rho, lh)
        R02 = t0 * t0 + d * d
        Rp = np.sqrt(lp * lp + R02)
        Rm = np.sqrt(lm * lm + R02)
        tiny = 1e-30 + 1e-24 * (lp * lp + lm * lm)
        ok = R02 > tiny
        R02s = np.where(ok, R02, 1.0)
        num = np.where(lp >= 0, Rp + lp, R02s / np.where(Rp - lp > 0, Rp - lp, 1.0))
        den = np.where(lm >= 0, Rm + lm, R02s / np.where(Rm - lm > 0, Rm - lm, 1.0))
        f = np.where(ok, np.log(np.where(ok, num, 1.0) / np.where(ok, den, 1.0)), 0.0)
        beta = np.where(ok, np.arctan2(t0 * lp, R02s + ad * Rp) - np.arctan2(t0 * lm, R02s + ad * Rm), 0.0)
        # arctan2(y, x) with x > 0 equals atan(y/x)
        Im1 += t0 * f - ad * beta
        S1 += t0 * (R02 * f + lp * Rp - lm * Rm)
    I1 = (d * d * Im1 + 0.5 * S1) / 3.0
    return Im1, I1


def tet_potentials(r, P, normals):
    """U = int_T 1/R dv' and W = int_T (r' - r)/R dv' for points r and tets with vertices P.

    U = 1/2 sum_f h_f int_f 1/R ds'  (h_f = n_f . (x_f - r), n_f outward),
    W = sum_f n_f int_f R ds'.
    r: (m, q, 3); P: (m, 4, 3); normals: (m, 4, 3).  Returns U (m, q), W (m, q, 3).
    """
    U = np.zeros(r.shape[:-1])
    W = np.zeros(r.shape)
    for a in range(4):
        i0, i1, i2 = _LOCAL_FACE[a]
        A, B, C = P[:, None, i0], P[:, None, i1], P[:, None, i2]
        nf = normals[:, None, a]
        h = np.einsum("mqi,mqi->mq", A - r, np.broadcast_to(nf, r.shape))
        Im1, I1 = tri_potentials(r, A, B, C)
        U += 0.5 * np.where(np.abs(h) > 0, h * Im1, 0.0)
        W += nf * I1[..., None]
    return U, W


# ----------------------------------------------------------------------------------
# element data
# ----------------------------------------------------------------------------------

class Elements:
    """Geometry and quadrature points of the tets and faces of a mesh."""

    def __init__(self, mesh: dict, k0: float):
        self.mesh = mesh
        self.k0 = float(k0)
        self.geo = tet_geometry(mesh)
        eps = mesh["eps"]
        self.kappa = (eps - 1.0) / eps
        self.inv_eps = 1.0 / eps
        fp, fm = mesh["face_tp"], mesh["face_tm"]
        kp = self.kappa[fp]
        km = np.where(fm >= 0, self.kappa[np.maximum(fm, 0)], 0.0)
        self.jump = km - kp                   # source surface density on face n
        self.boundary = fm < 0                # half-SWG faces carry the test density -1
        self.face_tri = mesh["verts"][mesh["faces"]]  # (nf, 3, 3)
        self.face_vox = mesh["vox_ijk"][mesh["tet_vox"][fp]]
        self.tet_vox = mesh["vox_ijk"][mesh["tet_vox"]]
        self.general = bool(np.all(np.asarray(mesh["tet_type"]) < 0))  # general tet mesh: tier cells
        self.tet_ids = np.asarray(mesh["tets"])
        self.face_owner = fp
        self.face_area = 0.5 * np.linalg.norm(
            np.cross(self.face_tri[:, 1] - self.face_tri[:, 0], self.face_tri[:, 2] - self.face_tri[:, 0]), axis=1)

    # quadrature points
    def tet_rule(self, t, rule):
        lam, w = rule
        P = self.geo["P"][t]
        pts = np.einsum("qa,mai->mqi", lam, P)
        return pts, w[None, :] * self.geo["vol"][t][:, None]

    def tri_rule(self, f, rule):
        lam, w = rule
        T = self.face_tri[f]
        pts = np.einsum("qa,mai->mqi", lam, T)
        return pts, w[None, :] * self.face_area[f][:, None]


def _tier(va, vb):
    return np.abs(va[:, None, :] - vb[None, :, :]).max(-1)


def _share_vertex(E, ta, tb, grid: bool):
    """Whether tets ta and tb share a vertex: for every (ta[i], tb[j]) (grid) or (ta[i], tb[i])."""
    A, B = E.tet_ids[ta], E.tet_ids[tb]
    if grid:
        return (A[:, None, :, None] == B[None, :, None, :]).any((-1, -2))
    return (A[:, :, None] == B[:, None, :]).any((-1, -2))


# ----------------------------------------------------------------------------------
# tet-tet blocks: P[T, T'][a, b] = Gram + (-k0^2 kappa_T' A + kappa_T' div_a div_b Phi)
# ----------------------------------------------------------------------------------

def _vol_vol_full(E, to, ts, rule_o, rule_s):
    """Full-kernel A[a, b] and Phi for pairs (to[i], ts[i])."""
    ro, wo = E.tet_rule(to, rule_o)
    rs, ws = E.tet_rule(ts, rule_s)
    R = np.linalg.norm(ro[:, :, None, :] - rs[:, None, :, :], axis=-1)
    G = green(R, E.k0) * wo[:, :, None] * ws[:, None, :]
    fo = swg_eval(E.geo, to, ro)
    fs = swg_eval(E.geo, ts, rs)
    A = np.einsum("piad,pij,pjbd->pab", fo, G, fs, optimize=True)
    return A, G.sum((1, 2))


def _vol_vol_near(E, to, ts):
    k0 = E.k0
    # static 1/R part: closed form over the source, tet_conical(3) over the observer
    ro, wo = E.tet_rule(to, RULES["near_tet"]())
    U, W = tet_potentials(ro, E.geo["P"][ts], E.geo["normal"][ts])
    fo = swg_eval(E.geo, to, ro)                                   # (p, q, 4, 3)
    Ps = E.geo["P"][ts]
    cs = E.geo["sign"][ts] * E.geo["area"][ts] / (3.0 * E.geo["vol"][ts][:, None])  # (p, 4)
    # int_T' f_b(r')/R dv' = c_b (W + (r - p_b) U)
    inner = cs[:, None, :, None] * (W[:, :, None, :] + (ro[:, :, None, :] - Ps[:, None, :, :]) * U[:, :, None, None])
    A = np.einsum("pq,pqad,pqbd->pab", wo, fo, inner, optimize=True) / FOUR_PI
    Phi = (wo * U).sum(1) / FOUR_PI
    # smooth remainder
    ro2, wo2 = E.tet_rule(to, RULES["smooth_tet"]())
    rs2, ws2 = E.tet_rule(ts, RULES["smooth_tet"]())
    R = np.linalg.norm(ro2[:, :, None, :] - rs2[:, None, :, :], axis=-1)
    G = green_smooth(R, k0) * wo2[:, :, None] * ws2[:, None, :]
    fo2 = swg_eval(E.geo, to, ro2)
    fs2 = swg_eval(E.geo, ts, rs2)
    A = A + np.einsum("piad,pij,pjbd->pab", fo2, G, fs2, optimize=True)
    Phi = Phi + G.sum((1, 2))
    return A, Phi


def tet_pair_blocks(E, to, ts):
    """(len(to), len(ts), 4, 4) contributions of every tet pair to the SWG entries."""
    k0 = E.k0
    tier = _tier(E.tet_vox[to], E.tet_vox[ts])
    if E.general:
        tier = np.where(_share_vertex(E, to, ts, grid=True), np.minimum(tier, 1), tier)
    I, J = np.meshgrid(np.arange(len(to)), np.arange(len(ts)), indexing="ij")
    out = np.zeros((len(to), len(ts), 4, 4), dtype=np.complex128)
    div_o = swg_div(E.geo, to)
    div_s = swg_div(E.geo, ts)
    for mask, kind in ((tier >= 3, "far"), (tier == 2, "mid"), (tier <= 1, "near")):
        ii, jj = I[mask], J[mask]
        for s in range(0, len(ii), 20000):
            a, b = ii[s:s + 20000], jj[s:s + 20000]
            if kind == "far":
                A, Phi = _vol_vol_full(E, to[a], ts[b], RULES["far_tet"](), RULES["far_tet"]())
            elif kind == "mid":
                A, Phi = _vol_vol_full(E, to[a], ts[b], RULES["mid_tet"](), RULES["mid_tet"]())
            else:
                A, Phi = _vol_vol_near(E, to[a], ts[b])
            kap = E.kappa[ts[b]][:, None, None]
            blk = -k0 * k0 * kap * A + kap * div_o[a][:, :, None] * div_s[b][:, None, :] * Phi[:, None, None]
            out[a, b] += blk
    # Gram term on coincident tets (tet4 is exact for the quadratic integrand)
    same = to[:, None] == ts[None, :]
    ii, jj = np.nonzero(same)
    if len(ii):
        t = to[ii]
        r, w = E.tet_rule(t, Q.tet4())
        f = swg_eval(E.geo, t, r)
        Gm = np.einsum("pq,pqad,pqbd->pab", w, f, f)
        out[ii, jj] += E.inv_eps[t][:, None, None] * Gm
    return out


# ----------------------------------------------------------------------------------
# surface elements (scalar-potential terms only)
# ----------------------------------------------------------------------------------

def _pair_scalar(E, kind_o, eo, kind_s, es, tier):
    """int int g over element pairs; kind 't' (tet) or 'f' (face)."""
    k0 = E.k0
    out = np.zeros(len(eo), dtype=np.complex128)

    def rule(kind, e, level):
        if kind == "t":
            return E.tet_rule(e, RULES[level + "_tet"]())
        return E.tri_rule(e, RULES[level + "_tri"]())

    for sel, lvl in ((tier >= 3, "far"), (tier == 2, "mid")):
        idx = np.nonzero(sel)[0]
        if len(idx) == 0:
            continue
        ro, wo = rule(kind_o, eo[idx], lvl)
        rs, ws = rule(kind_s, es[idx], lvl)
        R = np.linalg.norm(ro[:, :, None, :] - rs[:, None, :, :], axis=-1)
        out[idx] = (green(R, k0) * wo[:, :, None] * ws[:, None, :]).sum((1, 2))
    idx = np.nonzero(tier <= 1)[0]
    if len(idx):
        ro, wo = rule(kind_o, eo[idx], "near")
        if kind_s == "t":
            U, _ = tet_potentials(ro, E.geo["P"][es[idx]], E.geo["normal"][es[idx]])
        else:
            T = E.face_tri[es[idx]]
            U, _ = tri_potentials(ro, T[:, None, 0], T[:, None, 1], T[:, None, 2])
        val = (wo * U).sum(1) / FOUR_PI
        ro2, wo2 = rule(kind_o, eo[idx], "smooth")
        rs2, ws2 = rule(kind_s, es[idx], "smooth")
        R = np.linalg.norm(ro2[:, :, None, :] - rs2[:, None, :, :], axis=-1)
        val = val + (green_smooth(R, k0) * wo2[:, :, None] * ws2[:, None, :]).sum((1, 2))
        out[idx] = val
    return out


# ----------------------------------------------------------------------------------
# assembly of Z(rows, cols)
# ----------------------------------------------------------------------------------

def _incidence(mesh, faces):
    """Tets touching the faces and the (tet, local face) -> column map."""
    tp, tm = mesh["face_tp"][faces], mesh["face_tm"][faces]
    tets = np.unique(np.concatenate([tp, tm[tm >= 0]]))
    pos = {f: i for i, f in enumerate(faces)}
    tf = mesh["tet_faces"][tets]  # (nt, 4)
    rows, cols = [], []
    for i in range(len(tets)):
        for a in range(4):
            j = pos.get(int(tf[i, a]))
            if j is not None:
                rows.append(4 * i + a)
                cols.append(j)
    from scipy.sparse import csr_matrix

    M = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(4 * len(tets), len(faces)))
    return tets, M


def _all_pairs(E, kind_o, eo, kind_s, es, chunk: int = 40000):
    """int int g for every (eo[i], es[j]) element pair: (len(eo), len(es))."""
    vo = E.tet_vox[eo] if kind_o == "t" else E.face_vox[eo]
    vs = E.tet_vox[es] if kind_s == "t" else E.face_vox[es]
    I, J = np.meshgrid(np.arange(len(eo)), np.arange(len(es)), indexing="ij")
    I, J = I.ravel(), J.ravel()
    out = np.zeros(len(I), dtype=np.complex128)
    for s in range(0, len(I), chunk):
        a, b = I[s:s + chunk], J[s:s + chunk]
        tier = np.abs(vo[a] - vs[b]).max(1)
        if E.general:
            ta = eo[a] if kind_o == "t" else E.face_owner[eo[a]]
            tb = es[b] if kind_s == "t" else E.face_owner[es[b]]
            tier = np.where(_share_vertex(E, ta, tb, grid=False), np.minimum(tier, 1), tier)
        out[s:s + chunk] = _pair_scalar(E, kind_o, eo[a], kind_s, es[b], tier)
    return out.reshape(len(eo), len(es))


def zblock(E: Elements, rows, cols, chunk: int = 256) -> np.ndarray:
    """Z(rows, cols) of Eq. (5), complex128, plain sum over element pairs."""
    mesh = E.mesh
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    to, Mo = _incidence(mesh, rows)
    ts, Ms = _incidence(mesh, cols)
    Z = np.zeros((len(rows), len(cols)), dtype=np.complex128)
    for s in range(0, len(to), chunk):
        blk = tet_pair_blocks(E, to[s:s + chunk], ts)          # (c, nts, 4, 4)
        c = blk.shape[0]
        Pm = blk.transpose(0, 2, 1, 3).reshape(4 * c, 4 * len(ts))
        Z += (Mo[4 * s:4 * s + 4 * c].T @ (Ms.T @ Pm.T).T)
    bnd = np.nonzero(E.boundary[rows])[0]          # row positions of half-SWG faces
    jmp = np.nonzero(np.abs(E.jump[cols]) > 0)[0]  # column positions of faces with a charge jump
    if len(bnd):
        # test surface (density -1 on boundary face m) x source volume rho_n = kappa div f_n
        SV = _all_pairs(E, "f", rows[bnd], "t", ts)                        # (nb, nts)
        fac = (E.kappa[ts][:, None] * swg_div(E.geo, ts)).reshape(-1)       # (4 nts,)
        SVx = np.repeat(SV, 4, axis=1) * fac[None, :]
        Z[bnd] += -1.0 * (Ms.T @ SVx.T).T
    if len(jmp):
        # test volume div f_m x source surface (density jump on face n)
        VS = _all_pairs(E, "t", to, "f", cols[jmp])                         # (nto, nj)
        VSx = np.repeat(VS, 4, axis=0) * swg_div(E.geo, to).reshape(-1)[:, None]
        Z[:, jmp] += (Mo.T @ VSx) * E.jump[cols[jmp]][None, :]
        if len(bnd):
            SS = _all_pairs(E, "f", rows[bnd], "f", cols[jmp])
            Z[np.ix_(bnd, jmp)] += -1.0 * SS * E.jump[cols[jmp]][None, :]
    return Z


def rhs_planewave(E: Elements, khat, pol, rows=None) -> np.ndarray:
    """V(m) = int f_m . pol exp(-j k0 khat . r) dv (Eq. 5), tet_conical(3); (N, nrhs).

    With `rows` (face ids), only those entries are formed, from the tets that
    touch them: (len(rows), nrhs)."""
    mesh = E.mesh
    if rows is None:
        t = np.arange(len(mesh["tets"]))
    else:
        rows = np.asarray(rows, dtype=np.int64)
        t = np.unique(np.concatenate([mesh["face_tp"][rows], mesh["face_tm"][rows]]))
        t = t[t >= 0]
    r, w = E.tet_rule(t, Q.tet_conical(3))
    f = swg_eval(E.geo, t, r)  # (nt, q, 4, 3)
    khat = np.atleast_2d(khat)
    pol = np.atleast_2d(pol)
    V = np.zeros((len(mesh["faces"]), len(khat)), dtype=np.complex128)
    for j in range(len(khat)):
        ph = np.exp(-1j * E.k0 * (r @ khat[j]))  # (nt, q)
        val = np.einsum("tq,tqad,d->ta", w * ph, f, pol[j])
        np.add.at(V[:, j], mesh["tet_faces"][t].ravel(), val.ravel())
    return V if rows is None else V[rows]
