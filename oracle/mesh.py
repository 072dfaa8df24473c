"""Voxel body -> tetrahedral mesh -> SWG face table (oracle; test infrastructure only).

Sec. II / Eq. (3): the scatterer is discretized by a tetrahedral mesh with N
faces and one SWG basis function per face.  Reading of the mesh rule: each
voxel with lower corner v0 is split into the 6 Kuhn tetrahedra
[v0, v0+e_p0, v0+e_p0+e_p1, v0+(1,1,1)] over the 6 permutations p of the axes
(itertools order), which gives a conforming mesh on the voxel lattice.

Numbering (a definition both implementations follow):
  * tets: voxel-major in the order of the input voxel list, then permutation
    index 0..5;
  * vertices: unique lattice points sorted lexicographically by (i, j, k);
  * faces: unique sorted vertex-id triples sorted lexicographically;
    T+ = the lower tet id holding the face, T- = the other one or -1 on the
    boundary (half-SWG);
  * local face a of a tet is the face opposite its local vertex a.
"""
from __future__ import annotations

import itertools

import numpy as np

PERMS = list(itertools.permutations(range(3)))  # (0,1,2),(0,2,1),(1,0,2),(1,2,0),(2,0,1),(2,1,0)


def kuhn_offsets() -> np.ndarray:
    """(6, 4, 3) integer offsets of the Kuhn tetrahedra's vertices from the voxel corner."""
    out = np.zeros((6, 4, 3), dtype=np.int64)
    for t, p in enumerate(PERMS):
        v = np.zeros(3, dtype=np.int64)
        out[t, 0] = v
        for s in range(3):
            v = v.copy()
            v[p[s]] += 1
            out[t, s + 1] = v
    return out


def build_mesh(body) -> dict:
    """Build the tet mesh and the SWG face table of a ``workloads.VoxelBody``."""
    h = float(body.h)
    vox = np.asarray(body.ijk, dtype=np.int64)
    nvox = len(vox)
    off = kuhn_offsets()
    tet_lat = (vox[:, None, None, :] + off[None, :, :, :]).reshape(nvox * 6, 4, 3)  # lattice coords
    # unique vertices, lexicographic (i, j, k)
    flat = tet_lat.reshape(-1, 3)
    uniq, inv = np.unique(flat, axis=0, return_inverse=True)
    tets = inv.reshape(nvox * 6, 4).astype(np.int64)
    verts = uniq.astype(np.float64) * h
    nt = len(tets)
    tet_vox = np.repeat(np.arange(nvox), 6)
    tet_type = np.tile(np.arange(6), nvox)
    eps = np.repeat(np.asarray(body.eps, dtype=np.complex128), 6)

    # faces: local face a is opposite local vertex a
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tri = np.sort(tets[:, loc], axis=2).reshape(-1, 3)  # (nt*4, 3)
    faces, finv = np.unique(tri, axis=0, return_inverse=True)
    finv = finv.reshape(nt, 4)
    nf = len(faces)
    tp = np.full(nf, -1, dtype=np.int64)
    tm = np.full(nf, -1, dtype=np.int64)
    lp = np.full(nf, -1, dtype=np.int64)
    lm = np.full(nf, -1, dtype=np.int64)
    for t in range(nt):  # plain loop: tets in increasing id, so the first holder is T+
        for a in range(4):
            f = finv[t, a]
            if tp[f] < 0:
                tp[f], lp[f] = t, a
            else:
                assert tm[f] < 0, "a face is shared by at most two tets"
                tm[f], lm[f] = t, a
    return dict(h=h, verts=verts, tets=tets, tet_vox=tet_vox, tet_type=tet_type,
                vox_ijk=vox, eps=eps, faces=faces, face_tp=tp, face_tm=tm,
                face_lp=lp, face_lm=lm, tet_faces=finv)


def tet_geometry(mesh: dict) -> dict:
    """Per-tet volume and per (tet, local face) area, outward unit normal and SWG data.

    SWG (Eq. 3, Schaubert-Wilton-Glisson): for face n with area a_n,
    f_n(r) = +a_n/(3 V+) (r - p+) in T+ and -a_n/(3 V-) (r - p-) in T-, with p
    the vertex opposite the face; the normal flux across face n is 1 and the
    divergence is +-a_n/V+-.
    """
    P = mesh["verts"][mesh["tets"]]  # (nt, 4, 3)
    e1, e2, e3 = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]
    vol = np.abs(np.einsum("ij,ij->i", np.cross(e1, e2), e3)) / 6.0
    nt = len(P)
    area = np.zeros((nt, 4))
    normal = np.zeros((nt, 4, 3))
    for a in range(4):
        idx = [b for b in range(4) if b != a]
        A, B, C = P[:, idx[0]], P[:, idx[1]], P[:, idx[2]]
        n = np.cross(B - A, C - A)
        ln = np.linalg.norm(n, axis=1)
        n = n / ln[:, None]
        # orient outward: away from the opposite vertex
        s = np.sign(np.einsum("ij,ij->i", n, A - P[:, a]))
        normal[:, a] = n * s[:, None]
        area[:, a] = 0.5 * ln
    # SWG sign per (tet, local face): +1 if the tet is T+ of that face
    tf = mesh["tet_faces"]
    sign = np.where(mesh["face_tp"][tf] == np.arange(nt)[:, None], 1.0, -1.0)
    return dict(P=P, vol=vol, area=area, normal=normal, sign=sign)


def swg_eval(geo: dict, t: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Values of the 4 SWG functions of tets t at points r: (..., 4, 3).

    r has shape (len(t), q, 3); returns (len(t), q, 4, 3) with
    f_a(r) = s_a a_a / (3 V) (r - p_a).
    """
    P = geo["P"][t]  # (m, 4, 3)
    c = geo["sign"][t] * geo["area"][t] / (3.0 * geo["vol"][t][:, None])  # (m, 4)
    return c[:, None, :, None] * (r[:, :, None, :] - P[:, None, :, :])


def swg_div(geo: dict, t: np.ndarray) -> np.ndarray:
    """Divergence of the 4 SWG functions of tets t: s_a a_a / V, shape (len(t), 4)."""
    return geo["sign"][t] * geo["area"][t] / geo["vol"][t][:, None]


def tier_cells(verts: np.ndarray, tets: np.ndarray):
    """Cell pitch and per-tet cells of the quadrature-tier rule on a general tet mesh.

    Reading of the tier rule beyond voxel meshes (the paper is silent): the cell pitch
    h_c is the mean over the tets (in id order) of each tet's shortest edge, and tet t
    lives in cell floor(c_t / h_c) of its centroid c_t = (P0 + P1 + P2 + P3) / 4.  On a
    voxel/Kuhn mesh the shortest edge of every tet is the voxel pitch and each centroid
    lies at least h/4 inside its voxel, so the cells are the voxels and the rule is the
    voxel rule.  Every step is written with +, -, *, / and sqrt in a fixed order (no
    library reductions), so any implementation that follows it gets the same cells.
    (The entries also treat any two elements whose tets share a vertex as near; see
    oracle.entries.)"""
    P = verts[tets]
    nt = len(tets)
    emin = np.full(nt, np.inf)
    for a in range(4):
        for b in range(a + 1, 4):
            d = P[:, b] - P[:, a]
            emin = np.minimum(emin, np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]))
    s = 0.0
    for v in emin.tolist():  # sequential sum in tet order
        s += v
    hc = s / nt
    c = (((P[:, 0] + P[:, 1]) + P[:, 2]) + P[:, 3]) * 0.25
    return hc, np.floor(c / hc).astype(np.int64)


def build_mesh_general(verts, tets, eps) -> dict:
    """SWG face table of a general tetrahedral mesh (Sec. II, Eq. 3): vertices (nv, 3),
    tets (nt, 4) vertex ids in any orientation, eps (nt,) complex relative permittivity
    per tet.  Numbering as in ``build_mesh``: vertices and tets as given; faces are the
    unique sorted vertex-id triples sorted lexicographically; T+ is the lower tet id
    holding a face; local face a is opposite local vertex a.  The quadrature tiers use
    the cells of ``tier_cells`` in place of voxels."""
    verts = np.asarray(verts, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    nt = len(tets)
    hc, cells = tier_cells(verts, tets)
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tri = np.sort(tets[:, loc], axis=2).reshape(-1, 3)
    faces, finv = np.unique(tri, axis=0, return_inverse=True)
    finv = finv.reshape(nt, 4)
    nf = len(faces)
    tp = np.full(nf, -1, dtype=np.int64)
    tm = np.full(nf, -1, dtype=np.int64)
    lp = np.full(nf, -1, dtype=np.int64)
    lm = np.full(nf, -1, dtype=np.int64)
    for t in range(nt):
        for a in range(4):
            f = finv[t, a]
            if tp[f] < 0:
                tp[f], lp[f] = t, a
            else:
                assert tm[f] < 0, "a face is shared by at most two tets"
                tm[f], lm[f] = t, a
    return dict(h=hc, verts=verts, tets=tets, tet_vox=np.arange(nt), tet_type=np.full(nt, -1),
                vox_ijk=cells, eps=np.asarray(eps, dtype=np.complex128), faces=faces, face_tp=tp,
                face_tm=tm, face_lp=lp, face_lm=lm, tet_faces=finv)
