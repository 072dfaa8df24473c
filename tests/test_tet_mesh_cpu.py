"""General tetrahedral meshes on the CPU: the oracle's general mesh path pinned to its voxel
path (a Kuhn mesh given as a general mesh) and to the brute-force integration of Eq. 5 on
jittered, non-lattice tets; the library's host face table and tier cells against the oracle,
bit for bit; invalid meshes refused."""
import os

import numpy as np
import pytest

import workloads as W
from oracle.entries import Elements, zblock
from oracle.mesh import build_mesh, build_mesh_general

from test_oracle_entries import _raised_rules


def _probe_body():
    ijk = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [3, 0, 0], [0, 0, 3]], dtype=np.int32)
    eps = np.array([4 - 0.5j, 2 - 0.2j, 6 - 1j, 3 - 0.1j, 5 - 0.3j])
    return W.VoxelBody("probe", 0.1, ijk, eps)


def test_general_oracle_reduces_to_the_voxel_path():
    """A Kuhn voxel mesh handed to the general path: the same face table, cells equal to the
    voxels, and the same entries (every tier, every surface term) to rounding."""
    body = _probe_body()
    mv = build_mesh(body)
    mg = build_mesh_general(mv["verts"], mv["tets"], mv["eps"])
    for k in ("faces", "face_tp", "face_tm", "face_lp", "face_lm", "tet_faces"):
        assert np.array_equal(mv[k], mg[k]), k
    assert np.array_equal(mv["vox_ijk"][mv["tet_vox"]], mg["vox_ijk"][mg["tet_vox"]])
    n = len(mv["faces"])
    rows = np.arange(0, n, 3)
    cols = np.arange(1, n, 2)
    Zv = zblock(Elements(mv, W.K0), rows, cols)
    Zg = zblock(Elements(mg, W.K0), rows, cols)
    assert np.abs(Zv - Zg).max() <= 1e-12 * np.abs(Zv).max()


@pytest.fixture(scope="module")
def jittered():
    """The probe voxels cut into five tets each, every vertex jittered by up to 0.08 h."""
    from brute_vie import Brute, entries

    tm_ = W.tet_body(_probe_body(), jitter=0.08, seed=3)
    mesh = build_mesh_general(tm_.verts, tm_.tets, tm_.eps)
    E = Elements(mesh, W.K0)
    tp, tm = mesh["face_tp"], mesh["face_tm"]
    inter = np.nonzero(tm >= 0)[0]
    bnd = np.nonzero(tm < 0)[0]
    vox_of_tet = np.arange(len(mesh["tets"])) // 5
    jump = [f for f in inter if vox_of_tet[tp[f]] != vox_of_tet[tm[f]]]
    far = [f for f in range(len(tp)) if vox_of_tet[tp[f]] == 3][0]
    mid = [f for f in range(len(tp)) if vox_of_tet[tp[f]] == 4][0]
    near = [(inter[0], inter[0]), (bnd[0], bnd[0]), (jump[0], jump[0]), (inter[0], jump[0]),
            (jump[0], bnd[0]), (bnd[0], inter[0])]
    sep = [(inter[0], far), (bnd[0], mid), (far, jump[0])]
    br = Brute(mesh["verts"], mesh["tets"], mesh["faces"], tp, tm, mesh["eps"], W.K0)
    zb_near = entries(br, near, n_out=8)
    zb_sep = entries(br, sep, n_out=5)
    return E, near, sep, zb_near, zb_sep


def test_jittered_entries_vs_brute_force(jittered):
    """Off-lattice tets of two shapes (corner and central tets of the five-tet split): the
    oracle at raised rule orders against the brute-force integration, with the bounds of the
    voxel pin (near pairs 1e-4, separated pairs 1e-6)."""
    E, near, sep, zb_near, zb_sep = jittered
    with _raised_rules(near=20, smooth=10, far=8):
        zo = np.array([zblock(E, [m], [k])[0, 0] for m, k in near])
        zs = np.array([zblock(E, [m], [k])[0, 0] for m, k in sep])
    assert (np.abs(zo - zb_near) / np.abs(zb_near)).max() < 1e-4
    assert (np.abs(zs - zb_sep) / np.abs(zb_sep)).max() < 1e-6


def test_jittered_pin_catches_a_wrong_face_normal(jittered):
    """A planted mistake in the general geometry (the outward normals of the source tets
    flipped in the closed-form potentials) fails the brute-force pin."""
    E, near, sep, zb_near, zb_sep = jittered
    saved = E.geo["normal"].copy()
    try:
        E.geo["normal"] = -E.geo["normal"]
        with _raised_rules(near=20, smooth=10, far=8):
            zo = np.array([zblock(E, [m], [k])[0, 0] for m, k in near])
    finally:
        E.geo["normal"] = saved
    assert (np.abs(zo - zb_near) / np.abs(zb_near)).max() > 1e-2


def test_touching_elements_are_near():
    """On a jittered mesh, every pair of tets that share a vertex is in the near tier, whatever
    their cells (the singular treatment is never skipped)."""
    tm_ = W.tet_body(W.sphere(0.15, 4.0, 1.0 / 20), jitter=0.12, seed=9)
    mesh = build_mesh_general(tm_.verts, tm_.tets, tm_.eps)
    E = Elements(mesh, W.K0)
    from oracle.entries import _share_vertex, _tier

    t = np.arange(len(mesh["tets"]))
    tier = _tier(E.tet_vox[t], E.tet_vox[t])
    share = _share_vertex(E, t, t, grid=True)
    eff = np.where(share, np.minimum(tier, 1), tier)
    assert eff[share].max() <= 1


lib_needed = pytest.mark.skipif(
    not os.path.exists(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                    "paper_2111_01730_gb300", "libvie.so")),
    reason="libvie.so not built")


@lib_needed
@pytest.mark.parametrize("case", ["sphere_tet5", "shell_tet5", "kuhn"])
def test_host_face_table_and_cells_match_oracle(case):
    import paper_2111_01730_gb300 as pkg

    if case == "kuhn":
        body = W.sphere(0.2, 4.0, 1.0 / 20)
        mv = build_mesh(body)

        class M:
            pass

        m = M()
        m.verts, m.tets, m.eps = mv["verts"], mv["tets"], mv["eps"]
    elif case == "shell_tet5":
        m = W.tet_body(W.shell(0.25, 0.15, -2 - 0.2j, 1.0 / 20), jitter=0.1, seed=2)
    else:
        m = W.tet_body(W.sphere(0.2, 4.0 - 0.1j, 1.0 / 20), jitter=0.08, seed=1)
    r = pkg.mesh_host_tets(m, leaf=32)
    o = build_mesh_general(m.verts, m.tets, m.eps)
    assert np.array_equal(r["faces"], o["faces"])
    assert np.array_equal(r["tp"], o["face_tp"]) and np.array_equal(r["tm"], o["face_tm"])
    assert np.array_equal(r["cells"], o["vox_ijk"]) and r["cell_pitch"] == o["h"]
    if case == "kuhn":  # the same tree as the voxel path
        assert np.array_equal(r["perm"], pkg.mesh_host(body, leaf=32)["perm"])


@lib_needed
def test_host_rejects_invalid_meshes():
    import paper_2111_01730_gb300 as pkg

    base = W.tet_body(W.sphere(0.1, 4.0, 1.0 / 20), jitter=0.05, seed=4)

    class M:
        def __init__(self, v, t, e):
            self.verts, self.tets, self.eps = v, t, e

    bad_id = base.tets.copy()
    bad_id[0, 0] = len(base.verts)
    rep = base.tets.copy()
    rep[0, 1] = rep[0, 0]
    flat = base.verts.copy()
    t0 = base.tets[0]
    flat[t0[3]] = flat[t0[0]]  # two coincident vertices: zero volume
    triple = np.concatenate([base.tets, base.tets[:1]])
    eps3 = np.concatenate([base.eps, base.eps[:1]])
    zero_eps = base.eps.copy()
    zero_eps[0] = 0.0
    for m in (M(base.verts, bad_id, base.eps), M(base.verts, rep, base.eps), M(flat, base.tets, base.eps),
              M(base.verts, triple, eps3), M(base.verts, base.tets, zero_eps)):
        with pytest.raises(pkg.VieError) as e:
            pkg.mesh_host_tets(m, leaf=32)
        assert e.value.status == pkg.VIE_EINVAL


def test_jittered_reciprocity_and_zero_contrast():
    """Off-lattice tets: a homogeneous body's Galerkin matrix is symmetric in the continuum, so
    the asymmetry is the quadrature error of the two sides alone.  On 16 faces at raised orders
    it is 2.1e-6 of max |Z| (the voxel mesh: 7e-8; distorted tets converge more slowly under
    the collapsed rules), at the worst pair (two touching half-SWG faces) it falls below 1e-6
    with the orders raised once more; with eps_r = 1 only the Gram term is left, which is real,
    symmetric and exact."""
    tm_ = W.tet_body(W.tiny_block(2, 2, 1, h=0.1, eps=3.0 - 0.2j), jitter=0.1, seed=8)
    mesh = build_mesh_general(tm_.verts, tm_.tets, tm_.eps)
    E = Elements(mesh, W.K0)
    n = len(mesh["faces"])
    sel = np.random.default_rng(4).choice(n, size=16, replace=False)
    with _raised_rules(near=12, smooth=6, far=8):
        Zh = zblock(E, sel, sel)
    scale = np.abs(Zh).max()
    d = np.abs(Zh - Zh.T)
    assert d.max() < 3e-6 * scale
    i, j = np.unravel_index(d.argmax(), d.shape)
    with _raised_rules(near=16, smooth=8, far=8):
        a = zblock(E, [sel[i]], [sel[j]])[0, 0]
        b = zblock(E, [sel[j]], [sel[i]])[0, 0]
    assert abs(a - b) < min(1e-6 * scale, 0.5 * d.max())
    vac = build_mesh_general(tm_.verts, tm_.tets, np.ones(len(tm_.tets), dtype=np.complex128))
    Z0 = zblock(Elements(vac, W.K0), np.arange(n), np.arange(n))
    assert np.allclose(Z0.imag, 0.0, atol=1e-15) and np.allclose(Z0, Z0.T, atol=1e-15)
    assert np.all(np.linalg.eigvalsh(Z0.real) > 0)  # Gram matrix of independent SWG functions


@lib_needed
@pytest.mark.parametrize("offset", [(0.0, 0.0, 0.0), (37.3, -12.05, 101.7)])
def test_host_cells_bit_exact_off_origin(offset):
    """The tier cells and their pitch come out bit for bit the same in the library and the
    oracle also for a mesh far from the origin, where floor(centroid / pitch) is most exposed to
    rounding (both follow the same fixed sequence of +, -, *, / and sqrt)."""
    import paper_2111_01730_gb300 as pkg

    m = W.tet_body(W.sphere(0.15, 4.0, 1.0 / 20), jitter=0.11, seed=12)
    verts = m.verts + np.asarray(offset)
    m2 = W.TetMesh("shifted", verts, m.tets, m.eps)
    r = pkg.mesh_host_tets(m2, leaf=32)
    o = build_mesh_general(verts, m.tets, m.eps)
    assert r["cell_pitch"] == o["h"]
    assert np.array_equal(r["cells"], o["vox_ijk"])
    assert np.array_equal(r["faces"], o["faces"])
