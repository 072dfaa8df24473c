"""Pins of the voxel/Kuhn mesh and the SWG basis (Sec. II, Eq. 3)."""
import numpy as np
import pytest

import workloads as W
from oracle.mesh import build_mesh, swg_div, swg_eval, tet_geometry


def exposed_faces(ijk):
    s = set(map(tuple, ijk))
    n = 0
    for v in s:
        for ax in range(3):
            for d in (-1, 1):
                w = list(v)
                w[ax] += d
                n += tuple(w) not in s
    return n


@pytest.mark.parametrize("body,n_expect", [
    (W.sphere(0.3, 4.0, 1 / 14), 3960),
    (W.sphere(0.3, 4.0, 1 / 20), 11616),
    (W.tiny_block(2, 1, 1), None),
])
def test_face_count_closed_form(body, n_expect):
    mesh = build_mesh(body)
    n = len(mesh["faces"])
    assert n == 12 * body.nvox + exposed_faces(body.ijk)
    if n_expect is not None:
        assert n == n_expect
    assert len(mesh["tets"]) == 6 * body.nvox
    # each face held by one or two tets; boundary faces = 2 per exposed voxel face
    assert np.sum(mesh["face_tm"] < 0) == 2 * exposed_faces(body.ijk)


def test_tets_fill_voxels_and_swg_flux():
    body = W.tiny_block(2, 2, 1, h=0.1)
    mesh = build_mesh(body)
    geo = tet_geometry(mesh)
    assert np.allclose(geo["vol"], 0.1 ** 3 / 6, rtol=1e-13)
    # normal flux of f_n across its own face is 1 on both sides (constant over the face)
    for n in range(len(mesh["faces"])):
        for T, a in ((mesh["face_tp"][n], mesh["face_lp"][n]), (mesh["face_tm"][n], mesh["face_lm"][n])):
            if T < 0:
                continue
            tri = mesh["verts"][mesh["faces"][n]]
            pts = np.array([tri.mean(0), tri[0] * 0.6 + tri[1] * 0.2 + tri[2] * 0.2])
            f = swg_eval(geo, np.array([T]), pts[None])[0, :, a]
            nrm = geo["normal"][T, a] * (1.0 if mesh["face_tp"][n] == T else -1.0)
            assert np.allclose(f @ nrm, 1.0, atol=1e-12)
    # divergence = s a / V
    div = swg_div(geo, np.arange(len(mesh["tets"])))
    assert np.allclose(np.abs(div), geo["area"] / geo["vol"][:, None])


def test_constant_field_is_in_swg_span():
    """A constant field c equals sum_n (c . n_n) f_n with n_n oriented from T+ to T-."""
    body = W.tiny_block(2, 1, 1, h=0.1)
    mesh = build_mesh(body)
    geo = tet_geometry(mesh)
    c = np.array([0.3, -1.2, 0.7])
    coef = np.zeros(len(mesh["faces"]))
    for n in range(len(mesh["faces"])):
        T, a = mesh["face_tp"][n], mesh["face_lp"][n]
        coef[n] = c @ geo["normal"][T, a]
    rng = np.random.default_rng(1)
    for T in range(len(mesh["tets"])):
        lam = rng.dirichlet(np.ones(4), size=3)
        pts = lam @ geo["P"][T]
        f = swg_eval(geo, np.array([T]), pts[None])[0]  # (3, 4, 3)
        d = np.einsum("qad,a->qd", f, coef[mesh["tet_faces"][T]])
        assert np.allclose(d, c[None, :], atol=1e-12)
