"""GPU HOD-BF inverse (Algorithm 1) against the oracle's dense-defined HOD-BF inverse."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402
from oracle.dense import solve_dense  # noqa: E402
from oracle.entries import rhs_planewave  # noqa: E402
from oracle.hodbf import HODBF, HODBFInverse, cluster_tree, face_centroids  # noqa: E402


@pytest.fixture(scope="module")
def oracle_inv(lossy_sphere):
    mesh, Z = lossy_sphere["mesh"], lossy_sphere["Z"]
    perm, LH, bounds = cluster_tree(face_centroids(mesh), 64)
    Zt = Z[np.ix_(perm, perm)]
    H = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, 1e-4)
    Hd = H.dense()
    return perm, {tf: HODBFInverse(Hd, bounds, LH, tf) for tf in (1e-1, 1e-3)}


@pytest.mark.parametrize("tol_fact,bound", [(1e-1, 0.5), (1e-3, 3e-2)])
def test_zinv_quality_and_parity(lossy_sphere, oracle_inv, tol_fact, bound):
    Z = lossy_sphere["Z"]
    op = pkg.Operator(lossy_sphere["body"], W.K0, tol_con=1e-4, tol_fact=tol_fact, leaf=64)
    st = op.get_stats()
    assert st.entries_zinv > 0 and st.apply_stages_zinv > 1
    x = W.random_block(op.n, 2, seed=21)
    zx = torch.from_numpy(Z @ x).to(torch.complex64).cuda()
    y = op.apply(zx, op=pkg.VIE_OP_ZINV).cpu().numpy()
    assert np.linalg.norm(y - x) / np.linalg.norm(x) <= bound
    # against the oracle's inverse of the same operator (tree order <-> face order)
    perm, inv = oracle_inv
    v = W.random_block(op.n, 1, seed=22)
    yo = np.zeros_like(v)
    yo[perm] = inv[tol_fact].apply(v[perm])
    yg = op.apply(torch.from_numpy(v).to(torch.complex64).cuda(), op=pkg.VIE_OP_ZINV).cpu().numpy()
    # both inverses sit within `bound` of Z^-1 (row sampling on the GPU, full rows in the oracle)
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) <= bound


def test_preconditioned_solve(lossy_sphere):
    body, E, Z = lossy_sphere["body"], lossy_sphere["E"], lossy_sphere["Z"]
    plain = pkg.Operator(body, W.K0, tol_con=1e-5, leaf=64)
    pre = pkg.Operator(body, W.K0, tol_con=1e-5, tol_fact=1e-1, leaf=64)
    k, p = W.planewave_random(2, seed=4)
    V = pre.rhs_planewave(k, p)
    I0, it0, rel0, st0 = plain.solve(V, rtol=1e-6, restart=60, max_iter=600)
    I1, it1, rel1, st1 = pre.solve(V, rtol=1e-6, restart=60, max_iter=600)
    assert st0 == pkg.VIE_OK and st1 == pkg.VIE_OK
    assert it1.max() < it0.min()
    Io = solve_dense(Z, rhs_planewave(E, k, p))
    assert np.linalg.norm(I1.cpu().numpy() - Io) / np.linalg.norm(Io) < 1e-3
