"""HOD-BF inverse built from products only (Sec. III-B: Algorithm 1 line 7 and Algorithm 2,
BF_random_matvec), on the GPU, against the oracle's product-only construction
(oracle/bf_smw.HODBFInverseSMW) and against the identity Zinv Z = I; adjoint applies
(the products with A^H the construction needs) against the inner-product identity."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402
from oracle.bf_smw import HODBFInverseSMW  # noqa: E402
from oracle.hodbf import HODBF, cluster_tree, face_centroids  # noqa: E402


@pytest.fixture(scope="module")
def oracle_smw(lossy_sphere):
    """The oracle's Algorithms 1-2 from products (dense blocks below 512 unknowns, like the GPU)."""
    mesh, Z = lossy_sphere["mesh"], lossy_sphere["Z"]
    perm, LH, bounds = cluster_tree(face_centroids(mesh), 64)
    Zt = Z[np.ix_(perm, perm)]
    Hd = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, 1e-4).dense()
    return perm, LH, {tf: HODBFInverseSMW(Hd, bounds, LH, tf, dense_max=512) for tf in (1e-2, 1e-3)}


@pytest.mark.parametrize("tol_fact", [1e-2, 1e-3])
def test_product_inverse_against_oracle(lossy_sphere, oracle_smw, tol_fact):
    Z = lossy_sphere["Z"]
    perm, LH, inv = oracle_smw
    # inv_dense_max = 1: every level above the leaves from products only
    op = pkg.Operator(lossy_sphere["body"], W.K0, tol_con=1e-4, tol_fact=tol_fact, leaf=64, inv_dense_max=1)
    st = op.get_stats()
    assert st.zinv_top_level == 0 and st.zinv_product_levels == LH and st.inverse_products > 0
    bound = 10 * tol_fact  # each construction reaches about chi_fact (Sec. III-B); both sit within it
    x = W.random_block(op.n, 2, seed=31)
    y = op.apply(torch.from_numpy(Z @ x).to(torch.complex64).cuda(), op=pkg.VIE_OP_ZINV).cpu().numpy()
    err_gpu = np.linalg.norm(y - x) / np.linalg.norm(x)
    xo = x[perm]
    err_or = np.linalg.norm(inv[tol_fact].apply(Z[np.ix_(perm, perm)] @ xo) - xo) / np.linalg.norm(xo)
    assert err_gpu <= bound and err_or <= bound, (err_gpu, err_or)
    # the two product-built inverses agree to the same order (tree order <-> face order)
    v = W.random_block(op.n, 1, seed=32)
    yo = np.zeros_like(v)
    yo[perm] = inv[tol_fact].apply(v[perm])
    yg = op.apply(torch.from_numpy(v).to(torch.complex64).cuda(), op=pkg.VIE_OP_ZINV).cpu().numpy()
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) <= bound


@pytest.mark.parametrize("nrhs", [1, 3, 20])
def test_adjoint_applies(lossy_sphere, nrhs):
    """<y, A x> = <A^H y, x> for A = Z and Zinv (SIMT kernels below 16 columns, tensor cores above)."""
    op = pkg.Operator(lossy_sphere["body"], W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64, inv_dense_max=1)
    x = torch.from_numpy(W.random_block(op.n, nrhs, seed=1)).to(torch.complex64).cuda()
    y = torch.from_numpy(W.random_block(op.n, nrhs, seed=2)).to(torch.complex64).cuda()
    for which, adj in ((pkg.VIE_OP_Z, pkg.VIE_OP_ZH), (pkg.VIE_OP_ZINV, pkg.VIE_OP_ZINVH)):
        ax = op.apply(x, op=which)
        ahy = op.apply(y, op=adj)
        lhs = torch.sum(y.conj() * ax).item()
        rhs = torch.sum(ahy.conj() * x).item()
        assert abs(lhs - rhs) <= 1e-4 * abs(lhs), (which, nrhs, lhs, rhs)


def test_product_inverse_at_52k_unknowns():
    """Sphere r = 1 lambda0 (N = 52,584): the levels whose nodes exceed 4,096 unknowns (four of
    them) from products only; chi_fact 1e-3 gives Zinv Z within 1e-2 of the identity."""
    body = W.sphere(1.0, 4.0 - 0.1j, 1.0 / 10)
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-3, leaf=64, inv_dense_max=4096)
    st = op.get_stats()
    assert op.n == 52584 and st.zinv_top_level == 0 and st.zinv_product_levels >= 4
    x = torch.from_numpy(W.random_block(op.n, 2, seed=21)).to(torch.complex64).cuda()
    y = op.apply(op.apply(x), op=pkg.VIE_OP_ZINV)
    err = (torch.linalg.norm(y - x) / torch.linalg.norm(x)).item()
    assert err <= 1e-2, err
    op.check()
