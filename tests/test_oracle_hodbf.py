"""Pins of the oracle HOD-BF (Sec. III-A, Eqs. 7-10) and its inverse (Sec. III-B, Algorithm 1)."""
import numpy as np
import pytest

import workloads as W
from oracle.hodbf import HODBF, HODBFInverse, cluster_tree, face_centroids, interp_decomp, tree_depth


def test_tree_is_balanced_kd_bisection():
    pts = np.random.default_rng(3).random((1000, 3)) * [3.0, 1.0, 2.0]
    perm, LH, bounds = cluster_tree(pts, 64)
    assert LH == tree_depth(1000, 64) == 4
    assert sorted(perm.tolist()) == list(range(1000))
    for l in range(LH):
        b, c = bounds[l], bounds[l + 1]
        for i in range(len(b) - 1):
            lo, mid, hi = c[2 * i], c[2 * i + 1], c[2 * i + 2]
            assert lo == b[i] and hi == b[i + 1] and mid - lo == (hi - lo + 1) // 2
            p = pts[perm[lo:hi]]
            ax = int(np.argmax(p.max(0) - p.min(0)))
            assert pts[perm[lo:mid], ax].max() <= pts[perm[mid:hi], ax].min()
    assert np.diff(bounds[LH]).max() <= 64


def test_id_recovers_exact_rank():
    rng = np.random.default_rng(0)
    for m, n, k in ((40, 30, 7), (100, 64, 20), (10, 50, 10)):
        A = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))) @ (
            rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n)))
        J, V = interp_decomp(A, 1e-10)
        assert len(J) == k
        assert np.linalg.norm(A - A[:, J] @ V) < 1e-12 * np.linalg.norm(A)
        assert np.allclose(V[:, J], np.eye(k))


@pytest.fixture(scope="module")
def tree_Z(lossy_sphere):
    perm, LH, bounds = cluster_tree(face_centroids(lossy_sphere["mesh"]), 64)
    Zt = lossy_sphere["Z"][np.ix_(perm, perm)]
    return Zt, bounds, LH


def test_id_error_and_rank_vs_svd(tree_Z):
    Zt, bounds, LH = tree_Z
    tol = 1e-4
    for l in (1, 2, 3):
        a, m, b = bounds[l][0], bounds[l][1], bounds[l][2]
        A = Zt[a:m, m:b]
        J, V = interp_decomp(A, tol)
        assert np.linalg.norm(A - A[:, J] @ V) <= 10 * tol * np.linalg.norm(A)
        s = np.linalg.svd(A, compute_uv=False)
        r_svd = int(np.sum(s > tol * s[0]))
        assert r_svd <= len(J) <= 2 * r_svd + 4


@pytest.mark.parametrize("tol,bound", [(1e-2, 5e-2), (1e-3, 5e-3), (1e-4, 5e-4)])
def test_hodbf_apply_vs_dense(tree_Z, tol, bound):
    Zt, bounds, LH = tree_Z
    H = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, tol)
    X = W.random_block(len(Zt), 3, seed=11)
    assert np.linalg.norm(H.apply(X) - Zt @ X) <= bound * np.linalg.norm(Zt @ X)


def test_butterfly_ranks_shrink_off_the_middle(tree_Z):
    """Complementary low-rank property (Sec. III-A): butterfly ranks stay far below block sizes."""
    Zt, bounds, LH = tree_Z
    H = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, 1e-4)
    bf = H.B[(1, 0)]
    n = bounds[1][1]
    assert max(max(r) for r in bf.ranks()) < n / 4


@pytest.mark.parametrize("tol_fact,bound", [(1e-1, 0.5), (1e-3, 1e-2)])
def test_inverse_quality(tree_Z, tol_fact, bound):
    Zt, bounds, LH = tree_Z
    H = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, 1e-4)
    Hd = H.dense()
    Hi = HODBFInverse(Hd, bounds, LH, tol_fact)
    x = W.random_block(len(Zt), 2, seed=5)
    err = np.linalg.norm(Hi.apply(Hd @ x) - x) / np.linalg.norm(x)
    assert err <= bound


# ---- butterflies from products only (BF_random_matvec of Sec. III-B) ----------------

from oracle.bf_random import RandomButterfly  # noqa: E402
from oracle.hodbf import Butterfly, sub_bounds  # noqa: E402


def _level1_block(tree_Z):
    Zt, bounds, LH = tree_Z
    L = LH - 1
    ob, sb = sub_bounds(bounds, 1, 0, L), sub_bounds(bounds, 1, 1, L)
    return Zt[ob[0][0]:ob[0][-1], sb[0][0]:sb[0][-1]], ob, sb, L


def test_random_butterfly_exact_on_low_rank_block(tree_Z):
    """A rank-6 block is reproduced to rounding: every sketch sees the whole range."""
    _, ob, sb, L = _level1_block(tree_Z)
    rng = np.random.default_rng(2)
    m, n = ob[0][-1] - ob[0][0], sb[0][-1] - sb[0][0]
    A = (rng.standard_normal((m, 6)) + 1j * rng.standard_normal((m, 6))) @ (
        rng.standard_normal((6, n)) + 1j * rng.standard_normal((6, n)))
    rb = RandomButterfly(lambda X: A @ X, lambda Y: A.conj().T @ Y, ob, sb, L, 1e-12)
    x = W.random_block(n, 2, seed=3)
    assert np.linalg.norm(rb.apply(x) - A @ x) < 1e-10 * np.linalg.norm(A @ x)


@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_random_butterfly_accuracy_and_product_count(tree_Z, tol):
    """On a VIE off-diagonal block: error within 10 tol like the ID butterfly, storage of the same
    order, and no more product columns than the two half-depth sweeps need."""
    A, ob, sb, L = _level1_block(tree_Z)
    rb = RandomButterfly(lambda X: A @ X, lambda Y: A.conj().T @ Y, ob, sb, L, tol, p=8)
    x = W.random_block(A.shape[1], 2, seed=4)
    assert np.linalg.norm(rb.apply(x) - A @ x) <= 10 * tol * np.linalg.norm(A @ x)
    bf = Butterfly(lambda r, c: A[np.ix_(r - ob[0][0], c - sb[0][0])], ob, sb, L, tol)
    assert rb.entries() <= 2 * bf.entries()
    h = L // 2
    widest = int(max(np.diff(ob[L]).max(), np.diff(sb[L]).max()))  # largest leaf of either tree
    rmax = max([v.shape[0] for v in rb.V] + [u.shape[0] for Ut in rb.U for Ui in Ut for u in Ui])
    assert rb.products <= (2 ** (h + 1) + 2 ** (L - h + 1)) * (max(rmax, widest) + 8)


@pytest.mark.parametrize("tol_fact,bound", [(1e-1, 0.5), (1e-3, 1e-2)])
def test_inverse_from_products_quality(tree_Z, tol_fact, bound):
    """Algorithm 1 with every E_tau built from products with E_tau and E_tau^H only."""
    Zt, bounds, LH = tree_Z
    H = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, 1e-4)
    Hd = H.dense()
    Hi = HODBFInverse(Hd, bounds, LH, tol_fact, construct="random")
    x = W.random_block(len(Zt), 2, seed=5)
    err = np.linalg.norm(Hi.apply(Hd @ x) - x) / np.linalg.norm(x)
    assert err <= bound


def test_inverse_by_bf_smw_from_products(tree_Z):
    """Algorithms 1 and 2 as written: B'_tau from products with the children's inverses, E_tau by
    the recursive Sherman-Morrison-Woodbury split into quadrant butterflies, every butterfly built
    from products with the operator and its adjoint.  Same quality bound as the other
    constructions at chi_fact 1e-3, and the adjoint apply is the exact adjoint."""
    from oracle.bf_smw import HODBFInverseSMW

    Zt, bounds, LH = tree_Z
    H = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, 1e-4)
    Hd = H.dense()
    Hi = HODBFInverseSMW(Hd, bounds, LH, 1e-3, dense_max=128)
    x = W.random_block(len(Zt), 2, seed=5)
    assert np.linalg.norm(Hi.apply(Hd @ x) - x) / np.linalg.norm(x) <= 1e-2
    y, z = W.random_block(len(Zt), 2, seed=9).T
    lhs = np.vdot(y, Hi.apply(z))
    assert abs(lhs - np.vdot(Hi.apply(y, adjoint=True), z)) <= 1e-12 * abs(lhs)
