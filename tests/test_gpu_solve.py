"""GPU solve (GMRES + FP64 refinement) against the oracle's dense LU and Mie."""
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


def test_solve_matches_dense_lu(lossy_sphere):
    body, E, Z = lossy_sphere["body"], lossy_sphere["E"], lossy_sphere["Z"]
    op = pkg.Operator(body, W.K0, tol_con=1e-6, leaf=64)
    k, p = W.planewave_random(3, seed=2)
    V = op.rhs_planewave(k, p)
    I, iters, rel, st = op.solve(V, rtol=1e-6, restart=40, max_iter=400)
    assert st == pkg.VIE_OK, (iters, rel)
    assert np.all(rel <= 1e-6)
    Io = solve_dense(Z, rhs_planewave(E, k, p))
    err = np.linalg.norm(I.cpu().numpy() - Io) / np.linalg.norm(Io)
    assert err < 1e-3, err


def test_solve_reports_nonconvergence_and_nan(lossy_sphere):
    op = pkg.Operator(lossy_sphere["body"], W.K0, tol_con=1e-4, leaf=64)
    k, p = W.planewave_x_along_z()
    V = op.rhs_planewave(k, p)
    I, iters, rel, st = op.solve(V, rtol=1e-12, restart=5, max_iter=10)
    assert st == pkg.VIE_ENOTCONV and iters[0] == 10 and rel[0] > 1e-12
    V[3, 0] = float("nan")
    with pytest.raises(pkg.VieError) as e:
        op.solve(V, rtol=1e-6)
    assert e.value.status == pkg.VIE_ENAN


@pytest.mark.parametrize("tol_fact", [0.0, 1e-1])
def test_tfqmr_matches_dense_lu(lossy_sphere, tol_fact):
    """Left-preconditioned TFQMR (the paper's solver) with and without Zinv, three plane waves."""
    body, E, Z = lossy_sphere["body"], lossy_sphere["E"], lossy_sphere["Z"]
    op = pkg.Operator(body, W.K0, tol_con=1e-6, tol_fact=tol_fact, leaf=64)
    k, p = W.planewave_random(3, seed=4)
    V = op.rhs_planewave(k, p)
    I, iters, rel, st = op.solve_tfqmr(V, rtol=1e-6, max_iter=400)
    assert st == pkg.VIE_OK, (iters, rel)
    Io = solve_dense(Z, rhs_planewave(E, k, p))
    err = np.linalg.norm(I.cpu().numpy() - Io) / np.linalg.norm(Io)
    print("TFQMR chi_fact", tol_fact, "iterations", iters, "true relres", rel, "error vs LU", err)
    assert err < 1e-3, err
    if tol_fact > 0:
        assert iters.max() <= 10      # the preconditioner keeps TFQMR in single digits


def test_tfqmr_reports_nonconvergence_and_nan(lossy_sphere):
    op = pkg.Operator(lossy_sphere["body"], W.K0, tol_con=1e-4, leaf=64)
    k, p = W.planewave_x_along_z()
    V = op.rhs_planewave(k, p)
    I, iters, rel, st = op.solve_tfqmr(V, rtol=1e-12, max_iter=3)
    assert st == pkg.VIE_ENOTCONV and iters[0] == 3
    V[3, 0] = float("nan")
    with pytest.raises(pkg.VieError) as e:
        op.solve_tfqmr(V, rtol=1e-6)
    assert e.value.status == pkg.VIE_ENAN
