"""End-to-end validation on the GPU: far field vs the oracle, RCS vs Mie, bounded-wait failure path."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402
from oracle.dense import cut_directions, rcs, solve_dense  # noqa: E402
from oracle.entries import rhs_planewave  # noqa: E402
from oracle.mie import rcs_sphere  # noqa: E402


def test_farfield_matches_oracle(lossy_sphere):
    E, Z, body = lossy_sphere["E"], lossy_sphere["Z"], lossy_sphere["body"]
    k, p = W.planewave_x_along_z()
    I = solve_dense(Z, rhs_planewave(E, k, p))
    op = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64)
    dirs = np.concatenate([cut_directions(np.arange(0, 181, 15.0), 0.0), cut_directions(np.arange(0, 181, 15.0), 90.0)])
    g = op.farfield_rcs(torch.from_numpy(I).cuda(), dirs)[:, 0]
    o = rcs(E, I, dirs)[:, 0]
    assert np.abs(g - o).max() < 1e-10 * np.abs(o).max()


def test_sphere_rcs_vs_mie_end_to_end():
    """Config-1 body (r = 0.3, eps_r = 4, pitch 1/20, N = 11,616): GPU build, preconditioned solve, RCS."""
    body = W.sphere_small_fp64()
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-1, leaf=64)
    assert op.n == 11616
    k, p = W.planewave_x_along_z()
    V = op.rhs_planewave(k, p)
    I, it, rel, st = op.solve(V, rtol=1e-6, restart=30, max_iter=300)
    assert st == pkg.VIE_OK and it[0] <= 60
    req = (3 * body.nvox * body.h ** 3 / (4 * np.pi)) ** (1 / 3)
    th = np.arange(0, 181, 2.0)
    for ph in (0.0, 90.0):
        g = op.farfield_rcs(I, cut_directions(th, ph))[:, 0]
        m = rcs_sphere(req, 4.0, np.radians(th), np.radians(ph))
        assert np.sqrt(np.mean((g - m) ** 2)) / m.max() < 0.05      # the paper's relative RMSE


def test_bounded_wait_reports_timeout_and_context_survives():
    lib = pkg.load_library()
    st = lib.vie_wait_selftest(1000, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pkg.VIE_ETIMEOUT
    x = torch.ones(8, device="cuda")
    assert float(x.sum().item()) == 8.0       # the CUDA context is still usable


def test_five_layer_sphere_tfqmr_rcs_vs_multilayer_mie():
    """Layered-sphere geometry of Sec. IV-A at test size (five 0.1-thick layers, eps 2..6 from the
    outside in, pitch 1/20, N = 52,584): chi_con 1e-4, chi_fact 1e-1, left-preconditioned TFQMR to
    chi_sol 1e-3 as in the paper, bistatic RCS against the multilayer Mie series of the
    equal-volume layers."""
    body = W.five_layer_sphere()
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-1, leaf=64)
    assert op.n == 52584
    st_ = op.get_stats()
    k, p = W.planewave_x_along_z()
    V = op.rhs_planewave(k, p)
    I, it, rel, st = op.solve_tfqmr(V, rtol=1e-3, max_iter=200)
    radii = W.equal_volume_layers(body.h, [0.1, 0.2, 0.3, 0.4, 0.5])
    layers = list(zip(radii, [6.0, 5.0, 4.0, 3.0, 2.0]))
    th = np.arange(0, 181, 2.0)
    rmse = []
    for ph in (0.0, 90.0):
        g = op.farfield_rcs(I, cut_directions(th, ph))[:, 0]
        m = rcs_sphere(0.0, 0.0, np.radians(th), np.radians(ph), layers=layers)
        rmse.append(np.sqrt(np.mean((g - m) ** 2)) / m.max())
    print("five-layer sphere: zinv top level", st_.zinv_top_level, "TFQMR iterations", it[0], "relres", rel[0],
          "RCS relative RMSE", rmse)
    assert st == pkg.VIE_OK
    # the paper reports 2 TFQMR iterations at chi_fact 1e-1 for its layered sphere; the inverse
    # built here (sketched IDs of the dense E_tau, complex FP32) needs about 10
    assert st_.zinv_top_level == 0 and it[0] <= 15
    assert max(rmse) < 0.05


def test_two_shell_sphere_tfqmr_rcs_vs_multilayer_mie():
    """Two-shell geometry of Sec. IV-A at test size (vacuum core r = 0.3, shells eps 4 to 0.4 and
    eps 2 to 0.5, pitch 1/20, N = 42,312): chi_fact 1e-1, TFQMR to chi_sol 1e-3, RCS against the
    multilayer Mie series with a vacuum core."""
    body = W.two_shell_sphere()
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-1, leaf=64)
    assert op.n == 42312
    k, p = W.planewave_x_along_z()
    I, it, rel, st = op.solve_tfqmr(op.rhs_planewave(k, p), rtol=1e-3, max_iter=200)
    r0, r1, r2 = W.equal_volume_layers(body.h, [0.3, 0.4, 0.5])
    layers = [(r0, 1.0), (r1, 4.0), (r2, 2.0)]
    th = np.arange(0, 181, 2.0)
    rmse = []
    for ph in (0.0, 90.0):
        g = op.farfield_rcs(I, cut_directions(th, ph))[:, 0]
        m = rcs_sphere(0.0, 0.0, np.radians(th), np.radians(ph), layers=layers)
        rmse.append(np.sqrt(np.mean((g - m) ** 2)) / m.max())
    print("two-shell sphere: zinv top level", op.get_stats().zinv_top_level, "TFQMR iterations", it[0],
          "relres", rel[0], "RCS relative RMSE", rmse)
    assert st == pkg.VIE_OK and it[0] <= 15      # the paper: 7 for its two-shell sphere
    assert max(rmse) < 0.05
