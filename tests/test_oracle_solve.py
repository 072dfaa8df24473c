"""Pins of the oracle's solvers: GMRES (textbook finite termination) and the VIE RCS vs Mie."""
import numpy as np

import workloads as W
from oracle.dense import cut_directions, rcs, solve_dense
from oracle.entries import rhs_planewave
from oracle.gmres import gmres
from oracle.mie import rcs_sphere


def test_gmres_terminates_in_k_steps_for_k_eigenvalues():
    rng = np.random.default_rng(0)
    lam = np.repeat([1.0, 2 + 1j, 3.0, -4j, 5.5], 40)
    b = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    x, it, _ = gmres(lambda v: lam * v, b, rtol=1e-12, restart=30)
    assert it == 5 and np.linalg.norm(lam * x - b) < 1e-11 * np.linalg.norm(b)
    A = np.eye(60) + 0.3 * rng.standard_normal((60, 60)) / 8
    Ainv = np.linalg.inv(A)
    x, it, _ = gmres(lambda v: A @ v, b[:60], apply_M=lambda v: Ainv @ v, rtol=1e-12)
    assert it == 1


def test_gmres_matches_dense_lu(lossy_sphere):
    E, Z = lossy_sphere["E"], lossy_sphere["Z"]
    k, p = W.planewave_x_along_z()
    V = rhs_planewave(E, k, p)[:, 0]
    I = solve_dense(Z, V[:, None])[:, 0]
    x, it, _ = gmres(lambda v: Z @ v, V, rtol=1e-10, restart=100, max_iter=2000)
    assert np.linalg.norm(x - I) < 1e-8 * np.linalg.norm(I)


def test_rcs_vs_mie(lossy_sphere):
    """Bistatic RCS of the voxelized sphere against the Mie series of the equal-volume sphere."""
    E, Z, body = lossy_sphere["E"], lossy_sphere["Z"], lossy_sphere["body"]
    k, p = W.planewave_x_along_z()
    I = solve_dense(Z, rhs_planewave(E, k, p))
    req = (3 * body.nvox * body.h ** 3 / (4 * np.pi)) ** (1 / 3)
    th = np.arange(0, 181, 2.0)
    for ph in (0.0, 90.0):
        s = rcs(E, I, cut_directions(th, ph))[:, 0]
        m = rcs_sphere(req, complex(body.eps[0]), np.radians(th), np.radians(ph))
        rmse = np.sqrt(np.mean((s - m) ** 2)) / m.max()   # the paper's relative RMSE (linear RCS)
        assert rmse < 0.05
        # a sphere of ~3 voxels per radius is coarsely staircased: loose dB bound near the peak
        sel = m > m.max() / 10
        assert np.abs(10 * np.log10(s[sel] / m[sel])).max() < 2.0
