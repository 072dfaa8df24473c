"""The synthetic workloads against their stated recipes (inputs only; no method arithmetic):
unknown counts of the benchmark bodies from the mesh rule, the Drude permittivity of the plasma
shell, and the statistics of the Gaussian-random-field cube (seeded, reproducible)."""
import numpy as np
import pytest

import workloads as W


def _swg_count(body):
    """N = 12 V + S for the Kuhn split of a voxel body (V voxels, S exposed voxel faces): each
    voxel has 6 faces inside it and 12 triangles on its sides; a side shared with a neighbour
    holds 2 faces for the pair, an exposed side 2 faces of its own."""
    ijk = np.asarray(body.ijk, dtype=np.int64)
    lo = ijk.min(0) - 1
    dims = ijk.max(0) - lo + 2
    occ = np.zeros(dims, dtype=bool)
    occ[tuple((ijk - lo).T)] = True
    exposed = 0
    for ax in range(3):
        a = np.moveaxis(occ, ax, 0)
        exposed += np.count_nonzero(a[1:] & ~a[:-1]) + np.count_nonzero(a[:-1] & ~a[1:])
    return 12 * len(ijk) + exposed


@pytest.mark.parametrize("make,n_expect", [
    (lambda: W.sphere_small_fp64(), 11_616),       # config 1: r = 0.3, pitch lambda_d/10 = 1/20
    (lambda: W.sphere_large_c32(), 410_208),        # config 2: r = 2, pitch 1/10
    (lambda: W.plasma_shell(), 690_768),            # config 3: shell 1.5 / 1.2, pitch 1/20
    (lambda: W.cube_grf(5.0, 0.1), 1_515_000),      # config 4: 5 lambda0 cube, pitch 1/10
])
def test_benchmark_bodies_have_the_stated_unknown_counts(make, n_expect):
    body = make()
    assert len(np.unique(np.asarray(body.ijk), axis=0)) == len(body.ijk)
    assert _swg_count(body) == n_expect


def test_drude_permittivity():
    """1 - wp^2 / (w (w - j nu)) with wp / w = 1.8, nu / w = 0.05 (exp(+j w t): Im eps < 0)."""
    e = W.drude_eps()
    assert abs(e - (-2.2319 - 0.1616j)) < 1e-4
    assert np.allclose(W.plasma_shell().eps, e)


def test_grf_cube_statistics():
    """eps_r = 1 + 49 u, u = Phi(z), z a standardized field with covariance exp(-d^2 / (2 l^2)),
    l = 0.5 lambda0 (5 voxels): u is uniform, z is standard normal and correlates as exp(-1/2)
    at a lag of l; the same seed gives the same medium."""
    from scipy.special import ndtri
    from scipy.stats import kstest

    body = W.cube_grf(5.0, 0.1)
    eps = np.asarray(body.eps)
    assert np.all(eps.imag == 0) and eps.real.min() >= 1.0 and eps.real.max() <= 50.0
    u = (eps.real - 1.0) / 49.0
    assert kstest(u, "uniform").statistic < 0.05
    z = ndtri(np.clip(u, 1e-15, 1 - 1e-15)).reshape(50, 50, 50)
    assert abs(z.mean()) < 1e-6 and abs(z.std() - 1.0) < 1e-6
    for ax in range(3):
        a = np.moveaxis(z, ax, 0)
        rho = np.mean(a[5:] * a[:-5])
        assert abs(rho - np.exp(-0.5)) < 0.1, (ax, rho)
    assert np.array_equal(W.cube_grf(5.0, 0.1).eps, eps)
