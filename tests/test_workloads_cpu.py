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


def test_plane_wave_sets():
    """Config 3's 8 x 16 (theta, phi) grid with theta-hat and phi-hat polarizations (256 waves)
    and the serving requests' random waves: unit directions, unit polarizations orthogonal to them."""
    k, p = W.planewave_grid()
    assert k.shape == p.shape == (256, 3)
    assert np.allclose(np.linalg.norm(k, axis=1), 1) and np.allclose(np.linalg.norm(p, axis=1), 1)
    assert np.allclose((k * p).sum(1), 0, atol=1e-15)
    assert np.allclose((p[:128] * p[128:]).sum(1), 0, atol=1e-15)  # theta-hat, phi-hat per direction
    assert np.allclose(np.cross(p[:128], p[128:]), k[:128])       # (theta-hat, phi-hat, khat) right-handed
    assert len(np.unique(np.round(k[:128], 12), axis=0)) == 128
    th = np.arccos(np.clip(k[:128, 2], -1, 1))
    assert np.allclose(np.unique(np.round(th, 12)), (np.arange(8) + 0.5) * np.pi / 8)
    k, p = W.planewave_random(2000, seed=3)
    assert np.allclose(np.linalg.norm(k, axis=1), 1) and np.allclose(np.linalg.norm(p, axis=1), 1)
    assert np.abs((k * p).sum(1)).max() < 1e-14
    assert np.abs(k.mean(0)).max() < 0.06  # uniform on the sphere: mean direction ~ 0 (3 sigma ~ 0.04)
    k2, p2 = W.planewave_random(2000, seed=3)
    assert np.array_equal(k, k2) and np.array_equal(p, p2)


def test_layered_bodies_and_equal_volume_radii():
    """Layered spheres assign each voxel the permittivity of the layer holding its centre; the
    equal-volume radius of a staircase layer holds exactly the volume of its voxels."""
    body = W.five_layer_sphere()
    c = (body.ijk.astype(np.float64) + 0.5) * body.h
    r = np.linalg.norm(c, axis=1)
    radii, values = [0.5, 0.4, 0.3, 0.2, 0.1], [2.0, 3.0, 4.0, 5.0, 6.0]
    for i, e in enumerate(values):
        lo = radii[i + 1] if i + 1 < len(radii) else 0.0
        sel = (r < radii[i]) & (r >= lo)
        assert sel.any() and np.all(body.eps[sel] == e)
    h = 1.0 / 20
    for R, Req in zip(radii, W.equal_volume_layers(h, radii)):
        cnt = np.count_nonzero(r < R)
        assert abs(4.0 / 3.0 * np.pi * Req ** 3 - cnt * h ** 3) < 1e-12
        assert abs(Req - R) < h
