"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402
from oracle.entries import Elements, rhs_planewave, zblock  # noqa: E402
from oracle.hodbf import cluster_tree, face_centroids  # noqa: E402
from oracle.mesh import build_mesh  # noqa: E402


def _mixed_block():
    b = W.tiny_block(3, 2, 2, h=0.06)
    rng = np.random.default_rng(4)
    eps = rng.choice([1.0, 2.5, 4.0 - 0.3j, -2.0 - 0.2j, 9.0], size=b.nvox).astype(np.complex128)
    return W.VoxelBody("mixed", b.h, b.ijk, eps)


BODIES = {
    "mixed_block": _mixed_block,
    "sphere_lossy": lambda: W.sphere(0.2, 4.0 - 1.0j, 1.0 / 16),
    "shell_plasma": lambda: W.shell(0.25, 0.15, W.drude_eps(), 1.0 / 20),
}


@pytest.fixture(scope="module", params=list(BODIES))
def case(request):
    body = BODIES[request.param]()
    mesh = build_mesh(body)
    E = Elements(mesh, W.K0)
    n = len(mesh["faces"])
    Z = zblock(E, np.arange(n), np.arange(n))
    return dict(name=request.param, body=body, mesh=mesh, E=E, Z=Z, n=n)


def test_mesh_and_tree_bit_exact(case):
    op = pkg.Operator(case["body"], W.K0, tol_con=1e-4, leaf=64)
    f, tp, tm = op.faces()
    m = case["mesh"]
    assert op.n == case["n"]
    assert np.array_equal(f, m["faces"]) and np.array_equal(tp, m["face_tp"]) and np.array_equal(tm, m["face_tm"])
    perm, LH, _ = cluster_tree(face_centroids(m), 64)
    assert op.stats.levels == LH
    assert np.array_equal(op.tree_perm(), perm)


def test_entries_fp64(case):
    op = pkg.Operator(case["body"], W.K0, tol_con=1e-4, leaf=64)
    n = case["n"]
    r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rows = torch.from_numpy(r.ravel().astype(np.int32)).cuda()
    cols = torch.from_numpy(c.ravel().astype(np.int32)).cuda()
    z = op.entries(rows, cols).cpu().numpy().reshape(n, n)
    Z = case["Z"]
    err = np.abs(z - Z).max() / np.abs(Z).max()
    assert err < 1e-10, err


def test_rhs_fp64(case):
    op = pkg.Operator(case["body"], W.K0, tol_con=1e-4, leaf=64)
    k, p = W.planewave_grid(2, 3)
    V = op.rhs_planewave(k, p).cpu().numpy()
    Vo = rhs_planewave(case["E"], k, p)
    assert np.abs(V - Vo).max() < 1e-12 * np.abs(Vo).max()


@pytest.mark.parametrize("tol,fdt,bound", [(1e-4, "c64", 5e-4), (1e-3, "c64", 5e-3), (1e-6, "c128", 1e-5)])
def test_hodbf_apply_vs_dense(case, tol, fdt, bound):
    op = pkg.Operator(case["body"], W.K0, tol_con=tol, leaf=64, factor_dtype=fdt)
    Z = case["Z"]
    for nrhs in (1, 3, 11):
        X = W.random_block(case["n"], nrhs, seed=nrhs)
        ref = Z @ X
        for vdt in (torch.complex64, torch.complex128):
            Y = op.apply(torch.from_numpy(X).to(vdt).cuda()).cpu().numpy()
            err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
            lim = max(bound, 2e-6) if vdt == torch.complex64 else bound
            assert err < lim, (nrhs, vdt, err)


def test_apply_is_deterministic(case):
    op = pkg.Operator(case["body"], W.K0, tol_con=1e-4, leaf=32)
    X = torch.from_numpy(W.random_block(case["n"], 2, seed=9)).to(torch.complex64).cuda()
    a = op.apply(X).clone()
    b = op.apply(X).clone()
    assert torch.equal(a, b)


def test_autotune_keeps_results(case):
    op = pkg.Operator(case["body"], W.K0, tol_con=1e-4, leaf=32)
    X = torch.from_numpy(W.random_block(case["n"], 1, seed=19)[:, 0]).to(torch.complex64).cuda()
    before = op.apply(X).clone()
    choice = op.autotune()
    assert len(choice) == op.get_stats().apply_stages_z and np.all((choice >= 0) & (choice < 21))
    after = op.apply(X)
    assert (torch.linalg.norm(after - before) / torch.linalg.norm(before)).item() < 1e-6



@pytest.mark.parametrize("cand", [0, 4, 8, 9, 10, 11, 12, 16, 20])
def test_every_kernel_candidate_matches_dense(case, cand):
    """Each single-RHS candidate (streaming kernel with four loads in flight, variants 0, 4, 8;
    shared-memory bulk-staged kernel 9-11; streaming kernel with eight loads in flight 12, 16, 20)
    set on every stage gives the same apply."""
    op = pkg.Operator(case["body"], W.K0, tol_con=1e-4, leaf=32)
    X = torch.from_numpy(W.random_block(case["n"], 1, seed=23)[:, 0]).to(torch.complex64).cuda()
    ref = op.apply(X).clone()
    op.set_tiling([cand] * op.get_stats().apply_stages_z)
    got = op.apply(X)
    op.check()
    assert (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item() < 1e-6
    d = case["Z"] @ X.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got.cpu().numpy() - d) / np.linalg.norm(d) < 5e-4
