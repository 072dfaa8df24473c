"""Multi-RHS apply on the tensor cores (tcgen05, BF16x3) against the single-RHS path and the oracle."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402


@pytest.fixture(scope="module")
def op_pair(lossy_sphere):
    op = pkg.Operator(lossy_sphere["body"], W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64)
    return op, lossy_sphere["Z"]


@pytest.mark.parametrize("nrhs", [16, 37, 128, 130])
@pytest.mark.parametrize("which", [pkg.VIE_OP_Z, pkg.VIE_OP_ZINV])
def test_tensor_core_apply_matches_single_rhs(op_pair, nrhs, which):
    op, Z = op_pair
    X = torch.from_numpy(W.random_block(op.n, nrhs, seed=nrhs)).to(torch.complex64).cuda()
    X = X.t().contiguous().t()
    Y = op.apply(X, op=which)           # nrhs >= 16: tensor-core stages
    op.check()
    ref = torch.stack([op.apply(X[:, j].contiguous(), op=which) for j in range(nrhs)], 1)  # SIMT, one column each
    err = (torch.linalg.norm(Y - ref) / torch.linalg.norm(ref)).item()
    assert err < 2e-5, err
    if which == pkg.VIE_OP_Z:
        d = Z @ X.cpu().numpy()
        assert np.linalg.norm(Y.cpu().numpy() - d) / np.linalg.norm(d) < 5e-4


def test_tensor_core_apply_deterministic(op_pair):
    op, _ = op_pair
    X = torch.from_numpy(W.random_block(op.n, 64, seed=5)).to(torch.complex64).cuda().t().contiguous().t()
    a = op.apply(X).clone()
    b = op.apply(X).clone()
    op.check()
    assert torch.equal(a, b)


@pytest.fixture(scope="module")
def op_mid():
    """Sphere r = 0.8 (N = 27,360): ranks up to ~300, so work items fill 128 output rows and
    run many k-chunks, and each CTA streams several items through its copy ring."""
    return pkg.Operator(W.sphere(0.8, 4.0 - 0.1j, 1.0 / 10), W.K0, tol_con=1e-4, leaf=64)


@pytest.mark.parametrize("nrhs", [48, 128, 200])
def test_tensor_core_apply_mid_size_matches_single_rhs(op_mid, nrhs):
    op = op_mid
    X = torch.from_numpy(W.random_block(op.n, nrhs, seed=100 + nrhs)).to(torch.complex64).cuda()
    X = X.t().contiguous().t()
    Y = op.apply(X)
    op.check()
    cols = [0, 1, nrhs // 2, nrhs - 1]
    ref = torch.stack([op.apply(X[:, j].contiguous()) for j in cols], 1)
    err = (torch.linalg.norm(Y[:, cols] - ref) / torch.linalg.norm(ref)).item()
    assert err < 2e-5, err
