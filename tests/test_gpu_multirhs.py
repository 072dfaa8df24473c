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


def test_precision_selector():
    """vie_config.prec: FP64 stores complex FP64 factors, C32 never takes the tensor cores (its
    16-column apply equals 16 single-column applies), BF16x3 and TF32 take them from 16 columns,
    TF32 at its coarser rounding."""
    body = W.sphere(0.2, 4.0 - 1.0j, 1.0 / 16)
    X = torch.from_numpy(W.random_block(1824, 16, seed=9)).to(torch.complex64).cuda().t().contiguous().t()
    c32 = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64, prec=pkg.VIE_P_C32)
    assert c32.autotune_rhs() >= 1 << 30
    Y = c32.apply(X)
    cols = torch.stack([c32.apply(X[:, j].contiguous()) for j in range(16)], 1)
    assert (torch.linalg.norm(Y - cols) / torch.linalg.norm(cols)).item() < 1e-6
    tc = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64, prec=pkg.VIE_P_TC_BF16X3)
    assert tc.autotune_rhs() == 16
    err = (torch.linalg.norm(tc.apply(X) - cols) / torch.linalg.norm(cols)).item()
    assert 0 < err < 5e-5  # BF16x3 split products: close to, not equal to, the FP32 result
    f64 = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64, prec=pkg.VIE_P_FP64)
    assert f64.get_stats().bytes_z > 1.8 * tc.get_stats().bytes_z  # complex FP64 factors
    # TF32: one product per real product on operands rounded to TF32 (unit roundoff
    # u = 2^-11); each product carries at most 2u relative error and the apply chains about
    # ten stages, so the apply stays within about 6u = 3e-3 of the FP32 result, and is
    # coarser than the BF16x3 split
    tf = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64, prec=pkg.VIE_P_TC_TF32)
    assert tf.autotune_rhs() == 16
    Yt = tf.apply(X)
    tf.check()
    err_tf = (torch.linalg.norm(Yt - cols) / torch.linalg.norm(cols)).item()
    print("precision selector: BF16x3 vs FP32", err, "TF32 vs FP32", err_tf)
    assert err < err_tf < 3e-3
    # below the tensor-core column count TF32 runs the FP32 SIMT path
    y3 = tf.apply(X[:, 3].contiguous())
    assert (torch.linalg.norm(y3 - cols[:, 3]) / torch.linalg.norm(cols[:, 3])).item() < 1e-6
    # a grouped apply of the two tensor-core variants at once: one launch per variant and depth
    g = pkg.apply_group([(tc, X, pkg.VIE_OP_Z), (tf, X, pkg.VIE_OP_Z)])
    assert torch.equal(g[0], tc.apply(X)) and torch.equal(g[1], Yt)
