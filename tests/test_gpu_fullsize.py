"""Full-size parity: the benchmark workload (sphere r = 2, N = 410,208) in the benchmark's launch
configuration, checked on sampled output rows that the oracle computes one by one (Eq. 5 rows)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402
from oracle.entries import Elements, zblock  # noqa: E402
from oracle.mesh import build_mesh  # noqa: E402


@pytest.fixture(scope="module")
def full():
    body = W.sphere_large_c32()
    op = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64, factor_dtype="c64", seed=1)
    op.autotune()
    mesh = build_mesh(body)
    return body, op, mesh


def test_sampled_rows_of_the_full_size_apply(full):
    body, op, mesh = full
    n = op.n
    assert n == 410208 == len(mesh["faces"])
    x = W.random_block(n, 1, seed=77)[:, 0]
    y = op.apply(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    E = Elements(mesh, W.K0)
    rows = np.random.default_rng(5).choice(n, size=6, replace=False)
    exact = np.array([(zblock(E, [r], np.arange(n), chunk=2) @ x)[0] for r in rows])
    err = np.linalg.norm(y[rows] - exact) / np.linalg.norm(exact)
    assert err < 5e-4, (err, rows)


def test_full_size_apply_is_finite_and_linear(full):
    _, op, _ = full
    x1 = torch.from_numpy(W.random_block(op.n, 1, seed=1)[:, 0].astype(np.complex64)).cuda()
    x2 = torch.from_numpy(W.random_block(op.n, 1, seed=2)[:, 0].astype(np.complex64)).cuda()
    a = op.apply(x1).clone()
    b = op.apply(x2).clone()
    c = op.apply((x1 + 2.0 * x2).contiguous())
    assert torch.isfinite(c).all()
    assert (torch.linalg.norm(c - (a + 2.0 * b)) / torch.linalg.norm(c)).item() < 1e-5
