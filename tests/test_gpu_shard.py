"""The sharded apply on one GPU: every rank's rows, written one rank after another (no rank
waits on another), assemble to the unsharded apply of Z and of Zinv."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("nranks", [2, 4])
def test_ranks_assemble_the_full_apply(nranks):
    body = W.sphere(0.25, 4.0 - 0.5j, 1.0 / 14)
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64)
    perm = op.tree_perm()
    for nrhs in (1, 3, 20):
        X = torch.from_numpy(W.random_block(op.n, nrhs, seed=nrhs)).to(torch.complex64).cuda()
        X = X.t().contiguous().t()
        for which in (pkg.VIE_OP_Z, pkg.VIE_OP_ZINV):
            ref = op.apply(X, op=which)
            Y = torch.full_like(ref, float("nan"))
            covered = 0
            for r in range(nranks):
                lo, hi = op.shard_range(r, nranks)
                covered += hi - lo
                op.apply_shard(X, Y, r, nranks, op=which)
            torch.cuda.synchronize()
            assert covered == op.n
            assert torch.isfinite(Y).all()
            if nrhs < 16:
                assert torch.equal(Y, ref), (nranks, nrhs, which)
            else:
                err = (torch.linalg.norm(Y - ref) / torch.linalg.norm(ref)).item()
                assert err < 1e-6, (nranks, nrhs, which, err)
    assert len(perm) == op.n
    op.check()
