"""Grouped applies (vie_apply_group): several operators, each with its own columns, in one
launch per stage depth.  The results are bit-identical to the per-operator applies on the
same kernels' arithmetic: SIMT columns (1 and 5 columns), tensor-core columns (20), Z and
Zinv, and more operators than one launch's segment table holds."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402


def _x(n, nrhs, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn(n, nrhs, 2, generator=g, dtype=torch.float32)
    return torch.view_as_complex(x.contiguous()).cuda().t().contiguous().t()


@pytest.fixture(scope="module")
def three():
    a = pkg.Operator(W.sphere(0.3, 4.0 - 0.1j, 1.0 / 20), W.K0, tol_con=1e-4, tol_fact=1e-1, leaf=64)
    b = pkg.Operator(W.shell(0.22, 0.12, W.drude_eps(), 1.0 / 20), W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64)
    c = pkg.Operator(W.sphere(0.2, 10.0, 1.0 / 30), W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64)
    return a, b, c


def test_group_bit_identical_to_separate_applies(three):
    a, b, c = three
    jobs = [(a, _x(a.n, 1, 1)[:, 0], pkg.VIE_OP_Z), (b, _x(b.n, 5, 2), pkg.VIE_OP_ZINV),
            (c, _x(c.n, 20, 3), pkg.VIE_OP_Z)]
    got = pkg.apply_group(jobs)
    for (op, X, kind), Y in zip(jobs, got):
        ref = op.apply(X, op=kind)
        torch.cuda.synchronize()
        assert torch.equal(Y, ref), (op.n, kind, X.shape)
    # every kind on every operator, tensor-core columns on two of them at once
    jobs = [(a, _x(a.n, 24, 4), pkg.VIE_OP_ZINV), (b, _x(b.n, 17, 5), pkg.VIE_OP_Z),
            (c, _x(c.n, 3, 6), pkg.VIE_OP_ZINV)]
    got = pkg.apply_group(jobs)
    for (op, X, kind), Y in zip(jobs, got):
        assert torch.equal(Y, op.apply(X, op=kind)), (op.n, kind, X.shape)
    for op in three:
        op.check()


def test_group_beyond_one_segment_table():
    """18 small operators (more than the 16 segments of one launch): every result still equals
    its own apply."""
    ops = [pkg.Operator(W.sphere(0.1 + 0.005 * i, 4.0, 1.0 / 20), W.K0, tol_con=1e-4, tol_fact=0, leaf=32)
           for i in range(18)]
    jobs = [(op, _x(op.n, 1 + (i % 4), 10 + i), pkg.VIE_OP_Z) for i, op in enumerate(ops)]
    got = pkg.apply_group(jobs)
    for (op, X, kind), Y in zip(jobs, got):
        assert torch.equal(Y, op.apply(X, op=kind))


def test_group_rejects_bad_jobs(three):
    a, b, c = three
    X = _x(a.n, 2, 7)
    with pytest.raises(pkg.VieError) as e:
        pkg.apply_group([(a, X, pkg.VIE_OP_Z), (a, X, pkg.VIE_OP_ZINV)])
    assert e.value.status == pkg.VIE_EINVAL
    d = pkg.Operator(W.sphere(0.1, 4.0, 1.0 / 20), W.K0, tol_con=1e-4, tol_fact=0, leaf=32, factor_dtype="c128")
    with pytest.raises(pkg.VieError) as e:
        pkg.apply_group([(d, _x(d.n, 1, 8), pkg.VIE_OP_Z)])
    assert e.value.status == pkg.VIE_EINVAL
    e0 = pkg.Operator(W.sphere(0.1, 4.0, 1.0 / 20), W.K0, tol_con=1e-4, tol_fact=0, leaf=32)
    with pytest.raises(pkg.VieError) as e:
        pkg.apply_group([(e0, _x(e0.n, 1, 9), pkg.VIE_OP_ZINV)])
    assert e.value.status == pkg.VIE_ENOTSUP
    assert pkg.apply_group([]) == []
