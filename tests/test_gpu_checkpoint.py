"""vie_save / vie_load: a built operator (Z, and Zinv with product-built levels) read back from
its file applies bit-identically, and foreign or truncated files are refused."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402


def test_save_load_roundtrip_bit_identical(tmp_path):
    body = W.sphere(0.25, 4.0 - 0.5j, 1.0 / 14)
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64, inv_dense_max=256)
    op.autotune()  # the tuned single-RHS kernels and tiles travel with the file
    path = str(tmp_path / "op.vie")
    op.save(path)
    back = pkg.Operator.load(path)
    assert back.n == op.n
    assert back.get_stats().entries_zinv == op.get_stats().entries_zinv
    for nrhs in (1, 16):
        X = torch.from_numpy(W.random_block(op.n, nrhs, seed=nrhs)).to(torch.complex64).cuda()
        for which in (pkg.VIE_OP_Z, pkg.VIE_OP_ZINV):
            a = op.apply(X, op=which)
            b = back.apply(X, op=which)
            torch.cuda.synchronize()
            assert torch.equal(a, b), (nrhs, which)
    np.testing.assert_array_equal(back.tree_perm(), op.tree_perm())


def test_load_refuses_bad_files(tmp_path):
    lib = pkg.load_library()
    with pytest.raises(pkg.VieError) as e:
        pkg.Operator.load(str(tmp_path / "missing.vie"))
    assert e.value.status == pkg.VIE_EINVAL
    junk = tmp_path / "junk.vie"
    junk.write_bytes(b"not an operator file at all")
    with pytest.raises(pkg.VieError) as e:
        pkg.Operator.load(str(junk))
    assert e.value.status == pkg.VIE_EINVAL
    op = pkg.Operator(W.sphere(0.15, 4.0, 1.0 / 16), W.K0, tol_con=1e-4, leaf=32)
    full = tmp_path / "op.vie"
    op.save(str(full))
    cut = tmp_path / "cut.vie"
    cut.write_bytes(full.read_bytes()[: os.path.getsize(full) // 2])
    with pytest.raises(pkg.VieError) as e:
        pkg.Operator.load(str(cut))
    assert e.value.status == pkg.VIE_EINVAL
    assert lib is not None
