"""The Python binding's argument marshalling on the host (no GPU): column-major layout and
leading dimensions handed to the C ABI, dtype codes, and the cluster-tree node offsets the
sharded path derives from N alone."""
import numpy as np
import pytest

import paper_2111_01730_gb300 as pkg

torch = pytest.importorskip("torch")


def test_vectors_reach_the_abi_column_major():
    n = 7
    v = torch.arange(n, dtype=torch.float32).to(torch.complex64)
    t, nrhs, ld = pkg._colmajor(v, n)
    assert (nrhs, ld) == (1, n) and t.stride(0) == 1 and torch.equal(t[:, 0], v)
    rowmajor = torch.arange(3 * n, dtype=torch.float64).to(torch.complex128).reshape(n, 3)
    t, nrhs, ld = pkg._colmajor(rowmajor, n)
    assert (nrhs, ld) == (3, n) and t.stride() == (1, n) and torch.equal(t, rowmajor)
    colmajor = rowmajor.t().contiguous().t()
    t, nrhs, ld = pkg._colmajor(colmajor, n)
    assert t.data_ptr() == colmajor.data_ptr() and (nrhs, ld) == (3, n)
    # a block of a taller column-major array keeps its leading dimension (ld >= N in the ABI)
    tall = torch.zeros((4, n + 5), dtype=torch.complex64).t()
    t, nrhs, ld = pkg._colmajor(tall[:n], n)
    assert t.data_ptr() == tall.data_ptr() and (nrhs, ld) == (4, n + 5)


def test_dtype_codes():
    assert pkg._dtype_code(torch.zeros(1, dtype=torch.complex64)) == pkg.VIE_C64
    assert pkg._dtype_code(torch.zeros(1, dtype=torch.complex128)) == pkg.VIE_C128
    with pytest.raises(TypeError):
        pkg._dtype_code(torch.zeros(1, dtype=torch.float32))


def test_tree_bounds_follow_the_kd_split():
    """The first child of a node with n faces holds ceil(n/2) (the KD bisection)."""
    assert pkg.tree_bounds(10, 2) == [[0, 10], [0, 5, 10], [0, 3, 5, 8, 10]]
    b = pkg.tree_bounds(1824, 5)
    for lev in range(1, 6):
        assert b[lev][0] == 0 and b[lev][-1] == 1824 and len(b[lev]) == 2 ** lev + 1
        sizes = np.diff(b[lev])
        assert sizes.max() - sizes.min() <= 1
