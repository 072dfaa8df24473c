"""vie_apply_noalloc, called through the C ABI, against vie_apply.

The no-allocation entry point serves callers that must not have the library
allocate device memory (a cudaMalloc can stall every stream on the device, and
some processes leave no memory outside their own allocator).  It must give the
same result as vie_apply, call after call, with its work vectors in the
library's fixed device array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402


def _call(lib, op, fn, X, Y, which, nrhs, dtype):
    st = getattr(lib, fn)(op._h, which, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), nrhs,
                          op.n, op.n, dtype, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pkg.VIE_OK, lib.vie_last_error().decode()


@pytest.mark.parametrize("which,tol_fact", [(pkg.VIE_OP_Z, 0.0), (pkg.VIE_OP_ZINV, 1e-2)])
def test_noalloc_matches_apply_twice(which, tol_fact):
    lib = pkg.load_library()
    body = W.sphere(0.25, 4.0 - 0.5j, 1.0 / 14)
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=tol_fact, leaf=64)
    for nrhs, tdt, code in ((1, torch.complex64, pkg.VIE_C64), (3, torch.complex128, pkg.VIE_C128)):
        for call in range(2):  # two calls in a row share (and reuse) the fixed work array
            X = torch.from_numpy(W.random_block(op.n, nrhs, seed=100 + call)).to(tdt).cuda()
            X = X.t().contiguous().t()
            Y_ref = torch.empty((nrhs, op.n), dtype=tdt, device="cuda").t()
            Y_na = torch.full((nrhs, op.n), float("nan"), dtype=tdt, device="cuda").t()
            _call(lib, op, "vie_apply", X, Y_ref, which, nrhs, code)
            _call(lib, op, "vie_apply_noalloc", X, Y_na, which, nrhs, code)
            torch.cuda.synchronize()
            ref = Y_ref.cpu().numpy()
            err = np.linalg.norm(Y_na.cpu().numpy() - ref) / np.linalg.norm(ref)
            assert err <= 1e-6, (nrhs, call, err)


def test_noalloc_rejects_oversized_work():
    lib = pkg.load_library()
    body = W.sphere(0.25, 4.0 - 0.5j, 1.0 / 14)
    op = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64)
    nrhs = 4096  # 2 N nrhs complex128 elements alone exceed the fixed array
    X = torch.zeros((nrhs, op.n), dtype=torch.complex128, device="cuda").t()
    Y = torch.zeros_like(X)
    st = lib.vie_apply_noalloc(op._h, pkg.VIE_OP_Z, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                               nrhs, op.n, op.n, pkg.VIE_C128, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pkg.VIE_EINVAL
    assert "fixed scratch" in lib.vie_last_error().decode()
