"""vie_apply_noalloc, called through the C ABI, against vie_apply.

The no-allocation entry point serves callers that must not have the library
allocate device memory (a cudaMalloc can stall every stream on the device, and
some processes leave no memory outside their own allocator).  It runs the same
kernels as vie_apply, so its result must equal vie_apply's bit for bit, call
after call, with its work vectors in the library's fixed device array; and a
call must leave the device's free memory unchanged.  This file is collected
last on purpose.
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


def _block(n, nrhs, tdt, seed):
    X = torch.from_numpy(W.random_block(n, nrhs, seed=seed)).to(tdt).cuda()
    return X.t().contiguous().t()


def _out(n, nrhs, tdt, fill=float("nan")):
    return torch.full((nrhs, n), fill, dtype=tdt, device="cuda").t()


@pytest.mark.parametrize("which,tol_fact", [(pkg.VIE_OP_Z, 0.0), (pkg.VIE_OP_ZINV, 1e-2)])
def test_noalloc_matches_apply_twice(which, tol_fact):
    lib = pkg.load_library()
    body = W.sphere(0.25, 4.0 - 0.5j, 1.0 / 14)
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=tol_fact, leaf=64)
    # 1 and 3 columns (SIMT stage kernels), 16 columns (tensor-core stages once vie_apply has
    # packed the tiles): the same kernels run in both calls, so the outputs are identical
    for nrhs, tdt, code in ((1, torch.complex64, pkg.VIE_C64), (3, torch.complex128, pkg.VIE_C128),
                            (16, torch.complex64, pkg.VIE_C64)):
        for call in range(2):  # two calls in a row share (and reuse) the fixed work array
            X = _block(op.n, nrhs, tdt, 100 + call)
            Y_ref = _out(op.n, nrhs, tdt, 0.0)
            Y_na = _out(op.n, nrhs, tdt)
            _call(lib, op, "vie_apply", X, Y_ref, which, nrhs, code)
            _call(lib, op, "vie_apply_noalloc", X, Y_na, which, nrhs, code)
            torch.cuda.synchronize()
            assert torch.equal(Y_na, Y_ref), (nrhs, call)
    op.check()


def test_noalloc_allocates_nothing_on_a_fresh_operator():
    lib = pkg.load_library()
    body = W.sphere(0.25, 4.0 - 0.5j, 1.0 / 14)
    # load the library's kernels and its fixed array on this device with another operator first
    # (the same kernels, at both column counts, so that no lazy kernel load falls inside the check)
    warm = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64)
    for nrhs in (1, 16):
        Xw = _block(warm.n, nrhs, torch.complex64, 7)
        _call(lib, warm, "vie_apply_noalloc", Xw, _out(warm.n, nrhs, torch.complex64), pkg.VIE_OP_Z, nrhs,
              pkg.VIE_C64)
    torch.cuda.synchronize()
    op = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64, seed=5)  # never applied: no work vectors yet
    for nrhs in (1, 16):
        X = _block(op.n, nrhs, torch.complex64, 200 + nrhs)
        Y_na = _out(op.n, nrhs, torch.complex64)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _call(lib, op, "vie_apply_noalloc", X, Y_na, pkg.VIE_OP_Z, nrhs, pkg.VIE_C64)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, (nrhs, free0 - free1)
        Y_ref = _out(op.n, nrhs, torch.complex64, 0.0)
        _call(lib, op, "vie_apply", X, Y_ref, pkg.VIE_OP_Z, nrhs, pkg.VIE_C64)
        torch.cuda.synchronize()
        ref = Y_ref.cpu().numpy()
        err = np.linalg.norm(Y_na.cpu().numpy() - ref) / np.linalg.norm(ref)
        # 16 columns: vie_apply packs the tensor-core tiles and runs BF16x3 products, the
        # no-allocation call before it ran the SIMT kernels (FP32): the multi-RHS tolerance
        assert err <= (1e-6 if nrhs == 1 else 5e-5), (nrhs, err)


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
