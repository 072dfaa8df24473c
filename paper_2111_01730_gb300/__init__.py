"""GB300 butterfly-accelerated VIE: Python binding of the C ABI in include/vie.h.

Argument marshalling only: every step of the build, the apply and the solve
runs in libvie.so (CUDA, sm_103a).  PyTorch provides device memory and streams.
There is no CPU fallback: loading fails loudly when the library is missing.

Vectors are complex CUDA tensors of shape (N,) or (N, nrhs) in column-major
layout (``t.stride(0) == 1``), indexed by the faces of the mesh in the
library's face order (see ``Operator.faces``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvie.so")

VIE_OK, VIE_EINVAL, VIE_ENOMEM, VIE_ENOTCONV, VIE_ETIMEOUT, VIE_ENAN, VIE_ECUDA, VIE_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
VIE_OP_Z, VIE_OP_ZINV, VIE_OP_ZH, VIE_OP_ZINVH = 0, 1, 2, 3
VIE_C64, VIE_C128 = 0, 1
VIE_P_AUTO, VIE_P_FP64, VIE_P_C32, VIE_P_TC_BF16X3, VIE_P_TC_TF32 = 0, 1, 2, 3, 4

# every symbol declared in include/vie.h
EXPORTS = ["vie_build", "vie_apply", "vie_apply_noalloc", "vie_apply_profile", "vie_program_info", "vie_program_blocks", "vie_autotune", "vie_autotune_rhs", "vie_set_tiling", "vie_entries", "vie_rhs_planewave", "vie_solve", "vie_solve_tfqmr", "vie_farfield",
           "vie_mesh_faces", "vie_mesh_host", "vie_tree_perm", "vie_stats", "vie_check", "vie_wait_selftest", "vie_destroy", "vie_last_error",
           "vie_server_create", "vie_server_submit", "vie_server_step", "vie_server_result", "vie_server_destroy",
           "vie_save", "vie_load", "vie_shard_range", "vie_apply_shard", "vie_apply_group", "vie_build_mesh",
           "vie_mesh_host_tets", "vie_set_prec", "vie_server_cancel", "vie_server_memory"]


class VieError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"vie status {status}: {msg}")
        self.status = status


class _Voxels(ctypes.Structure):
    _fields_ = [("nvox", ctypes.c_int64), ("ijk", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("h", ctypes.c_double)]


class _Mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("nt", ctypes.c_int64), ("tet", ctypes.c_void_p),
                ("eps_r", ctypes.c_void_p)]


def _tetmesh(mesh):
    """vie_mesh of a workloads.TetMesh-like object (verts, tets, eps); returns (struct, arrays kept alive)."""
    xyz = np.ascontiguousarray(mesh.verts, dtype=np.float64)
    tet = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    eps = np.ascontiguousarray(np.stack([np.real(mesh.eps), np.imag(mesh.eps)], 1), dtype=np.float64)
    return _Mesh(len(xyz), xyz.ctypes.data, len(tet), tet.ctypes.data, eps.ctypes.data), (xyz, tet, eps)


class _Config(ctypes.Structure):
    _fields_ = [("tol_con", ctypes.c_double), ("tol_fact", ctypes.c_double), ("leaf", ctypes.c_int32),
                ("factor_dtype", ctypes.c_int32), ("seed", ctypes.c_uint64), ("oversample", ctypes.c_int32),
                ("id_tol_div", ctypes.c_int32), ("inv_dense_max", ctypes.c_int32), ("prec", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ntets", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("max_rank", ctypes.c_int32), ("entries_z", ctypes.c_int64), ("entries_zinv", ctypes.c_int64),
                ("bytes_z", ctypes.c_int64), ("bytes_zinv", ctypes.c_int64), ("entries_evaluated", ctypes.c_int64),
                ("build_seconds", ctypes.c_double), ("invert_seconds", ctypes.c_double),
                ("apply_stages_z", ctypes.c_int32), ("apply_stages_zinv", ctypes.c_int32),
                ("build_entries_seconds", ctypes.c_double), ("build_id_seconds", ctypes.c_double),
                ("build_host_seconds", ctypes.c_double), ("zinv_top_level", ctypes.c_int32),
                ("zinv_product_levels", ctypes.c_int32), ("inverse_products", ctypes.c_int64),
                ("invert_product_seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libvie.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libvie.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "vie_build": [P, D, P, P, P],
        "vie_apply": [P, I32, P, P, I64, I64, I64, I32, P],
        "vie_apply_noalloc": [P, I32, P, P, I64, I64, I64, I32, P],
        "vie_entries": [P, P, P, I64, P, P],
        "vie_apply_profile": [P, I32, P, P, I64, I64, I64, I32, P, P, P, I32],
        "vie_program_info": [P, I32, P, P, P, I32, P],
        "vie_program_blocks": [P, I32, I32, P, P, I64, P],
        "vie_autotune": [P, I32, P, I32, P],
        "vie_rhs_planewave": [P, P, P, I64, P, P],
        "vie_solve": [P, P, P, I64, D, I32, I32, P, P, P],
        "vie_solve_tfqmr": [P, P, P, I64, D, I32, P, P, P],
        "vie_set_tiling": [P, I32, P, I32, P],
        "vie_autotune_rhs": [P, I32, P, P],
        "vie_farfield": [P, P, I64, P, I64, P, P],
        "vie_mesh_faces": [P, P, P, P],
        "vie_mesh_host": [P, I32, P, P, P, P, P, P],
        "vie_tree_perm": [P, P],
        "vie_stats": [P, P],
        "vie_check": [P, P],
        "vie_wait_selftest": [I32, P],
        "vie_server_create": [P, I32, I32, I32, I64, P, P],
        "vie_server_submit": [P, I32, P, I64, D, P],
        "vie_server_step": [P, P, P],
        "vie_server_result": [P, I64, P, P, P, P],
        "vie_save": [P, ctypes.c_char_p, P],
        "vie_shard_range": [P, I32, I32, P, P],
        "vie_apply_shard": [P, I32, I32, I32, P, P, I64, I64, I64, I32, P],
        "vie_load": [ctypes.c_char_p, P, P],
        "vie_apply_group": [P, P, P, P, P, I32, P],
        "vie_build_mesh": [P, D, P, P, P],
        "vie_mesh_host_tets": [P, I32, P, P, P, P, P, P, P, P],
        "vie_set_prec": [P, I32],
        "vie_server_cancel": [P, I64],
        "vie_server_memory": [P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.vie_server_destroy.argtypes = [P]
    lib.vie_server_destroy.restype = None
    lib.vie_destroy.argtypes = [P]
    lib.vie_destroy.restype = None
    lib.vie_last_error.argtypes = []
    lib.vie_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != VIE_OK:
        raise VieError(status, _lib.vie_last_error().decode())


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor(t, n):
    """(N,) or (N, nrhs) complex tensor -> (tensor, nrhs, ld) with stride(0) == 1."""
    if t.dim() == 1:
        t = t.reshape(n, 1)
    nrhs = t.shape[1]
    if t.stride(0) != 1 or (nrhs > 1 and t.stride(1) < n):
        t = t.t().contiguous().t()
    return t, nrhs, (t.stride(1) if nrhs > 1 else n)


def _dtype_code(t):
    import torch

    if t.dtype == torch.complex64:
        return VIE_C64
    if t.dtype == torch.complex128:
        return VIE_C128
    raise TypeError(f"complex64 or complex128 tensor expected, got {t.dtype}")


def _voxels(body):
    ijk = np.ascontiguousarray(body.ijk, dtype=np.int32)
    eps = np.ascontiguousarray(np.stack([np.real(body.eps), np.imag(body.eps)], 1), dtype=np.float64)
    return _Voxels(len(ijk), ijk.ctypes.data, eps.ctypes.data, float(body.h)), (ijk, eps)


def mesh_host(body, leaf: int = 64):
    """Mesh face table and cluster-tree permutation made by the library on the host (no GPU)."""
    lib = load_library()
    vox, keep = _voxels(body)
    n = ctypes.c_int64(0)
    _check(lib.vie_mesh_host(ctypes.byref(vox), leaf, ctypes.byref(n), None, None, None, None, None))
    N = n.value
    f = np.zeros((N, 3), dtype=np.int32)
    tp = np.zeros(N, dtype=np.int32)
    tm = np.zeros(N, dtype=np.int32)
    perm = np.zeros(N, dtype=np.int32)
    lev = ctypes.c_int32(0)
    _check(lib.vie_mesh_host(ctypes.byref(vox), leaf, ctypes.byref(n), f.ctypes.data, tp.ctypes.data,
                             tm.ctypes.data, perm.ctypes.data, ctypes.byref(lev)))
    return dict(faces=f, tp=tp, tm=tm, perm=perm, levels=lev.value)


def mesh_host_tets(mesh, leaf: int = 64):
    """Face table, tier cells and cluster-tree permutation of a general tet mesh (host only)."""
    lib = load_library()
    mm, keep = _tetmesh(mesh)
    n = ctypes.c_int64(0)
    _check(lib.vie_mesh_host_tets(ctypes.byref(mm), leaf, ctypes.byref(n), None, None, None, None, None, None, None))
    N = n.value
    f = np.zeros((N, 3), dtype=np.int32)
    tp = np.zeros(N, dtype=np.int32)
    tm = np.zeros(N, dtype=np.int32)
    perm = np.zeros(N, dtype=np.int32)
    cells = np.zeros((len(mesh.tets), 3), dtype=np.int32)
    lev = ctypes.c_int32(0)
    hc = ctypes.c_double(0)
    _check(lib.vie_mesh_host_tets(ctypes.byref(mm), leaf, ctypes.byref(n), f.ctypes.data, tp.ctypes.data,
                                  tm.ctypes.data, perm.ctypes.data, ctypes.byref(lev), cells.ctypes.data,
                                  ctypes.byref(hc)))
    return dict(faces=f, tp=tp, tm=tm, perm=perm, levels=lev.value, cells=cells, cell_pitch=hc.value)


class Operator:
    """A HOD-BF compressed VIE operator Z (and Zinv) resident on the current GPU.

    ``body`` is a voxel body (``ijk``, ``eps``, ``h``: vie_build) or a general tetrahedral
    mesh (``verts``, ``tets``, ``eps`` per tet: vie_build_mesh)."""

    def __init__(self, body, k0: float, tol_con: float = 1e-4, tol_fact: float = 0.0, leaf: int = 64,
                 factor_dtype: str = "c64", seed: int = 1, oversample: int = 10, id_tol_div: int = 1,
                 inv_dense_max: int = 0, prec: int = 0, stream=None):
        lib = load_library()
        self._h = ctypes.c_void_p()
        cfg = _Config(tol_con, tol_fact, leaf, VIE_C64 if factor_dtype == "c64" else VIE_C128, seed, oversample,
                      id_tol_div, inv_dense_max, prec)
        if hasattr(body, "tets"):
            mm, keep = _tetmesh(body)
            _check(lib.vie_build_mesh(ctypes.byref(mm), float(k0), ctypes.byref(cfg), _stream_ptr(stream),
                                      ctypes.byref(self._h)))
        else:
            ijk = np.ascontiguousarray(body.ijk, dtype=np.int32)
            eps = np.ascontiguousarray(np.stack([np.real(body.eps), np.imag(body.eps)], 1), dtype=np.float64)
            vox = _Voxels(len(ijk), ijk.ctypes.data, eps.ctypes.data, float(body.h))
            _check(lib.vie_build(ctypes.byref(vox), float(k0), ctypes.byref(cfg), _stream_ptr(stream),
                                 ctypes.byref(self._h)))
        self.stats = self.get_stats()
        self.n = int(self.stats.n)

    @classmethod
    def load(cls, path: str, stream=None) -> "Operator":
        """An operator read back from a vie_save file (bit-identical applies)."""
        lib = load_library()
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p()
        _check(lib.vie_load(os.fsencode(path), _stream_ptr(stream), ctypes.byref(self._h)))
        self.stats = self.get_stats()
        self.n = int(self.stats.n)
        return self

    def shard_range(self, rank: int, nranks: int):
        """Tree positions [lo, hi) owned by `rank` of `nranks` (node `rank` at level log2(nranks))."""
        lo, hi = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(_lib.vie_shard_range(self._h, rank, nranks, ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def apply_shard(self, X, Y, rank: int, nranks: int, op: int = VIE_OP_Z, stream=None):
        """Write rank's rows of Y = op X (original face order) from the whole of X."""
        Xc, nrhs, ldx = _colmajor(X, self.n)
        Yc, _, ldy = _colmajor(Y, self.n)
        assert Yc.data_ptr() == Y.data_ptr() or Y.dim() == 1, "Y must be column-major"
        _check(_lib.vie_apply_shard(self._h, op, rank, nranks, ctypes.c_void_p(Xc.data_ptr()),
                                    ctypes.c_void_p(Yc.data_ptr()), nrhs, ldx, ldy, _dtype_code(Xc),
                                    _stream_ptr(stream)))
        return Y

    def set_prec(self, prec: int):
        """Switch the multi-RHS arithmetic (VIE_P_C32, VIE_P_TC_BF16X3, VIE_P_TC_TF32) of c64 factors."""
        _check(_lib.vie_set_prec(self._h, prec))

    def save(self, path: str, stream=None):
        _check(_lib.vie_save(self._h, os.fsencode(path), _stream_ptr(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None:
            _lib.vie_destroy(h)
            self._h = ctypes.c_void_p()

    def close(self):
        self.__del__()

    def check(self, stream=None):
        """Raise VieError(VIE_ETIMEOUT) if a bounded device wait of an earlier apply ran out."""
        _check(_lib.vie_check(self._h, _stream_ptr(stream)))

    def get_stats(self) -> Stats:
        st = Stats()
        _check(_lib.vie_stats(self._h, ctypes.byref(st)))
        return st

    def apply(self, X, Y=None, op: int = VIE_OP_Z, stream=None):
        """Y = Z X (op = VIE_OP_Z) or Zinv X; X complex CUDA tensor (N,) or (N, nrhs)."""
        import torch

        squeeze = X.dim() == 1
        Xc, nrhs, ldx = _colmajor(X, self.n)
        if Y is None:
            Y = torch.empty((nrhs, self.n), dtype=X.dtype, device=X.device).t()
        Yc, _, ldy = _colmajor(Y, self.n)
        assert Yc.data_ptr() == Y.data_ptr() or Y.dim() == 1, "Y must be column-major"
        _check(_lib.vie_apply(self._h, op, ctypes.c_void_p(Xc.data_ptr()), ctypes.c_void_p(Yc.data_ptr()), nrhs,
                              ldx, ldy, _dtype_code(Xc), _stream_ptr(stream)))
        return Yc[:, 0] if squeeze else Yc

    def apply_noalloc(self, X, Y, op: int = VIE_OP_Z, stream=None):
        """Y = op X like ``apply``, with the library's fixed work array instead of allocations."""
        Xc, nrhs, ldx = _colmajor(X, self.n)
        Yc, _, ldy = _colmajor(Y, self.n)
        assert Yc.data_ptr() == Y.data_ptr() or Y.dim() == 1, "Y must be column-major"
        _check(_lib.vie_apply_noalloc(self._h, op, ctypes.c_void_p(Xc.data_ptr()), ctypes.c_void_p(Yc.data_ptr()),
                                      nrhs, ldx, ldy, _dtype_code(Xc), _stream_ptr(stream)))
        return Y

    def apply_profile(self, X, Y, op: int = VIE_OP_Z, stream=None):
        """Apply with per-kernel CUDA-event times: (ms array [gather, stages..., scatter], launches)."""
        Xc, nrhs, ldx = _colmajor(X, self.n)
        Yc, _, ldy = _colmajor(Y, self.n)
        ms = np.zeros(64, dtype=np.float64)
        launches = ctypes.c_int64(0)
        _check(_lib.vie_apply_profile(self._h, op, ctypes.c_void_p(Xc.data_ptr()), ctypes.c_void_p(Yc.data_ptr()),
                                      nrhs, ldx, ldy, _dtype_code(Xc), _stream_ptr(stream), ms.ctypes.data,
                                      ctypes.byref(launches), 64))
        ns = self.program_info(op)[0].size + 2
        return ms[:ns], launches.value

    def program_info(self, op: int = VIE_OP_Z):
        """Per-stage (entries, bytes, tiles) numpy arrays of the apply program."""
        e = np.zeros(64, dtype=np.int64)
        b = np.zeros(64, dtype=np.int64)
        t = np.zeros(64, dtype=np.int64)
        ns = ctypes.c_int32(0)
        _check(_lib.vie_program_info(self._h, op, e.ctypes.data, b.ctypes.data, t.ctypes.data, 64, ctypes.byref(ns)))
        return e[:ns.value], b[:ns.value], t[:ns.value]

    def autotune(self, op: int = VIE_OP_Z, stream=None):
        """Tune the single-RHS stage tiling; returns the chosen candidate index per stage."""
        ch = np.zeros(64, dtype=np.int32)
        _check(_lib.vie_autotune(self._h, op, ch.ctypes.data, 64, _stream_ptr(stream)))
        return ch[: self.program_info(op)[0].size]

    def autotune_rhs(self, op: int = VIE_OP_Z, stream=None) -> int:
        """Time the SIMT and tensor-core multi-RHS paths; returns the column count from which
        applies use the tensor cores."""
        m = ctypes.c_int32(0)
        _check(_lib.vie_autotune_rhs(self._h, op, ctypes.byref(m), _stream_ptr(stream)))
        return int(m.value)

    def set_tiling(self, choice, op: int = VIE_OP_Z, stream=None):
        """Set every stage's single-RHS kernel/tiling to an autotuner candidate index (0-20)."""
        ch = np.ascontiguousarray(choice, dtype=np.int32)
        _check(_lib.vie_set_tiling(self._h, op, ch.ctypes.data, len(ch), _stream_ptr(stream)))

    def program_blocks(self, op: int, stage: int):
        """(M, K) int32 arrays of the blocks of one stage."""
        cnt = ctypes.c_int64(0)
        _check(_lib.vie_program_blocks(self._h, op, stage, None, None, 0, ctypes.byref(cnt)))
        M = np.zeros(cnt.value, dtype=np.int32)
        K = np.zeros(cnt.value, dtype=np.int32)
        _check(_lib.vie_program_blocks(self._h, op, stage, M.ctypes.data, K.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return M, K

    def entries(self, rows, cols, stream=None):
        """Z(rows[i], cols[i]) in FP64 (int32 CUDA tensors) -> complex128 CUDA tensor."""
        import torch

        rows = rows.to(torch.int32).contiguous()
        cols = cols.to(torch.int32).contiguous()
        out = torch.empty(rows.numel(), dtype=torch.complex128, device=rows.device)
        _check(_lib.vie_entries(self._h, ctypes.c_void_p(rows.data_ptr()), ctypes.c_void_p(cols.data_ptr()),
                                rows.numel(), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def rhs_planewave(self, khat, pol, stream=None):
        import torch

        khat = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
        pol = np.ascontiguousarray(np.atleast_2d(pol), dtype=np.float64)
        nrhs = len(khat)
        V = torch.empty((nrhs, self.n), dtype=torch.complex128, device="cuda").t()
        _check(_lib.vie_rhs_planewave(self._h, khat.ctypes.data, pol.ctypes.data, nrhs,
                                      ctypes.c_void_p(V.data_ptr()), _stream_ptr(stream)))
        return V

    def solve(self, V, rtol=1e-6, restart=30, max_iter=500, stream=None):
        import torch

        Vc, nrhs, ld = _colmajor(V.to(torch.complex128), self.n)
        assert ld == self.n
        I = torch.empty((nrhs, self.n), dtype=torch.complex128, device=V.device).t()
        iters = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs, dtype=np.float64)
        st = _lib.vie_solve(self._h, ctypes.c_void_p(Vc.data_ptr()), ctypes.c_void_p(I.data_ptr()), nrhs,
                            float(rtol), restart, max_iter, iters.ctypes.data, rel.ctypes.data, _stream_ptr(stream))
        if st not in (VIE_OK, VIE_ENOTCONV):
            _check(st)
        return I, iters, rel, st

    def solve_tfqmr(self, V, rtol=1e-3, max_iter=500, stream=None):
        """Left-preconditioned TFQMR (Eq. 6); returns (I, iterations, true relative residual, status)."""
        import torch

        Vc, nrhs, ld = _colmajor(V.to(torch.complex128), self.n)
        assert ld == self.n
        I = torch.empty((nrhs, self.n), dtype=torch.complex128, device=V.device).t()
        iters = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs, dtype=np.float64)
        st = _lib.vie_solve_tfqmr(self._h, ctypes.c_void_p(Vc.data_ptr()), ctypes.c_void_p(I.data_ptr()), nrhs,
                                  float(rtol), max_iter, iters.ctypes.data, rel.ctypes.data, _stream_ptr(stream))
        if st not in (VIE_OK, VIE_ENOTCONV):
            _check(st)
        return I, iters, rel, st

    def farfield_rcs(self, I, dirs, stream=None):
        Ic, nrhs, ld = _colmajor(I, self.n)
        assert ld == self.n
        dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        out = np.zeros((nrhs, len(dirs)), dtype=np.float64)
        _check(_lib.vie_farfield(self._h, ctypes.c_void_p(Ic.data_ptr()), nrhs, dirs.ctypes.data, len(dirs),
                                 out.ctypes.data, _stream_ptr(stream)))
        return out.T

    def faces(self):
        f = np.zeros((self.n, 3), dtype=np.int32)
        tp = np.zeros(self.n, dtype=np.int32)
        tm = np.zeros(self.n, dtype=np.int32)
        _check(_lib.vie_mesh_faces(self._h, f.ctypes.data, tp.ctypes.data, tm.ctypes.data))
        return f, tp, tm

    def tree_perm(self):
        p = np.zeros(self.n, dtype=np.int32)
        _check(_lib.vie_tree_perm(self._h, p.ctypes.data))
        return p


def tree_bounds(n: int, levels: int):
    """Node offsets of every level of the cluster tree (tree positions): the KD bisection
    gives the first child ceil(n/2) of a node's n faces, so the bounds follow from n alone."""
    b = [[0, n]]
    for _ in range(levels):
        nxt = [0]
        for lo, hi in zip(b[-1][:-1], b[-1][1:]):
            nxt += [lo + (hi - lo + 1) // 2, hi]
        b.append(nxt)
    return b


def shard_faces(perm, levels: int, nranks: int):
    """Faces owned by each of `nranks` ranks (node r at tree level log2(nranks)): a list of int arrays."""
    lev = int(nranks).bit_length() - 1
    assert 1 << lev == nranks and lev <= levels, "nranks must be a power of two, at most 2^levels"
    b = tree_bounds(len(perm), levels)[lev]
    return [np.asarray(perm[b[r]:b[r + 1]]) for r in range(nranks)]


def allgather_rows(x_rows, faces, n: int, group=None):
    """The whole of X on every rank from each rank's rows (torch.distributed all_gather of the
    rows, padded to the largest share, placed at their faces): the data plane of the sharded
    apply (Sec. III-D).  x_rows: (rows_r, nrhs) tensor of this rank's faces; faces: all ranks'
    face arrays; returns an (n, nrhs) tensor on x_rows' device."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    width = max(len(f) for f in faces)
    nrhs = x_rows.shape[1]
    pad = torch.zeros((width, nrhs), dtype=x_rows.dtype, device=x_rows.device)
    pad[: x_rows.shape[0]] = x_rows
    # complex tensors travel as real pairs (every backend moves real dtypes)
    parts = [torch.zeros((width, nrhs, 2), dtype=pad.real.dtype, device=pad.device) for _ in range(world)]
    dist.all_gather(parts, torch.view_as_real(pad).contiguous(), group=group)
    X = torch.zeros((n, nrhs), dtype=x_rows.dtype, device=x_rows.device)
    for r in range(world):
        idx = torch.as_tensor(faces[r], dtype=torch.long, device=x_rows.device)
        X[idx] = torch.view_as_complex(parts[r][: len(faces[r])].contiguous())
    return X


class ShardedOperator:
    """An operator applied across the ranks of a torch.distributed group by subtrees
    (vie_apply_shard): each rank owns node `rank` of tree level log2(world) and returns its
    rows of op X from its rows of X after one all-gather."""

    def __init__(self, op: Operator, group=None):
        import torch.distributed as dist

        self.op, self.group = op, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.faces = shard_faces(op.tree_perm(), int(op.stats.levels), self.world)

    def apply(self, x_rows, op: int = VIE_OP_Z, stream=None):
        import torch

        X = allgather_rows(x_rows, self.faces, self.op.n, self.group)
        Xc = X.t().contiguous().t()
        Y = torch.zeros_like(Xc)
        self.op.apply_shard(Xc, Y, self.rank, self.world, op=op, stream=stream)
        idx = torch.as_tensor(self.faces[self.rank], dtype=torch.long, device=Y.device)
        return Y[idx]


class Server:
    """Continuous-batching solve server over resident operators (vie_server_* in include/vie.h)."""

    def __init__(self, ops, restart: int = 30, max_iter: int = 300, mem_budget: int = 32 << 30, stream=None):
        lib = load_library()
        self.ops = list(ops)
        arr = (ctypes.c_void_p * len(self.ops))(*[o._h.value for o in self.ops])
        self._h = ctypes.c_void_p()
        self._keep = arr
        _check(lib.vie_server_create(arr, len(self.ops), restart, max_iter, int(mem_budget), _stream_ptr(stream),
                                     ctypes.byref(self._h)))

    def submit(self, op: int, V, rtol: float = 1e-3) -> int:
        """V: numpy complex128 (N, nrhs) or (N,); returns the request id."""
        V = np.asarray(V, dtype=np.complex128)
        if V.ndim == 1:
            V = V[:, None]
        Vf = np.asfortranarray(V)
        rid = ctypes.c_int64(0)
        _check(_lib.vie_server_submit(self._h, op, Vf.ctypes.data, V.shape[1], float(rtol), ctypes.byref(rid)))
        return rid.value

    def step(self):
        a, p = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(_lib.vie_server_step(self._h, ctypes.byref(a), ctypes.byref(p)))
        return a.value, p.value

    def result(self, rid: int, n: int, nrhs: int):
        """(I (N, nrhs) complex128, iters, relres, latency_s) or None while the request runs."""
        I = np.zeros((n, nrhs), dtype=np.complex128, order="F")
        it = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs, dtype=np.float64)
        lat = ctypes.c_double(0)
        st = _lib.vie_server_result(self._h, rid, I.ctypes.data, it.ctypes.data, rel.ctypes.data, ctypes.byref(lat))
        if st == VIE_ENOTCONV:
            return None
        _check(st)
        return I, it, rel, lat.value

    def cancel(self, rid: int):
        """Drop request rid (pending, running or finished); its memory returns to the budget."""
        _check(_lib.vie_server_cancel(self._h, rid))

    def memory(self):
        """(bytes held by the admitted requests' Krylov state, budget)."""
        used, budget = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(_lib.vie_server_memory(self._h, ctypes.byref(used), ctypes.byref(budget)))
        return used.value, budget.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.vie_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        self.close()


def apply_group(jobs, stream=None):
    """Grouped apply (``vie_apply_group``): ``jobs`` is a list of (Operator, X, op) with op
    VIE_OP_Z or VIE_OP_ZINV and X a complex64 CUDA tensor (N,) or (N, nrhs); the independent
    applies run as one launch per stage depth.  Returns the list of results (same shapes)."""
    import torch

    n = len(jobs)
    outs, keep = [], []
    ops = (ctypes.c_void_p * max(1, n))()
    which = (ctypes.c_int32 * max(1, n))()
    xs = (ctypes.c_void_p * max(1, n))()
    ys = (ctypes.c_void_p * max(1, n))()
    nr = (ctypes.c_int64 * max(1, n))()
    for i, (opr, X, kind) in enumerate(jobs):
        assert X.dtype == torch.complex64, "grouped applies take complex64 vectors"
        Xc, nrhs, ldx = _colmajor(X, opr.n)
        assert ldx == opr.n, "grouped applies take X with leading dimension N"
        Y = torch.empty((nrhs, opr.n), dtype=X.dtype, device=X.device).t()
        keep.append(Xc)
        outs.append(Y[:, 0] if X.dim() == 1 else Y)
        ops[i], which[i], xs[i], ys[i], nr[i] = opr._h.value, kind, Xc.data_ptr(), Y.data_ptr(), nrhs
    _check(_lib.vie_apply_group(ops, which, xs, ys, nr, n, _stream_ptr(stream)))
    return outs
