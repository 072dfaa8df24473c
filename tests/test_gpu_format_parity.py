"""Format parity: the factors the GPU built, read back from a vie_save file and applied on the
host in FP64, against the GPU apply of the same operator.

This separates the arithmetic of the apply kernels from the compression error.  The checkpoint
holds every stage of the Z and Zinv programs exactly as the kernels run them (block descriptors
and packed factor bytes).  The host applies each stage in FP64, reading its inputs before any of
its outputs are written.  Blocks of one stage are independent, which is what the GPU's
concurrent launch assumes.  Expected agreement:
* complex FP32 factors, complex FP32 vectors (FP32 accumulation): a few FP32 roundings per
  stage, bound 2e-6;
* the same on the tensor cores (16 columns, BF16x3 split products, FP32 accumulation): bound 5e-5;
* complex FP32 factors with complex FP64 vectors (the refinement residual's kernel), and complex
  FP64 factors: FP64 arithmetic on the same stored values, bound 1e-12.
"""
import ctypes
import struct

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402

# block descriptor of one stage: y[out] (=|+=) A (M x K, row-major, leading dimension ld) x[in]
OPDESC = np.dtype([("mat_off", "<i8"), ("in_off", "<i8"), ("out_off", "<i8"), ("M", "<i4"), ("K", "<i4"),
                   ("ld", "<i4"), ("in_space", "<i2"), ("out_space", "<i2"), ("accumulate", "<i4"),
                   ("pad", "<i4")])
SP_X, SP_Y, SP_C = 0, 1, 2


def read_checkpoint(path):
    """Programs of a vie_save file: [Z] or [Z, Zinv], each {n, ncoef, dtype, stages: [(ops, mats)]}."""
    raw = open(path, "rb").read()
    pos = 0

    def take(nb):
        nonlocal pos
        v = raw[pos:pos + nb]
        assert len(v) == nb, "truncated checkpoint"
        pos += nb
        return v

    def i64():
        return struct.unpack("<q", take(8))[0]

    def i32():
        return struct.unpack("<i", take(4))[0]

    assert take(8) == b"VIEOPv1\0"
    take(ctypes.sizeof(pkg._Config))
    take(16)  # k0, pitch
    nvox = i64()
    if nvox == -1:  # general tet mesh: vertices, tets, eps
        nv = i64()
        take(24 * nv)
        nt = i64()
        take(16 * nt + 16 * nt)
    else:  # voxel lattice: ijk, eps
        take(12 * nvox + 16 * nvox)
    stats = take(ctypes.sizeof(pkg.Stats))
    has_zinv = i32()
    take(12)  # Zinv top level, tensor-core crossovers of Z and Zinv

    def program():
        n, ncoef, entries, nbytes = i64(), i64(), i64(), i64()
        fdt = i32()
        nst = i32()
        dt = np.complex64 if fdt == pkg.VIE_C64 else np.complex128
        stages = []
        for _ in range(nst):
            nops, ntiles, mb, st_entries, st_bytes = i64(), i64(), i64(), i64(), i64()
            take(8)  # single-RHS kernel choice, padding
            ops = np.frombuffer(take(OPDESC.itemsize * nops), dtype=OPDESC)
            take(4 * nops + 16 * ntiles)  # tags, warp tiles
            mraw = take(mb)
            mats = np.frombuffer(mraw[: mb - mb % np.dtype(dt).itemsize], dtype=dt)
            stages.append((ops, mats))
        return dict(n=n, ncoef=ncoef, entries=entries, dtype=dt, stages=stages)

    progs = [program()]
    if has_zinv:
        progs.append(program())
    assert pos == len(raw), (pos, len(raw))
    return progs, struct.unpack("<q", stats[:8])[0]


def run_program(prog, xt):
    """Tree-ordered Y of the program applied to tree-ordered X (n x r), in FP64."""
    n, r = prog["n"], xt.shape[1]
    space = [xt.astype(np.complex128), np.zeros((n, r), np.complex128),
             np.zeros((max(prog["ncoef"], 1), r), np.complex128)]
    for ops, mats in prog["stages"]:
        snap = [a.copy() for a in space]  # every block of a stage reads the state before the stage
        out = []
        for o in ops:
            M, K, ld = int(o["M"]), int(o["K"]), int(o["ld"])
            if M == 0:
                continue
            if K == 0:
                v = np.zeros((M, r), np.complex128)
            else:
                off = int(o["mat_off"])
                A = mats[off:off + M * ld].reshape(M, ld)[:, :K].astype(np.complex128)
                v = A @ snap[int(o["in_space"])][int(o["in_off"]):int(o["in_off"]) + K]
            out.append((int(o["out_space"]), int(o["out_off"]), M, int(o["accumulate"]), v))
        for sp, off, M, acc, v in out:
            if acc:
                space[sp][off:off + M] += v
            else:
                space[sp][off:off + M] = v
    return space[SP_Y]


def host_apply(prog, perm, X):
    Y = np.zeros_like(X, dtype=np.complex128)
    Y[perm] = run_program(prog, X[perm])
    return Y


@pytest.mark.parametrize("factor_dtype,inv_dense_max", [("c64", 0), ("c128", 0), ("c64", 256)])
def test_gpu_apply_equals_host_apply_of_the_exported_factors(tmp_path, factor_dtype, inv_dense_max):
    """inv_dense_max 256: the inverse's levels above 256 unknowns per node come from products
    only (two-sided butterflies of Algorithms 1-2), the rest from dense blocks."""
    body = W.sphere(0.2, 4.0 - 1.0j, 1.0 / 16)  # N = 1,824
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64, factor_dtype=factor_dtype,
                      inv_dense_max=inv_dense_max)
    if inv_dense_max:
        assert op.get_stats().zinv_product_levels > 0
    path = str(tmp_path / "op.vie")
    op.save(path)
    progs, n_file = read_checkpoint(path)
    assert n_file == op.n and len(progs) == 2
    st = op.get_stats()
    for prog, which, nst, ent in ((progs[0], pkg.VIE_OP_Z, st.apply_stages_z, st.entries_z),
                                  (progs[1], pkg.VIE_OP_ZINV, st.apply_stages_zinv, st.entries_zinv)):
        assert prog["n"] == op.n and len(prog["stages"]) == nst and prog["entries"] == ent
    perm = op.tree_perm()
    cases = []
    if factor_dtype == "c64":
        cases += [(pkg.VIE_OP_Z, 1, torch.complex64, 2e-6), (pkg.VIE_OP_ZINV, 1, torch.complex64, 2e-6),
                  (pkg.VIE_OP_Z, 16, torch.complex64, 5e-5), (pkg.VIE_OP_ZINV, 16, torch.complex64, 5e-5),
                  (pkg.VIE_OP_Z, 2, torch.complex128, 1e-12)]
    else:
        cases += [(pkg.VIE_OP_Z, 1, torch.complex128, 1e-12), (pkg.VIE_OP_ZINV, 1, torch.complex128, 1e-12),
                  (pkg.VIE_OP_Z, 3, torch.complex128, 1e-12)]
    for which, nrhs, tdt, bound in cases:
        X = torch.from_numpy(W.random_block(op.n, nrhs, seed=40 + nrhs)).to(tdt)
        Xn = X.numpy().astype(np.complex128)  # the values the GPU reads, exactly
        Yg = op.apply(X.cuda(), op=which).cpu().numpy().reshape(op.n, nrhs)
        Yh = host_apply(progs[0 if which == pkg.VIE_OP_Z else 1], perm, Xn.reshape(op.n, nrhs))
        err = np.linalg.norm(Yg - Yh) / np.linalg.norm(Yh)
        print(f"format parity {factor_dtype} dense<={inv_dense_max} op={which} nrhs={nrhs} {tdt}: {err:.2e} "
              f"(bound {bound:g})")
        assert err <= bound, (factor_dtype, inv_dense_max, which, nrhs, err)
    op.check()
