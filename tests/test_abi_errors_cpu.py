"""Argument and file validation at the C ABI, on the host (no GPU, no device call reached).

Every entry point returns a status and never aborts: null handles and pointers, an invalid
voxel body or configuration, and unreadable, foreign or truncated checkpoint files are
rejected with VIE_EINVAL and a message from vie_last_error, before any CUDA call."""
import ctypes
import os

import numpy as np
import pytest

import paper_2111_01730_gb300 as pkg

P = ctypes.c_void_p


@pytest.fixture(scope="module")
def lib():
    return pkg.load_library()


def _msg(lib):
    return lib.vie_last_error().decode()


def _body():
    ijk = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    eps = np.array([[4.0, -0.5], [4.0, -0.5]], dtype=np.float64)
    return ijk, eps


def _cfg(**kw):
    c = dict(tol_con=1e-4, tol_fact=0.0, leaf=64, factor_dtype=pkg.VIE_C64, seed=1, oversample=10, id_tol_div=1,
             inv_dense_max=0, prec=pkg.VIE_P_AUTO)
    c.update(kw)
    return pkg._Config(c["tol_con"], c["tol_fact"], c["leaf"], c["factor_dtype"], c["seed"], c["oversample"],
                       c["id_tol_div"], c["inv_dense_max"], c["prec"])


@pytest.mark.parametrize("cfg,k0,text", [
    (dict(leaf=2), 6.28, "invalid configuration"),
    (dict(tol_con=0.0), 6.28, "invalid configuration"),
    (dict(), 0.0, "invalid configuration"),
    (dict(factor_dtype=7), 6.28, "factor dtype"),
    (dict(prec=99), 6.28, "bad precision"),
])
def test_build_rejects_invalid_configuration(lib, cfg, k0, text):
    ijk, eps = _body()
    vox = pkg._Voxels(len(ijk), ijk.ctypes.data, eps.ctypes.data, 0.1)
    c = _cfg(**cfg)
    out = P()
    assert lib.vie_build(ctypes.byref(vox), k0, ctypes.byref(c), None, ctypes.byref(out)) == pkg.VIE_EINVAL
    assert text in _msg(lib)
    assert not out.value
    mm = pkg._Mesh(0, None, 0, None, None)
    assert lib.vie_build_mesh(ctypes.byref(mm), k0, ctypes.byref(c), None, ctypes.byref(out)) == pkg.VIE_EINVAL
    assert text in _msg(lib)


def test_build_rejects_null_and_empty_bodies(lib):
    c = _cfg()
    out = P()
    assert lib.vie_build(None, 6.28, ctypes.byref(c), None, ctypes.byref(out)) == pkg.VIE_EINVAL
    assert "null argument" in _msg(lib)
    ijk, eps = _body()
    for nvox, h in ((0, 0.1), (2, 0.0), (2, -1.0)):
        vox = pkg._Voxels(nvox, ijk.ctypes.data, eps.ctypes.data, h)
        assert lib.vie_build(ctypes.byref(vox), 6.28, ctypes.byref(c), None, ctypes.byref(out)) == pkg.VIE_EINVAL
        assert "empty or invalid voxel body" in _msg(lib)
    assert lib.vie_build_mesh(None, 6.28, ctypes.byref(c), None, ctypes.byref(out)) == pkg.VIE_EINVAL


def test_null_handles_are_rejected(lib):
    x = ctypes.c_double(0)
    ptr = ctypes.addressof(x)
    assert lib.vie_apply(None, pkg.VIE_OP_Z, ptr, ptr, 1, 1, 1, pkg.VIE_C64, None) == pkg.VIE_EINVAL
    assert lib.vie_apply_noalloc(None, pkg.VIE_OP_Z, ptr, ptr, 1, 1, 1, pkg.VIE_C64, None) == pkg.VIE_EINVAL
    assert lib.vie_apply_shard(None, pkg.VIE_OP_Z, 0, 1, ptr, ptr, 1, 1, 1, pkg.VIE_C64, None) == pkg.VIE_EINVAL
    st = pkg.Stats()
    assert lib.vie_stats(None, ctypes.byref(st)) == pkg.VIE_EINVAL
    assert lib.vie_check(None, None) == pkg.VIE_EINVAL
    assert lib.vie_set_prec(None, pkg.VIE_P_TC_TF32) == pkg.VIE_EINVAL
    assert lib.vie_autotune(None, pkg.VIE_OP_Z, None, 0, None) == pkg.VIE_EINVAL
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    assert lib.vie_shard_range(None, 0, 1, ctypes.byref(lo), ctypes.byref(hi)) == pkg.VIE_EINVAL
    assert lib.vie_save(None, b"/nonexistent/x", None) == pkg.VIE_EINVAL
    # serving: no operators, no server
    srv = P()
    assert lib.vie_server_create(None, 0, 30, 100, 1 << 20, None, ctypes.byref(srv)) == pkg.VIE_EINVAL
    assert lib.vie_server_step(None, None, None) == pkg.VIE_EINVAL
    assert lib.vie_server_cancel(None, 0) == pkg.VIE_EINVAL
    rid = ctypes.c_int64()
    assert lib.vie_server_submit(None, 0, ptr, 1, 1e-3, ctypes.byref(rid)) == pkg.VIE_EINVAL
    lib.vie_destroy(None)          # no-ops on null handles
    lib.vie_server_destroy(None)
    # an empty group is a no-op, a group with missing arrays is not
    assert lib.vie_apply_group(None, None, None, None, None, 0, None) == pkg.VIE_OK
    assert lib.vie_apply_group(None, None, None, None, None, 1, None) == pkg.VIE_EINVAL
    assert lib.vie_wait_selftest(0, None) == pkg.VIE_EINVAL


def test_load_rejects_missing_foreign_and_truncated_files(lib, tmp_path):
    out = P()
    assert lib.vie_load(os.fsencode(tmp_path / "missing.vie"), None, ctypes.byref(out)) == pkg.VIE_EINVAL
    assert "cannot open" in _msg(lib)
    foreign = tmp_path / "foreign.vie"
    foreign.write_bytes(b"not a checkpoint of an operator")
    assert lib.vie_load(os.fsencode(foreign), None, ctypes.byref(out)) == pkg.VIE_EINVAL
    assert "not an operator file" in _msg(lib)
    for cut in (0, 3, 8, 8 + 16):  # empty, inside the magic, after it, inside the configuration
        trunc = tmp_path / f"trunc{cut}.vie"
        trunc.write_bytes(b"VIEOPv1\0" + bytes(64)[: max(0, cut - 8)] if cut >= 8 else b"VIEOPv1\0"[:cut])
        assert lib.vie_load(os.fsencode(trunc), None, ctypes.byref(out)) == pkg.VIE_EINVAL
        assert "truncated" in _msg(lib) or "not an operator file" in _msg(lib)
    assert not out.value
    assert lib.vie_load(None, None, ctypes.byref(out)) == pkg.VIE_EINVAL


def test_load_rejects_a_bad_body_header(lib, tmp_path):
    """A file with the right magic whose body header cannot describe a mesh (zero pitch, a
    negative voxel count) is refused before the library builds anything."""
    cfg = bytes(_cfg())
    out = P()
    for k0, h, nvox in ((6.28, 0.0, 2), (6.28, 0.1, -5), (0.0, 0.1, 2), (6.28, 0.1, 0)):
        f = tmp_path / "hdr.vie"
        f.write_bytes(b"VIEOPv1\0" + cfg + np.array([k0, h]).tobytes() + np.array([nvox], dtype=np.int64).tobytes())
        assert lib.vie_load(os.fsencode(f), None, ctypes.byref(out)) == pkg.VIE_EINVAL
        assert "bad body header" in _msg(lib)
    assert not out.value
    # a configuration no build accepts (leaf < 4, chi_con <= 0, unknown factor type or precision)
    for bad in (dict(leaf=2), dict(tol_con=0.0), dict(factor_dtype=7), dict(prec=99)):
        f = tmp_path / "cfg.vie"
        f.write_bytes(b"VIEOPv1\0" + bytes(_cfg(**bad)) + np.array([6.28, 0.1]).tobytes()
                      + np.array([2], dtype=np.int64).tobytes())
        assert lib.vie_load(os.fsencode(f), None, ctypes.byref(out)) == pkg.VIE_EINVAL
        assert "bad configuration" in _msg(lib)


def test_voxel_body_rejects_zero_or_non_finite_permittivity():
    """kappa = (eps_r - 1) / eps_r needs a finite, nonzero eps_r (host mesh builder, no GPU)."""
    import workloads as W

    ijk = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    for bad in (0.0, np.nan, np.inf, complex(1.0, np.nan)):
        body = W.VoxelBody("bad_eps", 0.1, ijk, np.array([4.0 - 0.5j, bad], dtype=np.complex128))
        with pytest.raises(pkg.VieError) as e:
            pkg.mesh_host(body)
        assert e.value.status == pkg.VIE_EINVAL and "eps_r" in str(e.value)
    ok = W.VoxelBody("ok", 0.1, ijk, np.array([4.0 - 0.5j, 1.0], dtype=np.complex128))
    assert len(pkg.mesh_host(ok)["perm"]) > 0
