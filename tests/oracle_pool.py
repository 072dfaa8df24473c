"""Dense oracle matrices assembled in parallel (test helper).

The oracle's plain element-pair sum (oracle/entries.zblock) is slow in Python; for the
mid-size validation bodies (N around 10^4) its rows are split over a pool of worker
processes started with `spawn` (safe after a CUDA context exists in the parent).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _rows(args):
    import workloads as W
    from oracle.entries import Elements, zblock
    from oracle.mesh import build_mesh

    body, k0, rows = args
    mesh = build_mesh(body)
    E = Elements(mesh, k0)
    return zblock(E, rows, np.arange(len(mesh["faces"])))


def dense_z(body, k0, procs: int | None = None, chunk: int = 256) -> np.ndarray:
    """Z(all, all) of the oracle for a voxel body, rows assembled by `procs` spawned workers."""
    from oracle.mesh import build_mesh

    n = len(build_mesh(body)["faces"])
    procs = procs or max(1, (os.cpu_count() or 2))
    parts = [np.arange(a, min(n, a + chunk)) for a in range(0, n, chunk)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        blocks = pool.map(_rows, [(body, k0, r) for r in parts])
    return np.concatenate(blocks, axis=0)


def _some_rows(args):
    import workloads as W  # noqa: F401
    from oracle.entries import Elements, zblock
    from oracle.mesh import build_mesh

    body, k0, rows = args
    mesh = build_mesh(body)
    E = Elements(mesh, k0)
    return zblock(E, rows, np.arange(len(mesh["faces"])), chunk=2)


def z_rows(body, k0, rows, procs: int | None = None, per: int = 4) -> np.ndarray:
    """Rows Z(rows, all) of the oracle, `per` rows per task over `procs` spawned workers."""
    rows = np.asarray(rows)
    procs = procs or max(1, (os.cpu_count() or 2))
    parts = [rows[a:a + per] for a in range(0, len(rows), per)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(procs, len(parts))) as pool:
        blocks = pool.map(_some_rows, [(body, k0, r) for r in parts])
    return np.concatenate(blocks, axis=0)


def _pair_task(args):
    from oracle import entries as EN
    from oracle import quadrature as Q
    from oracle.entries import Elements, zblock

    mesh, k0, m, n, orders = args
    near, smooth, far = orders
    EN.RULES.update({
        "far_tet": lambda: Q.tet_conical(far), "far_tri": lambda: Q.tri_conical(far),
        "mid_tet": lambda: Q.tet_conical(far), "mid_tri": lambda: Q.tri_conical(far),
        "near_tet": lambda: Q.tet_conical(near), "near_tri": lambda: Q.tri_conical(near),
        "smooth_tet": lambda: Q.tet_conical(smooth), "smooth_tri": lambda: Q.tri_conical(smooth),
    })
    return zblock(Elements(mesh, k0), [m], [n])[0, 0]


def raised_entries(mesh, k0, pairs, near: int, smooth: int, far: int, procs: int | None = None) -> np.ndarray:
    """Z(m, n) of the oracle for each pair with every rule raised to conical orders (near, smooth,
    far), one pair per spawned worker (the rule table is set in the worker, not in the caller)."""
    pairs = list(pairs)
    procs = min(len(pairs), procs or max(1, (os.cpu_count() or 2)))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return np.array(pool.map(_pair_task, [(mesh, k0, m, n, (near, smooth, far)) for m, n in pairs]))
