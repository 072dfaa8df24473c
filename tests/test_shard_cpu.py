"""Data plane and ownership of the sharded apply (Sec. III-D subtree ownership) on CPU ranks:
world size 2 over gloo.  Each rank owns node `rank` of tree level log2(world); the all-gather of
the ranks' rows rebuilds X exactly, the ownership follows the oracle's cluster tree, and the
ranks' rows of a dense matvec with the gathered X assemble to the full product."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import paper_2111_01730_gb300 as pkg
    import workloads as W
    from oracle.entries import Elements, zblock
    from oracle.hodbf import cluster_tree, face_centroids
    from oracle.mesh import build_mesh

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    body = W.sphere(0.15, 4.0 - 0.5j, 1.0 / 16)
    mh = pkg.mesh_host(body, leaf=32)  # the library's tree, host only
    perm, levels = mh["perm"], mh["levels"]
    n = len(perm)
    faces = pkg.shard_faces(perm, levels, world)
    # ownership = the oracle's cluster-tree node bounds at level log2(world)
    operm, LH, bounds = cluster_tree(face_centroids(build_mesh(body)), 32)
    lev = world.bit_length() - 1
    mine = operm[bounds[lev][rank]:bounds[lev][rank + 1]]
    assert LH == levels and np.array_equal(np.sort(mine), np.sort(faces[rank]))
    assert sorted(np.concatenate(faces).tolist()) == list(range(n))
    x = torch.from_numpy(W.random_block(n, 3, seed=8))
    X = pkg.allgather_rows(x[torch.as_tensor(faces[rank])], faces, n)
    assert torch.equal(X, x)  # bit for bit
    mesh = build_mesh(body)
    Z = zblock(Elements(mesh, W.K0), faces[rank], np.arange(n))
    y_rows = Z @ X.numpy()
    np.save(os.path.join(out_dir, f"y{rank}.npy"), y_rows)
    np.save(os.path.join(out_dir, f"f{rank}.npy"), faces[rank])
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_data_plane_two_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as W
    from oracle.entries import Elements, zblock
    from oracle.mesh import build_mesh

    body = W.sphere(0.15, 4.0 - 0.5j, 1.0 / 16)
    mesh = build_mesh(body)
    n = len(mesh["faces"])
    x = W.random_block(n, 3, seed=8)
    y = np.zeros((n, 3), dtype=np.complex128)
    for r in range(world):
        y[np.load(tmp_path / f"f{r}.npy")] = np.load(tmp_path / f"y{r}.npy")
    Z = zblock(Elements(mesh, W.K0), np.arange(n), np.arange(n))
    assert np.allclose(y, Z @ x, rtol=1e-12, atol=1e-14 * np.abs(Z @ x).max())
