"""CPU checks of the library's host logic (mesh, SWG face table, cluster tree) against the oracle, bit for bit."""
import numpy as np
import pytest

import workloads as W
from oracle.hodbf import cluster_tree, face_centroids
from oracle.mesh import build_mesh


@pytest.mark.parametrize("body", [
    W.tiny_block(3, 2, 2, h=0.06),
    W.sphere(0.2, 4.0 - 1.0j, 1.0 / 16),
    W.shell(0.25, 0.15, W.drude_eps(), 1.0 / 20),
    W.sphere(0.3, 4.0, 1.0 / 14),
], ids=["block", "sphere", "shell", "sphere3960"])
def test_mesh_and_tree_match_oracle(body):
    import paper_2111_01730_gb300 as pkg

    r = pkg.mesh_host(body, 64)
    m = build_mesh(body)
    assert np.array_equal(r["faces"], m["faces"])
    assert np.array_equal(r["tp"], m["face_tp"]) and np.array_equal(r["tm"], m["face_tm"])
    perm, LH, _ = cluster_tree(face_centroids(m), 64)
    assert r["levels"] == LH
    assert np.array_equal(r["perm"], perm)


def test_mesh_host_rejects_bad_input():
    import paper_2111_01730_gb300 as pkg

    bad = W.VoxelBody("bad", -1.0, np.zeros((1, 3), np.int32), np.ones(1, np.complex128))
    with pytest.raises(pkg.VieError) as e:
        pkg.mesh_host(bad)
    assert e.value.status == pkg.VIE_EINVAL
    dup = W.VoxelBody("dup", 0.1, np.zeros((2, 3), np.int32), np.ones(2, np.complex128))
    with pytest.raises(pkg.VieError):
        pkg.mesh_host(dup)
