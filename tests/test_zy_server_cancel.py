"""Serving: cancelling requests (failure handling on the host, no device fault).  A running
request leaves the batch and its Krylov memory returns to the budget, a pending one is dropped
before admission, a finished one discards its result, and the request that stays gives the
same solution as alone."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_2111_01730_gb300 as pkg  # noqa: E402


def _finish(srv, rid, n, nrhs, max_steps=500):
    for _ in range(max_steps):
        srv.step()
        r = srv.result(rid, n, nrhs)
        if r is not None:
            return r
    raise AssertionError("request did not finish")


def test_cancel_running_pending_and_finished_requests():
    a = pkg.Operator(W.sphere(0.2, 4.0 - 1.0j, 1.0 / 16), W.K0, tol_con=1e-4, tol_fact=1e-1, leaf=64)
    k, p = W.planewave_random(3, seed=41)
    V = a.rhs_planewave(k, p).cpu().numpy()
    # the request alone
    solo = pkg.Server([a], restart=30, max_iter=300, mem_budget=4 << 30)
    r0 = solo.submit(0, V, rtol=1e-4)
    alone = _finish(solo, r0, a.n, 3)
    assert solo.memory()[0] == 0
    solo.close()
    # the same request next to one that is cancelled while running and one cancelled while pending
    srv = pkg.Server([a], restart=30, max_iter=300, mem_budget=4 << 30)
    r1 = srv.submit(0, V, rtol=1e-4)
    r2 = srv.submit(0, V[:, :2], rtol=1e-4)
    srv.step()
    used_both, budget = srv.memory()
    assert 0 < used_both <= budget
    srv.cancel(r2)
    used_one = srv.memory()[0]
    assert 0 < used_one < used_both
    r3 = srv.submit(0, V[:, :1], rtol=1e-4)
    srv.cancel(r3)
    mixed = _finish(srv, r1, a.n, 3)
    assert np.all(mixed[2] <= 1e-4)
    err = np.linalg.norm(mixed[0] - alone[0]) / np.linalg.norm(alone[0])
    assert err < 1e-9, err
    assert srv.memory()[0] == 0
    for rid in (r2, r3):
        with pytest.raises(pkg.VieError) as e:
            srv.result(rid, a.n, 1)
        assert e.value.status == pkg.VIE_EINVAL
    # a finished request whose result nobody collected
    r4 = srv.submit(0, V[:, :1], rtol=1e-4)
    for _ in range(500):
        act, pend = srv.step()
        if act == 0 and pend == 0:
            break
    srv.cancel(r4)
    with pytest.raises(pkg.VieError):
        srv.result(r4, a.n, 1)
    with pytest.raises(pkg.VieError) as e:
        srv.cancel(12345)
    assert e.value.status == pkg.VIE_EINVAL
    srv.close()
