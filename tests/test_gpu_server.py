"""Request server on the GPU: every permutation equals the plain ordering of
that matrix alone (bit-exact: the permutation is integer work), whether the
request ran alone or mixed into batches with others that arrived while
earlier ones were on the device; admission stays within the memory budget;
cancellation and rejection behave as documented."""
import time

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4490_gb300 as P
    assert torch.cuda.is_available()
    return P


PARAMS = dict(d=3, seed=3)


def _plain(V, A):
    hg = V.Hypergraph.from_matrix(A)
    rp, _, _ = hg.order(V.Params(**PARAMS), None, sbd=False, with_tree=False)
    return rp.cpu().numpy()


def _mix(count, seed):
    return W.batch_mix(count, seed, nmin=200, nmax=3000)


def test_alone_equals_mixed_equals_plain(V):
    mats = _mix(24, 41) + [W.grid_laplacian_3d(20)]
    target = len(mats) - 1
    ref = {i: _plain(V, A) for i, A in enumerate(mats)}
    # alone
    with V.Server(V.Params(**PARAMS), slots=2) as srv:
        rid = srv.submit_matrix(mats[target])
        info = srv.wait(rid, 120.0)
        assert info["state"] == "done" and info["batch_size"] == 1
        assert np.array_equal(srv.result(rid), ref[target])
    # mixed: staggered arrivals while earlier batches run, small batches
    with V.Server(V.Params(**PARAMS), slots=3, max_batch=6) as srv:
        ids = []
        for i, A in enumerate(mats):
            ids.append(srv.submit_matrix(A))
            if i % 5 == 4:
                time.sleep(0.02)
        infos = [srv.wait(r, 300.0) for r in ids]
        assert all(d["state"] == "done" for d in infos)
        for i, r in enumerate(ids):
            assert np.array_equal(srv.result(r), ref[i]), i
        st = srv.stats()
        assert st["completed"] == len(mats) and st["failed"] == 0
        assert st["batches"] >= 2
        assert max(d["batch_size"] for d in infos) >= 2          # requests were batched together
        # work of different batches overlapped in time (continuous admission)
        spans = sorted((d["t_admit"], d["t_done"], d["batch"]) for d in infos)
        overlap = any(a2 < d1 and b1 != b2 for (a1, d1, b1), (a2, d2, b2) in zip(spans, spans[1:]))
        assert overlap


def test_budget_admission(V):
    mats = _mix(16, 43)
    est = [V.server.estimate_bytes(A.m, A.colidx.size) for A in mats]
    budget = int(max(est) * 1.6)
    with V.Server(V.Params(**PARAMS), slots=4, budget_bytes=budget) as srv:
        ids = [srv.submit_matrix(A) for A in mats]
        for r in ids:
            assert srv.wait(r, 300.0)["state"] == "done"
        st = srv.stats()
        assert st["bytes_peak"] <= budget and st["bytes_in_use"] == 0
        big = W.grid_laplacian_2d(400)
        with pytest.raises(V.VmoError) as e:
            srv.submit_matrix(big)
        assert e.value.status == 5  # VMO_ERR_BUDGET


def test_cancel_and_reject(V):
    mats = _mix(8, 44)
    with V.Server(V.Params(**PARAMS), slots=1, max_batch=1) as srv:
        ids = [srv.submit_matrix(A) for A in mats]
        srv.cancel(ids[-1])
        last = srv.wait(ids[-1], 60.0)
        assert last["state"] == "cancelled"
        for r in ids[:-1]:
            assert srv.wait(r, 300.0)["state"] == "done"
        # malformed patterns are rejected at submission
        with pytest.raises(V.VmoError):
            srv.submit(np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32))
        with pytest.raises(V.VmoError):
            srv.submit(np.array([0, 1, 2], np.int32), np.array([0, 5], np.int32))
        assert srv.stats()["cancelled"] == 1


def test_cancel_running_stays_running_until_batch_ends(V):
    """A request cancelled while its batch runs is not terminal until the batch
    ends (the batch may still read its host arrays); it then turns cancelled
    with nothing written, and release frees its record only then."""
    big = W.grid_laplacian_3d(48)  # long enough to be caught running
    with V.Server(V.Params(**PARAMS), slots=1, max_batch=1) as srv:
        rid = srv.submit_matrix(big)
        t0 = time.time()
        while srv.poll(rid)["state"] == "queued" and time.time() - t0 < 60:
            time.sleep(0.001)
        assert srv.poll(rid)["state"] == "running"
        srv.cancel(rid)
        st = srv.poll(rid)["state"]
        assert st in ("running", "cancelled")
        if st == "running":
            assert srv.release(rid) is False  # not terminal yet: nothing freed
        info = srv.wait(rid, 300.0)
        assert info["state"] == "cancelled"
        assert srv.stats()["cancelled"] == 1 and srv.stats()["completed"] == 0
        assert srv.release(rid) is True
        with pytest.raises(V.VmoError):
            srv.poll(rid)  # the record is gone
        # the server keeps serving after a cancelled batch
        A = _mix(1, 45)[0]
        r2 = srv.submit_matrix(A)
        assert srv.wait(r2, 300.0)["state"] == "done"
        assert np.array_equal(srv.result(r2), _plain(V, A))
        assert srv.release(r2) is True
