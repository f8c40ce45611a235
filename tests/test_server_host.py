"""Host logic of the request server (no GPU): the admission estimate, the
batch-forming rule of a free slot, and an event simulation of the rule with
the server's accounting showing that the budget is never exceeded and that
every request is admitted in arrival order."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    from paper_1105_4490_gb300 import _build_lib
    _build_lib.build()
    from paper_1105_4490_gb300 import server
    return server


def test_estimate(S):
    assert S.estimate_bytes(0, 0) == 1 << 20
    assert S.estimate_bytes(1000, 5000) == 512 * 1000 + 64 * 5000 + (1 << 20)


def test_plan_rules(S):
    b = [10, 10, 10, 10]
    z = [5, 5, 5, 5]
    assert S.plan(b, z, 100, 8, 100) == 4          # everything fits
    assert S.plan(b, z, 25, 8, 100) == 2           # budget
    assert S.plan(b, z, 100, 3, 100) == 3          # max_batch
    assert S.plan(b, z, 100, 8, 12) == 2           # nonzeros per batch
    assert S.plan(b, z, 9, 8, 100) == 0            # head does not fit yet
    assert S.plan([10, 1], [500, 1], 100, 8, 100) == 1  # a large head runs alone...
    assert S.plan([10, 1], [50, 1], 100, 8, 100) == 2
    assert S.plan([1, 50, 1], [1, 1, 1], 20, 8, 100) == 1  # ...and the queue is never reordered
    assert S.plan([], [], 100, 8, 100) == 0


def test_admission_simulation(S):
    """Random arrivals and run times; slots take batches by the rule.  The
    estimate in use never exceeds the budget, admission follows arrival
    order, and every request is admitted."""
    rng = np.random.default_rng(7)
    n = 400
    nnz = rng.integers(100, 200000, n)
    nnz[rng.choice(n, 8, replace=False)] = 5_000_000
    rows = np.maximum(nnz // 10, 1)
    est = np.array([S.estimate_bytes(int(r), int(z)) for r, z in zip(rows, nnz)])
    budget = int(est.max() * 1.5)
    arrive = np.cumsum(rng.exponential(0.002, n))
    slots, max_batch, max_nnz = 3, 32, 1_000_000
    t = 0.0
    queue, admitted_order = [], []
    running = []  # (end time, bytes)
    in_use, nxt, peak = 0, 0, 0
    free_slots = slots
    while len(admitted_order) < n:
        # next event: an arrival or a completion
        t_arr = arrive[nxt] if nxt < n else np.inf
        t_end = min(running)[0] if running else np.inf
        t = min(t_arr, t_end)
        if t == t_end:
            running.sort()
            _, b = running.pop(0)
            in_use -= b
            free_slots += 1
        else:
            queue.append(nxt)
            nxt += 1
        while free_slots and queue:
            take = S.plan(est[queue], nnz[queue], budget - in_use, max_batch, max_nnz)
            if take == 0:
                break
            batch, queue = queue[:take], queue[take:]
            admitted_order += batch
            b = int(est[batch].sum())
            in_use += b
            peak = max(peak, in_use)
            free_slots -= 1
            running.append((t + 1e-7 * nnz[batch].sum() + 1e-3, b))
    assert peak <= budget
    assert admitted_order == list(range(n))


def test_default_config(S):
    import ctypes
    from paper_1105_4490_gb300 import vmo
    cfg = vmo._ServerConfig()
    vmo.load().vmo_server_default_config(ctypes.byref(cfg))
    assert (cfg.slots, cfg.max_batch, cfg.max_batch_nnz, cfg.budget_bytes, cfg.sbd) == (4, 256, 8_000_000, 0, 0)
    assert cfg.params.d == 3 and cfg.params.iters == 100
