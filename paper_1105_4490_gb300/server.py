"""Python binding of the request server (vmo_server_* in include/vmo.h).

Requests are host (numpy) patterns; the binding keeps every request's arrays
alive until the request is terminal, as the C-ABI requires, and hands back
the permutation the server wrote into the request's host buffer."""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from .vmo import Params, VmoError, _check, _RequestInfo, _ServerConfig, _ServerStats, load

STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


def estimate_bytes(n: int, nnz: int) -> int:
    """Admission estimate of an n x n request with nnz nonzeros."""
    return int(load().vmo_server_estimate_bytes(n, nnz))


def plan(bytes_, nnz, budget_free: int, max_batch: int, max_batch_nnz: int) -> int:
    """Requests from the head of a queue that the next free slot admits."""
    b = np.ascontiguousarray(bytes_, dtype=np.int64)
    z = np.ascontiguousarray(nnz, dtype=np.int64)
    P64 = C.POINTER(C.c_int64)
    return int(load().vmo_server_plan(b.ctypes.data_as(P64), z.ctypes.data_as(P64), len(b), budget_free, max_batch,
                                      max_batch_nnz))


def _info(ri: _RequestInfo) -> dict:
    d = {f: getattr(ri, f) for f, _ in _RequestInfo._fields_}
    d["state"] = STATES.get(ri.state, "?")
    d["latency"] = ri.t_done - ri.t_submit if ri.state >= 2 else None
    return d


class Server:
    """Continuous-batching ordering server on the current GPU."""

    def __init__(self, params: Params | None = None, sbd: bool = False, slots: int = 4, max_batch: int = 256,
                 max_batch_nnz: int = 8_000_000, budget_bytes: int = 0):
        lib = load()
        cfg = _ServerConfig()
        lib.vmo_server_default_config(C.byref(cfg))
        cfg.params = (params or Params())._c()
        cfg.sbd = int(sbd)
        cfg.slots = slots
        cfg.max_batch = max_batch
        cfg.max_batch_nnz = max_batch_nnz
        cfg.budget_bytes = budget_bytes
        h = C.c_void_p()
        _check(lib.vmo_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._keep: dict[int, tuple] = {}
        self._mu = threading.Lock()

    def submit(self, rowptr, colidx, n: int | None = None) -> int:
        """Queues the pattern (host int32 CSR); returns the request id."""
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colidx, dtype=np.int32)
        n = len(rp) - 1 if n is None else n
        out = np.empty(max(n, 1), dtype=np.int32)
        rid = C.c_uint64()
        _check(load().vmo_server_submit(self._h, n, rp.ctypes.data, ci.ctypes.data if ci.size else None,
                                        out.ctypes.data, C.byref(rid)))
        with self._mu:
            self._keep[rid.value] = (rp, ci, out, n)
        return rid.value

    def submit_matrix(self, A) -> int:
        return self.submit(A.rowptr, A.colidx, A.m)

    def poll(self, rid: int) -> dict:
        ri = _RequestInfo()
        _check(load().vmo_server_poll(self._h, rid, C.byref(ri)))
        return _info(ri)

    def wait(self, rid: int, timeout: float = -1.0) -> dict:
        ri = _RequestInfo()
        st = load().vmo_server_wait(self._h, rid, timeout, C.byref(ri))
        if st not in (0, 4):
            _check(st)
        d = _info(ri)
        d["timed_out"] = st == 4
        return d

    def result(self, rid: int) -> np.ndarray:
        """Permutation of a finished request (perm[new] = old)."""
        d = self.poll(rid)
        if d["state"] != "done":
            raise VmoError(1, f"request {rid} is {d['state']}")
        with self._mu:
            _, _, out, n = self._keep[rid]
        return out[:n].copy()

    def release(self, rid: int) -> bool:
        """Frees a terminal request: the server's record (vmo_server_release)
        and the binding's references to its arrays.  Returns False (nothing
        freed) while the request is queued or running."""
        if self.poll(rid)["state"] not in ("done", "failed", "cancelled"):
            return False
        _check(load().vmo_server_release(self._h, rid))
        with self._mu:
            self._keep.pop(rid, None)
        return True

    def cancel(self, rid: int) -> None:
        _check(load().vmo_server_cancel(self._h, rid))

    def stats(self) -> dict:
        s = _ServerStats()
        _check(load().vmo_server_get_stats(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}

    def close(self) -> None:
        if self._h:
            load().vmo_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
