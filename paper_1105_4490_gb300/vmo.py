"""Python binding of the VMO C-ABI (include/vmo.h).

Argument marshalling only: every step of the method runs in the CUDA library
``libvmo.so``.  PyTorch provides device memory and the current stream.  There
is no CPU fallback; if the library is missing or no GPU is present the calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, fields

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvmo.so")
_lib = None

MODELS = {"symmetric": 0, "bipartite": 1, "rownet": 2, "colnet": 3, "finegrain": 4}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "device wait timed out",
          5: "over admission budget", 6: "unsupported"}


class VmoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"vmo status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class _Csr(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colidx", C.c_void_p)]


class _HostCsr(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colidx", C.c_void_p), ("values", C.c_void_p)]


class _Tuning(C.Structure):
    _fields_ = [("small_step_threads", C.c_int64), ("radix_max_bits", C.c_int32), ("assign_items", C.c_int32),
                ("small_bin_points", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("d", C.c_int32), ("iters", C.c_int32), ("sigma", C.c_float), ("decay", C.c_float),
                ("occupancy", C.c_int32), ("multilevel", C.c_int32), ("match_rounds", C.c_int32),
                ("coarse_min", C.c_int32), ("km_iters", C.c_int32), ("min_part", C.c_int32),
                ("max_depth", C.c_int32), ("sep_recursion", C.c_int32), ("cut_order", C.c_int32),
                ("sep_order_free", C.c_int32),
                ("seed", C.c_uint64)]


class _Tree(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("count", C.c_int32), ("heap", C.c_void_p), ("offset", C.c_void_p),
                ("n1", C.c_void_p), ("n2", C.c_void_p), ("nsep", C.c_void_p), ("depth", C.c_void_p),
                ("component", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("step_launches", C.c_uint64), ("step_ms", C.c_double),
                ("step_points", C.c_uint64), ("step_interactions", C.c_uint64), ("device_allocations", C.c_uint64)]


@dataclass
class Params:
    """Method parameters (defaults of vmo_default_params)."""

    d: int = 3
    iters: int = 100
    sigma: float = 1.0
    decay: float = 0.9
    occupancy: int = 8
    multilevel: int = 1
    match_rounds: int = 4
    coarse_min: int = 64
    km_iters: int = 20
    min_part: int = 64
    max_depth: int = 62
    sep_recursion: int = 0
    cut_order: int = 0
    sep_order_free: int = 0
    seed: int = 1

    def _c(self) -> _Params:
        p = _Params()
        for f in fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


SYMBOLS = ["vmo_default_params", "vmo_build_hypergraph", "vmo_hg_vertices", "vmo_hg_nets", "vmo_hg_arrays",
           "vmo_components", "vmo_init_coords", "vmo_layout", "vmo_layout_step", "vmo_coarsen",
           "vmo_hierarchy_level", "vmo_hierarchy_prolong", "vmo_hierarchy_step", "vmo_bisect",
           "vmo_order_bbd", "vmo_order_sbd", "vmo_order_vertices", "vmo_order_matched", "vmo_perfect_matching_host", "vmo_read_matrix_market",
           "vmo_write_matrix_market", "vmo_free_host_csr", "vmo_finegrain_coords", "vmo_get_tuning",
           "vmo_set_tuning",
           "vmo_autotune", "vmo_cut_size", "vmo_destroy",
           "vmo_status_string", "vmo_last_error", "vmo_stats_reset", "vmo_stats_get", "vmo_batch_order",
           "vmo_batch_layout", "vmo_bisect_noalloc", "vmo_server_default_config", "vmo_server_estimate_bytes",
           "vmo_server_plan", "vmo_server_create", "vmo_server_submit", "vmo_server_poll", "vmo_server_wait",
           "vmo_server_cancel", "vmo_server_release", "vmo_server_get_stats", "vmo_server_destroy", "vmo_kmeans",
           "vmo_measure_alu_peaks"]


class _ServerConfig(C.Structure):
    _fields_ = [("params", _Params), ("sbd", C.c_int32), ("slots", C.c_int32), ("max_batch", C.c_int32),
                ("max_batch_nnz", C.c_int64), ("budget_bytes", C.c_int64)]


class _RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("n", C.c_int64), ("nnz", C.c_int64),
                ("bytes", C.c_int64), ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("batch", C.c_int64), ("batch_size", C.c_int32), ("slot", C.c_int32)]


class _ServerStats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("submitted", "completed", "failed", "cancelled", "queued", "running",
                                         "batches", "nnz_completed", "budget_bytes", "bytes_in_use", "bytes_peak",
                                         "pool_peak_bytes")]


def load(path: str | None = None):
    """Loads libvmo.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} not found: build the CUDA library first (python -m paper_1105_4490_gb300._build_lib)")
    lib = C.CDLL(p)
    V, I32, I64, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    P32, P64 = C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    lib.vmo_default_params.argtypes = [C.POINTER(_Params)]
    lib.vmo_default_params.restype = None
    lib.vmo_build_hypergraph.argtypes = [C.POINTER(_Csr), C.c_int, V, V, C.POINTER(V)]
    lib.vmo_hg_vertices.argtypes = [V]
    lib.vmo_hg_vertices.restype = I32
    lib.vmo_hg_nets.argtypes = [V]
    lib.vmo_hg_nets.restype = I64
    lib.vmo_hg_arrays.argtypes = [V, C.POINTER(V), C.POINTER(V), P64, C.POINTER(V), C.POINTER(V), P64,
                                  C.POINTER(V), C.POINTER(V), P64]
    lib.vmo_components.argtypes = [V, V, V]
    lib.vmo_init_coords.argtypes = [I32, I32, U64, V, V]
    lib.vmo_layout.argtypes = [V, C.POINTER(_Params), V, I32, V]
    lib.vmo_layout_step.argtypes = [V, C.POINTER(_Params), V, C.c_float, V, V, P32, V]
    lib.vmo_coarsen.argtypes = [V, C.POINTER(_Params), V, V, P32, P32, P32, V]
    lib.vmo_hierarchy_level.argtypes = [V, C.POINTER(_Params), I32, P32, P64, V, V, V, V, V, V]
    lib.vmo_hierarchy_prolong.argtypes = [V, C.POINTER(_Params), I32, V, V, V]
    lib.vmo_hierarchy_step.argtypes = [V, C.POINTER(_Params), I32, V, C.c_float, V, V]
    lib.vmo_bisect.argtypes = [V, I32, V, V, I32, U64, U64, I32, V, V, P32, V]
    lib.vmo_bisect_noalloc.argtypes = [I32, V, V, I32, U64, U64, I32, V, V, P32, V]
    lib.vmo_kmeans.argtypes = [I32, V, V, I32, I32, U64, U64, I32, V, V, P32, V]
    for nm in ("vmo_order_bbd", "vmo_order_sbd"):
        getattr(lib, nm).argtypes = [V, V, C.POINTER(_Params), V, V, C.POINTER(_Tree), V]
    lib.vmo_order_vertices.argtypes = [V, V, C.POINTER(_Params), I32, V, C.POINTER(_Tree), V]
    lib.vmo_order_matched.argtypes = [V, V, C.POINTER(_Params), I32, V, V, V, V, C.POINTER(_Tree), V]
    lib.vmo_finegrain_coords.argtypes = [V, V, V, V]
    lib.vmo_perfect_matching_host.argtypes = [I32, V, V, V, V, C.POINTER(I32)]
    lib.vmo_read_matrix_market.argtypes = [C.c_char_p, I32, C.POINTER(_HostCsr)]
    lib.vmo_write_matrix_market.argtypes = [C.c_char_p, C.POINTER(_HostCsr), I32]
    lib.vmo_free_host_csr.argtypes = [C.POINTER(_HostCsr)]
    lib.vmo_free_host_csr.restype = None
    lib.vmo_get_tuning.argtypes = [C.POINTER(_Tuning)]
    lib.vmo_get_tuning.restype = None
    lib.vmo_set_tuning.argtypes = [C.POINTER(_Tuning)]
    lib.vmo_autotune.argtypes = [C.POINTER(_Csr), I32, C.POINTER(_Params), I32, C.POINTER(_Tuning),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), V]
    lib.vmo_cut_size.argtypes = [V, V, I32, P64, P64, V]
    lib.vmo_batch_order.argtypes = [C.POINTER(_Csr), I32, V, C.POINTER(_Params), I32, V, V]
    lib.vmo_batch_layout.argtypes = [C.POINTER(_Csr), I32, C.POINTER(_Params), V, V]
    lib.vmo_destroy.argtypes = [V]
    lib.vmo_destroy.restype = None
    lib.vmo_status_string.argtypes = [C.c_int]
    lib.vmo_status_string.restype = C.c_char_p
    lib.vmo_last_error.argtypes = []
    lib.vmo_last_error.restype = C.c_char_p
    lib.vmo_stats_reset.argtypes = [I32, I32]
    lib.vmo_stats_reset.restype = None
    lib.vmo_stats_get.argtypes = [C.POINTER(_Stats)]
    lib.vmo_server_default_config.argtypes = [C.POINTER(_ServerConfig)]
    lib.vmo_server_default_config.restype = None
    lib.vmo_server_estimate_bytes.argtypes = [I64, I64]
    lib.vmo_server_estimate_bytes.restype = I64
    lib.vmo_server_plan.argtypes = [P64, P64, I32, I64, I32, I64]
    lib.vmo_server_plan.restype = I32
    lib.vmo_server_create.argtypes = [C.POINTER(_ServerConfig), C.POINTER(V)]
    lib.vmo_server_submit.argtypes = [V, I32, V, V, V, C.POINTER(U64)]
    lib.vmo_server_poll.argtypes = [V, U64, C.POINTER(_RequestInfo)]
    lib.vmo_server_wait.argtypes = [V, U64, C.c_double, C.POINTER(_RequestInfo)]
    lib.vmo_server_cancel.argtypes = [V, U64]
    lib.vmo_server_release.argtypes = [V, U64]
    D = C.POINTER(C.c_double)
    lib.vmo_measure_alu_peaks.argtypes = [D, D, D, P32, V]
    lib.vmo_server_get_stats.argtypes = [V, C.POINTER(_ServerStats)]
    lib.vmo_server_destroy.argtypes = [V]
    lib.vmo_server_destroy.restype = None
    for nm in SYMBOLS:
        if nm not in ("vmo_default_params", "vmo_hg_vertices", "vmo_hg_nets", "vmo_destroy", "vmo_status_string",
                      "vmo_last_error", "vmo_stats_reset", "vmo_server_default_config", "vmo_server_estimate_bytes",
                      "vmo_server_plan", "vmo_server_destroy", "vmo_get_tuning", "vmo_free_host_csr"):
            getattr(lib, nm).restype = C.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise VmoError(status, load().vmo_last_error().decode())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


class _View:
    """Zero-copy view of a device array owned by the library."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


def default_params() -> Params:
    p = _Params()
    load().vmo_default_params(C.byref(p))
    return Params(**{f.name: getattr(p, f.name) for f in fields(Params)})


def init_coords(k: int, d: int, seed: int) -> torch.Tensor:
    """Random initial layout of Algorithm 3 (fp32 [k, 4])."""
    x = torch.zeros((k, 4), dtype=torch.float32, device="cuda")
    _check(load().vmo_init_coords(k, d, seed & (2 ** 64 - 1), _ptr(x), _stream()))
    return x


class Hypergraph:
    """Device hypergraph model of a sparsity pattern (Table 1)."""

    def __init__(self, rowptr: torch.Tensor, colidx: torch.Tensor, m: int, n: int, model: str = "symmetric",
                 weights: torch.Tensor | None = None):
        lib = load()
        rowptr = rowptr.to(device="cuda", dtype=torch.int32).contiguous()
        colidx = colidx.to(device="cuda", dtype=torch.int32).contiguous()
        csr = _Csr(m, n, colidx.numel(), rowptr.data_ptr(), colidx.data_ptr() if colidx.numel() else None)
        self._h = C.c_void_p()
        w = None if weights is None else weights.to(device="cuda", dtype=torch.float32).contiguous()
        _check(lib.vmo_build_hypergraph(C.byref(csr), MODELS[model], _ptr(w), _stream(), C.byref(self._h)))
        self.model = model
        self.m, self.n = m, n
        self.k = int(lib.vmo_hg_vertices(self._h))
        self.nets = int(lib.vmo_hg_nets(self._h))

    @classmethod
    def from_matrix(cls, mat, model: str = "symmetric", weights=None) -> "Hypergraph":
        return cls(torch.as_tensor(mat.rowptr), torch.as_tensor(mat.colidx), mat.m, mat.n, model, weights)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.vmo_destroy(self._h)
            self._h = None

    def arrays(self) -> dict:
        """Copies of the model's device arrays (torch int32 tensors)."""
        ptrs = [C.c_void_p() for _ in range(6)]
        cnt = [C.c_int64() for _ in range(3)]
        _check(load().vmo_hg_arrays(self._h, C.byref(ptrs[0]), C.byref(ptrs[1]), C.byref(cnt[0]), C.byref(ptrs[2]),
                                    C.byref(ptrs[3]), C.byref(cnt[1]), C.byref(ptrs[4]), C.byref(ptrs[5]),
                                    C.byref(cnt[2])))
        torch.cuda.current_stream().synchronize()

        def view(p, n):
            if not p.value or n == 0:
                return torch.zeros(0, dtype=torch.int32, device="cuda")
            return torch.as_tensor(_View(p.value, n, "<i4"), device="cuda").clone()

        out = {"net_ptr": view(ptrs[2], self.nets + 1), "pins": view(ptrs[3], cnt[1].value),
               "vtx_ptr": view(ptrs[4], self.k + 1), "vnets": view(ptrs[5], cnt[2].value)}
        if self.model in ("symmetric", "bipartite"):
            out["adj_ptr"] = view(ptrs[0], self.k + 1)
            out["adj"] = view(ptrs[1], cnt[0].value)
        return out

    def components(self) -> torch.Tensor:
        lab = torch.empty(self.k, dtype=torch.int32, device="cuda")
        _check(load().vmo_components(self._h, _ptr(lab), _stream()))
        return lab

    def layout(self, params: Params | None = None, coords: torch.Tensor | None = None) -> torch.Tensor:
        """Geometry of Sec. 2: fp32 [k, 4] coordinates."""
        p = (params or Params())._c()
        x = coords if coords is not None else torch.zeros((self.k, 4), dtype=torch.float32, device="cuda")
        _check(load().vmo_layout(self._h, C.byref(p), _ptr(x), int(coords is not None), _stream()))
        return x

    def layout_step(self, coords: torch.Tensor, step: float, params: Params | None = None):
        """One step of Algorithm 4: (new coords, gradient y, level-L keys, L)."""
        p = (params or Params())._c()
        x = coords.clone().contiguous()
        y = torch.zeros_like(x)
        keys = torch.zeros(self.k, dtype=torch.int32, device="cuda")
        L = C.c_int32()
        _check(load().vmo_layout_step(self._h, C.byref(p), _ptr(x), step, _ptr(y), _ptr(keys), C.byref(L), _stream()))
        return x, y, keys, int(L.value)

    def coarsen(self, params: Params | None = None):
        """Level-0 matching (mate, pi, kc) and the sizes of all levels."""
        p = (params or Params())._c()
        mate = torch.empty(self.k, dtype=torch.int32, device="cuda")
        pi = torch.empty(self.k, dtype=torch.int32, device="cuda")
        kc = C.c_int32()
        sizes = (C.c_int32 * 41)()
        nl = C.c_int32()
        _check(load().vmo_coarsen(self._h, C.byref(p), _ptr(mate), _ptr(pi), C.byref(kc), sizes, C.byref(nl),
                                  _stream()))
        return mate, pi, int(kc.value), [int(sizes[i]) for i in range(nl.value)]

    def hierarchy_level(self, level: int, params: Params | None = None) -> dict:
        """Level `level` of the coarsening hierarchy of Algorithm 3: dict with
        k, adj_ptr, adj, acost (edge costs), weight (vertex weights) and pi
        (level-1 vertex -> level vertex; None for level 0), device tensors."""
        p = (params or Params())._c()
        lib = load()
        k, nadj = C.c_int32(), C.c_int64()
        _check(lib.vmo_hierarchy_level(self._h, C.byref(p), level, C.byref(k), C.byref(nadj), None, None, None, None,
                                       None, _stream()))
        k, nadj = int(k.value), int(nadj.value)
        kf = None
        if level > 0:
            kf_c = C.c_int32()
            _check(lib.vmo_hierarchy_level(self._h, C.byref(p), level - 1, C.byref(kf_c), None, None, None, None, None,
                                           None, _stream()))
            kf = int(kf_c.value)
        out = {"k": k, "adj_ptr": torch.empty(k + 1, dtype=torch.int32, device="cuda"),
               "adj": torch.empty(max(nadj, 1), dtype=torch.int32, device="cuda"),
               "acost": torch.empty(max(nadj, 1), dtype=torch.float32, device="cuda"),
               "weight": torch.empty(max(k, 1), dtype=torch.float32, device="cuda"),
               "pi": torch.empty(max(kf, 1), dtype=torch.int32, device="cuda") if kf is not None else None}
        _check(lib.vmo_hierarchy_level(self._h, C.byref(p), level, None, None, _ptr(out["adj_ptr"]), _ptr(out["adj"]),
                                       _ptr(out["acost"]), _ptr(out["weight"]), _ptr(out["pi"]), _stream()))
        out["adj"], out["acost"], out["weight"] = out["adj"][:nadj], out["acost"][:nadj], out["weight"][:k]
        if kf is not None:
            out["pi"] = out["pi"][:kf]
        return out

    def hierarchy_prolong(self, level: int, coarse: torch.Tensor, kf: int, params: Params | None = None):
        """Prolongation of Algorithm 3 from `level` to level - 1 (kf points)."""
        p = (params or Params())._c()
        fine = torch.empty((max(kf, 1), 4), dtype=torch.float32, device="cuda")
        _check(load().vmo_hierarchy_prolong(self._h, C.byref(p), level, _ptr(coarse.contiguous()), _ptr(fine),
                                            _stream()))
        return fine[:kf]

    def hierarchy_step(self, level: int, coords: torch.Tensor, step: float, params: Params | None = None):
        """One step of Algorithm 4 on a level of the hierarchy: (new coords, y)."""
        p = (params or Params())._c()
        x = coords.clone().contiguous()
        y = torch.zeros_like(x)
        _check(load().vmo_hierarchy_step(self._h, C.byref(p), level, _ptr(x), step, _ptr(y), _stream()))
        return x, y

    def bisect(self, coords: torch.Tensor, verts: torch.Tensor, seed: int, key: int = 1, km_iters: int = 20,
               d: int = 3):
        """2-means of coords[verts] (Algorithm 5, m = 2): (split, labels, z1, z2)."""
        verts = verts.to(device="cuda", dtype=torch.int32).contiguous()
        labels = torch.zeros(verts.numel(), dtype=torch.uint8, device="cuda")
        z = torch.zeros(8, dtype=torch.float32, device="cuda")
        split = C.c_int32()
        _check(load().vmo_bisect(self._h, d, _ptr(coords), _ptr(verts), verts.numel(), seed & (2 ** 64 - 1), key,
                                 km_iters, _ptr(labels), _ptr(z), C.byref(split), _stream()))
        return bool(split.value), labels, z[:4], z[4:]

    def _tree(self, cap: int):
        t = {"heap": torch.zeros(cap, dtype=torch.int64, device="cuda")}
        for f in ("offset", "n1", "n2", "nsep", "depth", "comp"):
            t[f] = torch.zeros(cap, dtype=torch.int32, device="cuda")
        ct = _Tree(cap, 0, *(t[f].data_ptr() for f in ("heap", "offset", "n1", "n2", "nsep", "depth", "comp")))
        return t, ct

    def order(self, params: Params | None = None, coords: torch.Tensor | None = None, sbd: bool = False,
              with_tree: bool = True):
        """Recursive BBD (or SBD) ordering: (row_perm, col_perm, tree)."""
        p = (params or Params())._c()
        rows = self.m
        cols = self.n if self.model == "bipartite" else self.m
        rp = torch.empty(rows, dtype=torch.int32, device="cuda")
        cp = torch.empty(cols, dtype=torch.int32, device="cuda")
        t, ct = self._tree(2 * self.k + 16) if with_tree else (None, None)
        fn = load().vmo_order_sbd if sbd else load().vmo_order_bbd
        _check(fn(self._h, _ptr(coords), C.byref(p), _ptr(rp), _ptr(cp), C.byref(ct) if ct else None, _stream()))
        tree = {f: v[:ct.count] for f, v in t.items()} if t else None
        return rp, cp, tree

    def order_vertices(self, params: Params | None = None, coords: torch.Tensor | None = None, sbd: bool = False):
        """Vertex permutation of the recursive ordering and its tree."""
        p = (params or Params())._c()
        perm = torch.empty(self.k, dtype=torch.int32, device="cuda")
        t, ct = self._tree(2 * self.k + 16)
        _check(load().vmo_order_vertices(self._h, _ptr(coords), C.byref(p), int(sbd), _ptr(perm), C.byref(ct),
                                         _stream()))
        return perm, {f: v[:ct.count] for f, v in t.items()}

    def order_matched(self, match: torch.Tensor, params: Params | None = None, coords: torch.Tensor | None = None,
                      sbd: bool = False):
        """Ordering that keeps a strengthened diagonal (bipartite model of a
        square pattern; match[i] = column matched to row i):
        (row_perm, col_perm, vertex_perm, tree), col_perm = match[row_perm]."""
        p = (params or Params())._c()
        match = torch.as_tensor(match).to(device="cuda", dtype=torch.int32).contiguous()
        rp = torch.empty(self.m, dtype=torch.int32, device="cuda")
        cp = torch.empty(self.m, dtype=torch.int32, device="cuda")
        vp = torch.empty(self.k, dtype=torch.int32, device="cuda")
        t, ct = self._tree(2 * self.k + 16)
        _check(load().vmo_order_matched(self._h, _ptr(coords), C.byref(p), int(sbd), _ptr(match), _ptr(rp), _ptr(cp),
                                        _ptr(vp), C.byref(ct), _stream()))
        return rp, cp, vp, {f: v[:ct.count] for f, v in t.items()}

    def finegrain_coords(self, bipartite_coords: torch.Tensor) -> torch.Tensor:
        """Finegrain layout from the bipartite model's coordinates (this
        handle: the finegrain model): every entry at the mean of its row's and
        its column's points (k x 4 on the device)."""
        xb = bipartite_coords.to(device="cuda", dtype=torch.float32).contiguous()
        out = torch.empty((self.k, 4), dtype=torch.float32, device="cuda")
        _check(load().vmo_finegrain_coords(self._h, _ptr(xb), _ptr(out), _stream()))
        return out

    def cut_size(self, part: torch.Tensor, nparts: int):
        """(cut-net count, lambda - 1) of a vertex partition over the nets."""
        part = part.to(device="cuda", dtype=torch.int32).contiguous()
        a, b = C.c_int64(), C.c_int64()
        _check(load().vmo_cut_size(self._h, _ptr(part), nparts, C.byref(a), C.byref(b), _stream()))
        return int(a.value), int(b.value)


def stats_reset(time_step_kernel: bool = False, count_interactions: bool = False) -> None:
    """Resets the library's launch counter and step-kernel instrumentation."""
    load().vmo_stats_reset(int(time_step_kernel), int(count_interactions))


def stats() -> dict:
    """Launches since the last reset; step-kernel time (ms), launches, points and
    interactions when enabled."""
    s = _Stats()
    _check(load().vmo_stats_get(C.byref(s)))
    return {f: getattr(s, f) for f, _ in _Stats._fields_}


def _csr_array(mats):
    keep = []
    arr = (_Csr * max(len(mats), 1))()
    offs = [0]
    for i, mt in enumerate(mats):
        if isinstance(mt, tuple):
            rp, ci, m = mt
            n = m
        else:
            rp, ci, m, n = torch.as_tensor(mt.rowptr), torch.as_tensor(mt.colidx), mt.m, mt.n
        rp = rp.to(device="cuda", dtype=torch.int32).contiguous()
        ci = ci.to(device="cuda", dtype=torch.int32).contiguous()
        keep += [rp, ci]
        arr[i] = _Csr(m, n, ci.numel(), rp.data_ptr(), ci.data_ptr() if ci.numel() else None)
        offs.append(offs[-1] + m)
    return arr, offs, keep


def batch_layout(mats, params: Params | None = None):
    """Geometry of many square patterns in one batch: float32 [sum m, 4] and offsets."""
    arr, offs, keep = _csr_array(mats)
    x = torch.zeros((max(offs[-1], 1), 4), dtype=torch.float32, device="cuda")
    p = (params or Params())._c()
    _check(load().vmo_batch_layout(arr, len(mats), C.byref(p), _ptr(x), _stream()))
    return x[:offs[-1]], offs


def batch_order(mats, params: Params | None = None, sbd: bool = False, coords: torch.Tensor | None = None):
    """Orders many square patterns in one batch (vmo_batch_order).

    mats: list of (rowptr, colidx, m) with int32 tensors on the GPU (or objects
    with .rowptr/.colidx/.m numpy arrays, copied to the GPU).  Returns the
    concatenated permutation tensor and the list of offsets (len(mats) + 1).
    coords: optional float32 [sum m, 4] coordinates (ordering only)."""
    arr, offs, keep = _csr_array(mats)
    perm = torch.empty(max(offs[-1], 1), dtype=torch.int32, device="cuda")
    p = (params or Params())._c()
    _check(load().vmo_batch_order(arr, len(mats), _ptr(coords), C.byref(p), int(sbd), _ptr(perm), _stream()))
    return perm[:offs[-1]], offs


class HostMatrix:
    """A host CSR pattern with values (row-major, sorted columns), as read from
    a Matrix Market file; accepted wherever a matrix with .m, .n, .rowptr and
    .colidx is (Hypergraph.from_matrix, perfect_matching, batch_order)."""

    def __init__(self, name, m, n, rowptr, colidx, values):
        self.name, self.m, self.n = name, m, n
        self.rowptr, self.colidx, self.values = rowptr, colidx, values

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def read_matrix_market(path: str, expand_symmetric: bool = True) -> HostMatrix:
    """vmo_read_matrix_market: a coordinate Matrix Market file as a HostMatrix
    (duplicates summed; symmetric storage expanded to both triangles unless
    expand_symmetric is False)."""
    import numpy as np
    c = _HostCsr()
    _check(load().vmo_read_matrix_market(os.fsencode(path), int(expand_symmetric), C.byref(c)))
    try:
        def arr(p, n, dt):
            return np.ctypeslib.as_array(C.cast(p, C.POINTER(dt)), shape=(n,)).copy() if n else \
                np.zeros(0, dtype=np.dtype(dt))
        rp = arr(c.rowptr, c.m + 1, C.c_int32)
        ci = arr(c.colidx, c.nnz, C.c_int32)
        vv = arr(c.values, c.nnz, C.c_float)
        return HostMatrix(os.path.basename(path), c.m, c.n, rp, ci, vv)
    finally:
        load().vmo_free_host_csr(C.byref(c))


def write_matrix_market(path: str, mat, values=None) -> None:
    """vmo_write_matrix_market: a general coordinate file of the pattern (and
    the values, if given or present on the matrix)."""
    import numpy as np
    rp = np.ascontiguousarray(mat.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(mat.colidx, dtype=np.int32)
    if values is None:
        values = getattr(mat, "values", None)
        if callable(values):
            values = values()
    vv = None if values is None else np.ascontiguousarray(values, dtype=np.float32)
    c = _HostCsr(mat.m, mat.n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data if ci.size else None,
                 vv.ctypes.data if vv is not None and vv.size else None)
    _check(load().vmo_write_matrix_market(os.fsencode(path), C.byref(c), int(vv is None)))


def perfect_matching(mat, values=None):
    """vmo_perfect_matching_host: a strengthened diagonal for order_matched
    (heavy-edge start from |values|, Hopcroft-Karp augmentation) of a square
    host pattern (object with .m, .rowptr, .colidx numpy arrays).  Returns
    (match int32 numpy [m], matched); raises VmoError when no perfect
    matching exists."""
    import numpy as np
    rp = np.ascontiguousarray(mat.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(mat.colidx, dtype=np.int32)
    vv = None if values is None else np.ascontiguousarray(values, dtype=np.float32)
    match = np.empty(max(mat.m, 1), dtype=np.int32)
    got = C.c_int32(0)
    st = load().vmo_perfect_matching_host(mat.m, rp.ctypes.data, ci.ctypes.data if ci.size else None,
                                          vv.ctypes.data if vv is not None else None, match.ctypes.data,
                                          C.byref(got))
    _check(st)
    return match[:mat.m], int(got.value)


def get_tuning() -> dict:
    """The launch-shape setting (vmo_get_tuning): none of it changes a result."""
    t = _Tuning()
    load().vmo_get_tuning(C.byref(t))
    return {f: getattr(t, f) for f, _ in _Tuning._fields_}


def set_tuning(small_step_threads: int, radix_max_bits: int, assign_items: int, small_bin_points: int = 2048) -> None:
    """vmo_set_tuning: all four choices at once."""
    t = _Tuning(small_step_threads, radix_max_bits, assign_items, small_bin_points)
    _check(load().vmo_set_tuning(C.byref(t)))


def autotune(mats, params: Params | None = None, reps: int = 3):
    """vmo_autotune: timed search over the launch shapes on these matrices
    (as for batch_order); sets and returns (setting, best_ms, default_ms)."""
    arr, offs, keep = _csr_array(mats)
    p = (params or Params())._c()
    t = _Tuning()
    b, dflt = C.c_double(), C.c_double()
    _check(load().vmo_autotune(arr, len(mats), C.byref(p), reps, C.byref(t), C.byref(b), C.byref(dflt), _stream()))
    return {f: getattr(t, f) for f, _ in _Tuning._fields_}, b.value, dflt.value


def bisect_noalloc(coords: torch.Tensor, verts: torch.Tensor, seed: int, key: int = 1, km_iters: int = 20,
                   d: int = 3):
    """vmo_bisect_noalloc: 2-means of coords[verts] without any device
    allocation inside the library (fixed scratch, at most 131072 points).
    Returns (split, labels, z1, z2); the output tensors are allocated here,
    by the caller side."""
    verts = verts.to(device="cuda", dtype=torch.int32).contiguous()
    labels = torch.zeros(max(verts.numel(), 1), dtype=torch.uint8, device="cuda")
    z = torch.zeros(8, dtype=torch.float32, device="cuda")
    split = C.c_int32()
    _check(load().vmo_bisect_noalloc(d, _ptr(coords), _ptr(verts), verts.numel(), seed & (2 ** 64 - 1), key,
                                     km_iters, _ptr(labels), _ptr(z), C.byref(split), _stream()))
    return bool(split.value), labels[:verts.numel()], z[:4], z[4:]


def kmeans(coords: torch.Tensor, verts: torch.Tensor, m: int, seed: int, key: int = 1, km_iters: int = 20,
           d: int = 3):
    """m-way k-means++ of coords[verts] (Algorithm 5): (labels in [0, m),
    centres [m, 4], number of non-empty clusters)."""
    verts = verts.to(device="cuda", dtype=torch.int32).contiguous()
    labels = torch.zeros(max(verts.numel(), 1), dtype=torch.int32, device="cuda")
    centres = torch.zeros((max(m, 1), 4), dtype=torch.float32, device="cuda")
    ne = C.c_int32()
    _check(load().vmo_kmeans(d, _ptr(coords), _ptr(verts), verts.numel(), m, seed & (2 ** 64 - 1),
                             key & (2 ** 64 - 1), km_iters, _ptr(labels), _ptr(centres), C.byref(ne), _stream()))
    return labels[:verts.numel()], centres[:m], int(ne.value)


def measure_alu_peaks() -> dict:
    """vmo_measure_alu_peaks: measured FP32 fma / packed fma2 TFLOP/s, the
    reciprocal square root rate (T/s) and the SM count of the current GPU."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int32()
    _check(load().vmo_measure_alu_peaks(C.byref(a), C.byref(b), C.byref(c), C.byref(n), _stream()))
    return {"ffma_tflops": a.value, "ffma2_tflops": b.value, "rsqrt_tops": c.value, "sms": int(n.value)}
