"""CPU oracle for visual matrix ordering (VMO) — TEST INFRASTRUCTURE ONLY.

A thin ctypes wrapper around ``vmo_oracle.c``, the plain FP64 restatement of
the method of Fagginger Auer and Bisseling, "A Geometric Approach to Matrix
Ordering".  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the GPU library never calls it.
It shares no code with the CUDA path; the two meet only through the seeded
input generators in ``workloads``.

Functions without an independent pin are marked "parity unpinned" in their
docstring; every other function is checked in ``tests/test_oracle_*.py``
against closed forms, brute force or the paper's worked examples.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vmo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libvmo_oracle.so")
_lock = threading.Lock()
_lib = None

MODELS = {"symmetric": 0, "bipartite": 1, "rownet": 2, "colnet": 3, "finegrain": 4}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE semantics; OpenMP
    over the per-vertex gradient loop when the compiler has it)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", tmp,
                _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _HG(C.Structure):
    _fields_ = [("model", C.c_int32), ("k", C.c_int32), ("l", C.c_int32),
                ("net_ptr", C.POINTER(C.c_int32)), ("pins", C.POINTER(C.c_int32)),
                ("vtx_ptr", C.POINTER(C.c_int32)), ("vnets", C.POINTER(C.c_int32)),
                ("adj_ptr", C.POINTER(C.c_int32)), ("adj", C.POINTER(C.c_int32))]


class _Tree(C.Structure):
    _fields_ = [("count", C.c_int32), ("heap", C.POINTER(C.c_uint64)),
                ("offset", C.POINTER(C.c_int32)), ("n1", C.POINTER(C.c_int32)),
                ("n2", C.POINTER(C.c_int32)), ("nsep", C.POINTER(C.c_int32)),
                ("depth", C.POINTER(C.c_int32)), ("comp", C.POINTER(C.c_int32))]


class _Diag(C.Structure):
    _fields_ = [("n_inter", C.POINTER(C.c_int64)), ("w_seen", C.POINTER(C.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.ora_set_threads.restype = None
            lib.ora_set_threads.argtypes = [C.c_int32]
            lib.ora_get_threads.restype = C.c_int32
            lib.ora_get_threads.argtypes = []
            lib.ora_rand64.restype = C.c_uint64
            lib.ora_rand64.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
            lib.ora_build.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, P, C.POINTER(_HG)]
            lib.ora_hg_free.argtypes = [C.POINTER(_HG)]
            lib.ora_dual.argtypes = [C.c_int32, C.c_int32, P, P, C.POINTER(C.POINTER(C.c_int32)),
                                     C.POINTER(C.POINTER(C.c_int32))]
            lib.ora_free.argtypes = [P]
            lib.ora_components.argtypes = [C.c_int32, C.c_int32, P, P, P]
            lib.ora_init_side.restype = C.c_int32
            lib.ora_init_side.argtypes = [C.c_int32, C.c_int32]
            lib.ora_init_coords.argtypes = [C.c_int32, C.c_int32, C.c_uint64, P]
            lib.ora_levels.restype = C.c_int32
            lib.ora_levels.argtypes = [C.c_int32, C.c_int32, C.c_int32]
            lib.ora_energy.restype = C.c_double
            lib.ora_energy.argtypes = [C.POINTER(_HG), C.c_int32, P, P, P]
            lib.ora_gradient.argtypes = [C.POINTER(_HG), C.c_int32, C.c_int32, P, P, P, P, P,
                                         C.POINTER(C.c_int32), C.POINTER(_Diag)]
            lib.ora_step0.restype = C.c_double
            lib.ora_step0.argtypes = [C.c_int32, C.c_int32, C.c_double, P]
            lib.ora_layout_step.argtypes = [C.POINTER(_HG), C.c_int32, C.c_int32, P, P, P, C.c_double, P, P,
                                            C.POINTER(C.c_int32)]
            lib.ora_layout.argtypes = [C.POINTER(_HG), C.c_int32, C.c_int32, C.c_double, C.c_double,
                                       C.c_int32, P, P, P]
            lib.ora_match.restype = C.c_int32
            lib.ora_match.argtypes = [C.c_int32, P, P, P, C.c_uint64, C.c_int32, C.c_int32, P, P]
            lib.ora_hierarchy.restype = C.c_int32
            lib.ora_hierarchy.argtypes = [C.POINTER(_HG), C.c_uint64, C.c_int32, C.c_int32, P]
            lib.ora_hierarchy_level.restype = C.c_int32
            lib.ora_hierarchy_level.argtypes = [C.POINTER(_HG), P, C.c_uint64, C.c_int32, C.c_int32, C.c_int32,
                                                C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                                C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.POINTER(C.c_int32)),
                                                C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.POINTER(C.c_double)),
                                                C.POINTER(C.POINTER(C.c_int32))]
            lib.ora_prolong.restype = None
            lib.ora_prolong.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, P, P, P]
            lib.ora_layout_multilevel.restype = C.c_int
            lib.ora_layout_multilevel.argtypes = [C.POINTER(_HG), C.c_int32, C.c_int32, C.c_double, C.c_double,
                                                  C.c_int32, C.c_uint64, C.c_int32, C.c_int32, P, P]
            lib.ora_bisect.restype = C.c_int
            lib.ora_bisect.argtypes = [C.c_int32, P, P, C.c_int32, C.c_uint64, C.c_uint64, C.c_int32,
                                       P, P, P]
            lib.ora_order.argtypes = [C.POINTER(_HG), C.c_int32, P, C.c_uint64, C.c_int32, C.c_int32,
                                      C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, C.c_int32, P,
                                      C.POINTER(_Tree)]
            lib.ora_tree_free.argtypes = [C.POINTER(_Tree)]
            lib.ora_finegrain_coords.argtypes = [C.POINTER(_HG), P, P]
            lib.ora_kmeans.argtypes = [C.c_int32, P, P, C.c_int32, C.c_int32, C.c_uint64, C.c_uint64, C.c_int32,
                                       P, P]
            lib.ora_kmeans.restype = C.c_int32
            lib.ora_cut_size.argtypes = [C.c_int32, P, P, P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            lib.ora_cholesky_nnz.restype = C.c_int64
            lib.ora_cholesky_nnz.argtypes = [C.c_int32, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


@dataclass
class Hypergraph:
    """Oracle hypergraph: nets (net_ptr/pins), incidence (vtx_ptr/vnets) and, for
    graph models, the vertex adjacency (adj_ptr/adj); all lists ascending."""

    model: int
    k: int
    l: int
    net_ptr: np.ndarray
    pins: np.ndarray
    vtx_ptr: np.ndarray
    vnets: np.ndarray
    adj_ptr: np.ndarray | None
    adj: np.ndarray | None

    def _struct(self) -> _HG:
        s = _HG()
        s.model, s.k, s.l = self.model, self.k, self.l
        self._keep = [np.ascontiguousarray(a, dtype=np.int32) if a is not None else None
                      for a in (self.net_ptr, self.pins, self.vtx_ptr, self.vnets, self.adj_ptr, self.adj)]
        ptrs = [C.cast(_p(a), C.POINTER(C.c_int32)) if a is not None else None for a in self._keep]
        s.net_ptr, s.pins, s.vtx_ptr, s.vnets, s.adj_ptr, s.adj = ptrs
        return s


def build_hypergraph(model: str | int, m: int, n: int, rowptr: np.ndarray, colidx: np.ndarray) -> Hypergraph:
    """Hypergraph model of an m x n pattern (Table 1): symmetric, bipartite,
    row-net or column-net."""
    lib = _load()
    mdl = MODELS[model] if isinstance(model, str) else int(model)
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    s = _HG()
    if lib.ora_build(mdl, m, n, _p(rp), _p(ci), C.byref(s)) != 0:
        raise ValueError("bad model")
    k, l = s.k, s.l
    npins = s.net_ptr[l] if l > 0 else 0
    hg = Hypergraph(mdl, k, l, _arr(s.net_ptr, l + 1, np.int32), _arr(s.pins, npins, np.int32),
                    _arr(s.vtx_ptr, k + 1, np.int32), _arr(s.vnets, s.vtx_ptr[k] if k > 0 else 0, np.int32),
                    None, None)
    if mdl in (0, 1):
        hg.adj_ptr = _arr(s.adj_ptr, k + 1, np.int32)
        hg.adj = _arr(s.adj, s.adj_ptr[k] if k > 0 else 0, np.int32)
    lib.ora_hg_free(C.byref(s))
    return hg


def build_from_matrix(model: str | int, mat) -> Hypergraph:
    return build_hypergraph(model, mat.m, mat.n, mat.rowptr, mat.colidx)


def dual(k: int, l: int, net_ptr: np.ndarray, pins: np.ndarray):
    """Nets of the dual hypergraph G* (Definition 1.2): vertex v of G gives the
    net {e : v in e}; returns (net_ptr*, pins*) with k nets over l vertices."""
    lib = _load()
    np_ = np.ascontiguousarray(net_ptr, dtype=np.int32)
    pi = np.ascontiguousarray(pins, dtype=np.int32)
    a = C.POINTER(C.c_int32)()
    b = C.POINTER(C.c_int32)()
    lib.ora_dual(k, l, _p(np_), _p(pi), C.byref(a), C.byref(b))
    ptr = _arr(a, k + 1, np.int32)
    out = _arr(b, int(ptr[-1]), np.int32)
    lib.ora_free(C.cast(a, C.c_void_p))
    lib.ora_free(C.cast(b, C.c_void_p))
    return ptr, out


def components(hg: Hypergraph) -> np.ndarray:
    """Algorithm 1: component label (smallest vertex id) of every vertex."""
    lib = _load()
    p = np.zeros(hg.k, dtype=np.int32)
    s = hg._struct()
    lib.ora_components(hg.k, hg.l, _p(hg._keep[0]), _p(hg._keep[1]), _p(p))
    del s
    return p


def set_threads(n: int) -> None:
    """Threads of the oracle's per-vertex loops (results are the same for any
    count: every vertex's sums are one thread's, in a fixed order)."""
    _load().ora_set_threads(int(n))


def threads() -> int:
    return int(_load().ora_get_threads())


def rand64(seed: int, a: int, b: int) -> int:
    return int(_load().ora_rand64(seed & (2**64 - 1), a, b))


def init_side(k: int, d: int) -> int:
    return int(_load().ora_init_side(k, d))


def init_coords(k: int, d: int, seed: int) -> np.ndarray:
    """Random initial layout, fp32 [k, 4] (unused components 0)."""
    x = np.zeros((k, 4), dtype=np.float32)
    _load().ora_init_coords(k, d, seed & (2**64 - 1), _p(x))
    return x


def levels(k: int, d: int, occ: int = 8) -> int:
    return int(_load().ora_levels(k, d, occ))


def _x64(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 2 and x.shape[1] != 4:
        x = np.concatenate([x, np.zeros((x.shape[0], 4 - x.shape[1]))], axis=1)
    return np.ascontiguousarray(x.reshape(-1, 4))


def _opt64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def energy(hg: Hypergraph, d: int, x, w=None, c=None) -> float:
    """Energy of eq. graphenergysimple (log kernel for d = 2)."""
    s = hg._struct()
    xx, ww, cc = _x64(x), _opt64(w), _opt64(c)
    return float(_load().ora_energy(C.byref(s), d, _p(xx), _p(ww), _p(cc)))


def gradient(hg: Hypergraph, d: int, x, occ: int = 8, w=None, c=None):
    """Gradient y (eq. graphenergygradientsimple, repulsion on the grid pyramid),
    level-L cell keys (row-major index), L, and per-target (interaction count,
    summed source weight)."""
    s = hg._struct()
    xx, ww, cc = _x64(x), _opt64(w), _opt64(c)
    y = np.zeros_like(xx)
    keys = np.zeros(hg.k, dtype=np.uint32)
    L = C.c_int32(0)
    ninter = np.zeros(hg.k, dtype=np.int64)
    wseen = np.zeros(hg.k, dtype=np.float64)
    dg = _Diag(C.cast(_p(ninter), C.POINTER(C.c_int64)), C.cast(_p(wseen), C.POINTER(C.c_double)))
    _load().ora_gradient(C.byref(s), d, occ, _p(xx), _p(ww), _p(cc), _p(y), _p(keys), C.byref(L), C.byref(dg))
    return y, keys, int(L.value), ninter, wseen


def step0(k: int, d: int, x, sigma: float = 1.0) -> float:
    """Initial step length of a level: sigma times the mean point spacing."""
    xx = _x64(x)
    return float(_load().ora_step0(k, d, sigma, _p(xx)))


def layout_step(hg: Hypergraph, d: int, x, step: float, occ: int = 8, w=None, c=None):
    """One steepest-descent step (Algorithm 4) with step length ``step``:
    returns (x_new, y, keys, L)."""
    s = hg._struct()
    xx, ww, cc = _x64(x).copy(), _opt64(w), _opt64(c)
    y = np.zeros_like(xx)
    keys = np.zeros(hg.k, dtype=np.uint32)
    L = C.c_int32(0)
    _load().ora_layout_step(C.byref(s), d, occ, _p(ww), _p(cc), _p(xx), float(step), _p(y), _p(keys),
                            C.byref(L))
    return xx, y, keys, int(L.value)


def layout(hg: Hypergraph, d: int, x0, iters: int = 100, occ: int = 8, sigma: float = 1.0, decay: float = 0.9,
           w=None, c=None) -> np.ndarray:
    """T steps of Algorithm 4 on one level from x0; returns FP64 [k, 4]."""
    s = hg._struct()
    xx, ww, cc = _x64(x0).copy(), _opt64(w), _opt64(c)
    _load().ora_layout(C.byref(s), d, occ, sigma, decay, iters, _p(ww), _p(cc), _p(xx))
    return xx


def match(k: int, adj_ptr, adj, acost, seed: int, level: int = 0, rounds: int = 4):
    """Handshake heavy-edge matching of one coarsening level: (kc, mate, pi)."""
    ap = np.ascontiguousarray(adj_ptr, dtype=np.int32)
    aj = np.ascontiguousarray(adj, dtype=np.int32)
    ac = np.ascontiguousarray(acost, dtype=np.float64)
    mate = np.zeros(k, dtype=np.int32)
    pi = np.zeros(k, dtype=np.int32)
    kc = _load().ora_match(k, _p(ap), _p(aj), _p(ac), seed & (2**64 - 1), level, rounds, _p(mate), _p(pi))
    return int(kc), mate, pi


def hierarchy(hg: Hypergraph, seed: int, rounds: int = 4, kmin: int = 64) -> list[int]:
    """Vertex counts of the coarsening levels of Algorithm 3."""
    s = hg._struct()
    ks = np.zeros(41, dtype=np.int32)
    n = _load().ora_hierarchy(C.byref(s), seed & (2**64 - 1), rounds, kmin, _p(ks))
    return [int(v) for v in ks[:n]]


def hierarchy_level(hg: Hypergraph, j: int, seed: int, rounds: int = 4, kmin: int = 64, w=None):
    """Level j of the coarsening hierarchy of Algorithm 3 built from the whole
    graph: dict with k, adj_ptr, adj (neighbours ascending), acost (summed
    costs of the merged fine edges), w (summed vertex weights), pi (level j-1
    vertex -> level j vertex; None for j = 0) and nlevels.  None if j is not a
    level."""
    if hg.adj_ptr is None:
        raise ValueError("the hierarchy needs a graph model")
    lib = _load()
    s = hg._struct()
    ww = _opt64(w)
    k, nadj = C.c_int32(), C.c_int64()
    ap, aj, pi = C.POINTER(C.c_int32)(), C.POINTER(C.c_int32)(), C.POINTER(C.c_int32)()
    ac, wo = C.POINTER(C.c_double)(), C.POINTER(C.c_double)()
    nl = lib.ora_hierarchy_level(C.byref(s), _p(ww), seed & (2**64 - 1), rounds, kmin, j, C.byref(k), C.byref(nadj),
                                 C.byref(ap), C.byref(aj), C.byref(ac), C.byref(wo), C.byref(pi))
    if nl < 0:
        return None
    kk, na = int(k.value), int(nadj.value)
    kf = hg.k if j == 1 else None
    out = dict(k=kk, adj_ptr=_arr(ap, kk + 1, np.int32), adj=_arr(aj, na, np.int32),
               acost=_arr(ac, na, np.float64), w=_arr(wo, kk, np.float64), nlevels=int(nl), pi=None)
    if j > 0:
        if kf is None:
            kf = hierarchy(hg, seed, rounds, kmin)[j - 1]
        out["pi"] = _arr(pi, kf, np.int32)
    for ptr in (ap, aj, ac, wo, pi):
        if ptr:
            lib.ora_free(C.cast(ptr, C.c_void_p))
    return out


def prolong(kf: int, kc: int, d: int, seed: int, j: int, pi: np.ndarray, xc) -> np.ndarray:
    """Prolongation of Algorithm 3 from level j (kc points xc) to level j-1 (kf
    points, grouping pi): FP64 [kf, 4]."""
    xx = _x64(xc)
    pp = np.ascontiguousarray(pi, dtype=np.int32)
    out = np.zeros((max(kf, 1), 4), dtype=np.float64)
    _load().ora_prolong(kf, kc, d, seed & (2**64 - 1), j, _p(pp), _p(xx), _p(out))
    return out[:kf]


def graph_nets(k: int, adj_ptr: np.ndarray, adj: np.ndarray, acost: np.ndarray | None = None):
    """The graph given by a symmetric adjacency as a hypergraph of 2-pin nets
    (edges u < v in lexicographic order, the layout of the symmetric model),
    with the cost of every net taken from the adjacency entry (u, v)."""
    ap = np.asarray(adj_ptr, dtype=np.int64)
    aj = np.asarray(adj, dtype=np.int64)
    rows = np.repeat(np.arange(k, dtype=np.int64), np.diff(ap))
    keep = aj > rows
    u, v = rows[keep], aj[keep]
    l = len(u)
    pins = np.stack([u, v], axis=1).reshape(-1).astype(np.int32)
    net_ptr = (2 * np.arange(l + 1)).astype(np.int32)
    order = np.lexsort((np.arange(2 * l), pins))
    vtx_ptr = np.zeros(k + 1, dtype=np.int32)
    np.add.at(vtx_ptr, pins.astype(np.int64) + 1, 1)
    vtx_ptr = np.cumsum(vtx_ptr).astype(np.int32)
    vnets = (order // 2).astype(np.int32)
    hg = Hypergraph(0, k, l, net_ptr, pins, vtx_ptr, vnets, np.asarray(adj_ptr, dtype=np.int32),
                    np.asarray(adj, dtype=np.int32))
    cost = None if acost is None else np.asarray(acost, dtype=np.float64)[keep]
    return hg, cost


def layout_multilevel(hg: Hypergraph, d: int, seed: int, iters: int = 100, occ: int = 8, sigma: float = 1.0,
                      decay: float = 0.9, rounds: int = 4, kmin: int = 64, w=None) -> np.ndarray:
    """Multilevel layout (Algorithm 3 around Algorithm 4) of every connected
    component on its own; graph models only."""
    if hg.adj_ptr is None:
        raise ValueError("multilevel layout needs a graph model")
    s = hg._struct()
    x = np.zeros((hg.k, 4), dtype=np.float64)
    ww = _opt64(w)
    _load().ora_layout_multilevel(C.byref(s), d, occ, sigma, decay, iters, seed & (2**64 - 1), rounds, kmin,
                                  _p(ww), _p(x))
    return x


def bisect(d: int, x4: np.ndarray, verts: np.ndarray, seed: int, key: int = 1, km_iters: int = 20):
    """2-means of the points x4[verts] (Algorithm 5, m = 2): (split, labels, z1, z2)."""
    xf = np.ascontiguousarray(x4, dtype=np.float32).reshape(-1, 4)
    vv = np.ascontiguousarray(verts, dtype=np.int32)
    lab = np.zeros(len(vv), dtype=np.uint8)
    z1 = np.zeros(4, dtype=np.float32)
    z2 = np.zeros(4, dtype=np.float32)
    ok = _load().ora_bisect(d, _p(xf), _p(vv), len(vv), seed & (2**64 - 1), key, km_iters, _p(lab), _p(z1), _p(z2))
    return bool(ok), lab, z1, z2


def order(hg: Hypergraph, d: int, x4: np.ndarray, seed: int, km_iters: int = 20, min_part: int = 64,
          max_depth: int = 62, sbd: bool = False, sep_rec: bool = False, cut_order: bool = False,
          match: np.ndarray | None = None, order_free: bool = False):
    """Recursive BBD (or SBD) ordering from fp32 coordinates: (perm, tree).
    Connected components are ordered one after the other (block diagonal),
    each by its own recursion; tree records are sorted by (comp, heap).
    sep_rec: the separator of a split node is ordered recursively as well
    (children 3h-1, 3h, 3h+1 for V1, V2, V3; depth at most 39).
    cut_order: b (0: off; True counts as 1): without sep_rec, every
    separator is stably sorted by b two-bit numbers of its vertices' links
    into the parts of the splits of the descendants 1..b levels down.
    match: strengthened diagonal of a square matrix in the bipartite model
    (Sec. 4.2, the matching M as the map mu): match[i] is the column matched to
    row i; a vertex moved into a separator takes its partner with it, in the
    loop of Algorithm 7 over the cut edges in canonical order (a partner moved
    early leaves later edges at it uncut), or, with order_free, in the
    order-free reading (every cut edge's selected end and its partner)."""
    if hg.adj_ptr is None:
        raise ValueError("ordering needs a graph model (symmetric or bipartite)")
    mu = None
    if match is not None:
        mu = mu_from_match(hg, match)
    s = hg._struct()
    xf = np.ascontiguousarray(x4, dtype=np.float32).reshape(-1, 4)
    perm = np.zeros(hg.k, dtype=np.int32)
    t = _Tree()
    _load().ora_order(C.byref(s), d, _p(xf), seed & (2**64 - 1), km_iters, min_part, max_depth, int(sbd),
                      int(sep_rec), int(cut_order), _p(mu) if mu is not None else None, int(bool(order_free)),
                      _p(perm), C.byref(t))
    n = t.count
    tree = dict(heap=_arr(t.heap, n, np.uint64), offset=_arr(t.offset, n, np.int32), n1=_arr(t.n1, n, np.int32),
                n2=_arr(t.n2, n, np.int32), nsep=_arr(t.nsep, n, np.int32), depth=_arr(t.depth, n, np.int32),
                comp=_arr(t.comp, n, np.int32))
    _load().ora_tree_free(C.byref(t))
    return perm, tree


def finegrain_coords(fg: Hypergraph, xb: np.ndarray) -> np.ndarray:
    """Finegrain layout from the bipartite one (Sec. 4.2): every entry at the
    mean of its row's and its column's points (FP64, k x 4)."""
    if fg.model != MODELS["finegrain"]:
        raise ValueError("needs the finegrain model")
    s = fg._struct()
    xf = np.ascontiguousarray(xb, dtype=np.float32).reshape(-1, 4)
    out = np.zeros((max(fg.k, 1), 4), dtype=np.float64)
    _load().ora_finegrain_coords(C.byref(s), _p(xf), _p(out))
    return out[:fg.k]


def mu_from_match(hg: Hypergraph, match: np.ndarray) -> np.ndarray:
    """The map mu of a perfect matching M of the bipartite model of a square
    m x m pattern (Sec. 4.2): rows are vertices 0..m-1, columns m..2m-1, and
    row i is matched to column match[i].  Checks that M is a perfect matching
    of the pattern's edges."""
    if hg.model != MODELS["bipartite"] or hg.k % 2:
        raise ValueError("a strengthened diagonal needs the bipartite model of a square pattern")
    m = hg.k // 2
    match = np.asarray(match, dtype=np.int64)
    if match.shape != (m,) or not np.array_equal(np.sort(match), np.arange(m)):
        raise ValueError("match must be a permutation of the columns")
    for i in range(m):
        nb = hg.adj[hg.adj_ptr[i]:hg.adj_ptr[i + 1]]
        if not np.isin(m + match[i], nb):
            raise ValueError(f"row {i} is not linked to its matched column {match[i]}")
    mu = np.empty(2 * m, dtype=np.int32)
    mu[:m] = m + match
    mu[m + match] = np.arange(m)
    return mu


def kmeans(d: int, x4: np.ndarray, verts: np.ndarray, m: int, seed: int, key: int = 1, km_iters: int = 20):
    """m-way k-means++ (Algorithm 5): (labels in [0, m), centres m x 4, number
    of non-empty clusters).  For m = 2 it equals bisect with labels - 1."""
    xf = np.ascontiguousarray(x4, dtype=np.float32).reshape(-1, 4)
    vv = np.ascontiguousarray(verts, dtype=np.int32)
    lab = np.zeros(max(len(vv), 1), dtype=np.int32)
    z = np.zeros((max(m, 1), 4), dtype=np.float32)
    ne = _load().ora_kmeans(d, _p(xf), _p(vv), len(vv), m, seed & (2**64 - 1), key & (2**64 - 1), km_iters,
                            _p(lab), _p(z))
    return lab[:len(vv)], z[:m], int(ne)


def cut_size(net_ptr: np.ndarray, pins: np.ndarray, part: np.ndarray):
    """Cut-net count and (lambda - 1) of a vertex partition over the nets."""
    np_ = np.ascontiguousarray(net_ptr, dtype=np.int32)
    pi = np.ascontiguousarray(pins, dtype=np.int32)
    pa = np.ascontiguousarray(part, dtype=np.int32)
    a, b = C.c_int64(0), C.c_int64(0)
    _load().ora_cut_size(len(np_) - 1, _p(np_), _p(pi), _p(pa), C.byref(a), C.byref(b))
    return int(a.value), int(b.value)


def cholesky_nnz(n: int, rowptr: np.ndarray, colidx: np.ndarray, perm: np.ndarray) -> int:
    """nz(L) (with diagonal) of the symmetrically permuted pattern P(A+A^T)P^T."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    pp = np.ascontiguousarray(perm, dtype=np.int32)
    return int(_load().ora_cholesky_nnz(n, _p(rp), _p(ci), _p(pp)))


def fill_in(mat, perm: np.ndarray) -> float:
    """(nz(L) + nz(U) - nz(I)) / nz(A) for LU without pivoting of P A P^T
    (structurally symmetric patterns)."""
    nzl = cholesky_nnz(mat.n, mat.rowptr, mat.colidx, perm)
    return (2 * nzl - mat.n) / float(mat.nnz)


def parts_from_tree(k: int, perm: np.ndarray, tree: dict, sbd: bool = False) -> np.ndarray:
    """Final owner of every vertex: the index (in heap order) of its leaf, or of
    the internal node whose separator holds it."""
    part = np.full(k, -1, dtype=np.int32)
    for idx in range(len(tree["heap"])):
        o, n1, n2, ns = (int(tree[f][idx]) for f in ("offset", "n1", "n2", "nsep"))
        if n2 == 0 and ns == 0:
            part[perm[o:o + n1]] = idx
        else:
            so = o + n1 if sbd else o + n1 + n2
            part[perm[so:so + ns]] = idx
    return part
