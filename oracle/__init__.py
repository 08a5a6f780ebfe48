"""CPU oracle for the consolidated dynamic-parallelism hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the product path. It shares no
code with the CUDA library and never imports it.

The arithmetic lives in ``dpc_oracle.c`` (plain single-threaded C, compiled with
gcc on first use); this module only marshals numpy arrays. See the header of
``dpc_oracle.c`` for the passage of the paper each function follows.

Parity pins (in ``tests/test_oracle_*.py``): Floyd-Warshall and hand-worked
graphs for SSSP, dense / integer-exact matrix-vector products for SpMV,
brute-force ancestor walks and closed forms (chains, stars) for the trees, and
hand-counted launch tables (including the two-child example of Fig. 2) for the
consolidation launch counts, and for PageRank the stationary vector of the
Google matrix from numpy's eigen-solver, closed forms (cycles, complete graphs,
a star into a dangling hub) and conservation of total rank; for BFS the
unweighted shortest paths of scipy's csgraph, Dijkstra with unit weights and
the level invariants of a breadth-first tree.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

INF = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile dpc_oracle.c into liboracle.so (gcc, -O2, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the argument and result types of every oracle function on `lib`."""
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.oracle_sssp_dijkstra.argtypes = [i32, P, P, P, i32, P]
    lib.oracle_sssp_dijkstra.restype = ctypes.c_int
    lib.oracle_sssp_frontier.argtypes = [i32, P, P, P, i32, i32, P, i64, P, P, P]
    lib.oracle_sssp_frontier.restype = i64
    lib.oracle_sssp_nearfar.argtypes = [i32, P, P, P, i32, ctypes.c_uint32, ctypes.c_uint32, i32, P, i64, P, P, P, P,
                                        P]
    lib.oracle_sssp_nearfar.restype = i64
    lib.oracle_spmv_f64.argtypes = [i32, i32, P, P, P, P, P, P]
    lib.oracle_spmv_f64.restype = ctypes.c_int
    lib.oracle_tree_descendants.argtypes = [i32, P, P, i32, P]
    lib.oracle_tree_descendants.restype = ctypes.c_int
    lib.oracle_tree_height.argtypes = [i32, P, P, i32, P]
    lib.oracle_tree_height.restype = ctypes.c_int
    lib.oracle_tree_levels.argtypes = [i32, P, P, i32, i32, i32, P, P, P, P]
    lib.oracle_tree_levels.restype = i32
    lib.oracle_pagerank.argtypes = [i32, P, P, ctypes.c_double, i32, P]
    lib.oracle_pagerank.restype = ctypes.c_int
    lib.oracle_bfs.argtypes = [i32, P, P, i32, P]
    lib.oracle_bfs.restype = i32
    lib.oracle_color_jp.argtypes = [i32, P, P, P, i32, P, i64, P, P]
    lib.oracle_color_jp.restype = i32
    lib.oracle_consolidation_launches.argtypes = [i64, P, i32, i32, P]
    lib.oracle_consolidation_launches.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def load_variant(path: str):
    """Bind a library built from another copy of dpc_oracle.c (the CPU tests
    build deliberately broken copies to show that the pins catch them)."""
    return _bind(ctypes.CDLL(path))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray):
    return a.ctypes.data if a.size else None


def sssp_dijkstra(off, col, w, source: int) -> np.ndarray:
    """Unique shortest-path distances (uint32, unreachable = 0xFFFFFFFF)."""
    off, col, w = _c(off, np.int32), _c(col, np.int32), _c(w, np.uint32)
    n = off.shape[0] - 1
    dist = np.empty(n, np.uint32)
    rc = _load().oracle_sssp_dijkstra(n, _p(off), _p(col), _p(w), source, _p(dist))
    if rc != 0:
        raise ValueError(f"oracle_sssp_dijkstra failed ({rc})")
    return dist


@dataclass
class FrontierRun:
    dist: np.ndarray
    frontier_size: np.ndarray
    heavy: np.ndarray
    relaxations: int

    @property
    def rounds(self) -> int:
        return int(self.frontier_size.shape[0])


def sssp_frontier(off, col, w, source: int, threshold: int, max_rounds: int = 1 << 20) -> FrontierRun:
    """Frontier rounds of relaxation: distances plus per-round frontier statistics."""
    off, col, w = _c(off, np.int32), _c(col, np.int32), _c(w, np.uint32)
    n = off.shape[0] - 1
    dist = np.empty(n, np.uint32)
    cap = min(max_rounds, n + 1)
    fs = np.zeros(cap, np.int64)
    hv = np.zeros(cap, np.int64)
    relax = ctypes.c_int64(0)
    r = _load().oracle_sssp_frontier(n, _p(off), _p(col), _p(w), source, threshold, _p(dist), cap, _p(fs), _p(hv),
                                     ctypes.addressof(relax))
    if r < 0:
        raise ValueError("oracle_sssp_frontier failed")
    return FrontierRun(dist, fs[:r].copy(), hv[:r].copy(), int(relax.value))


@dataclass
class NearFarRun(FrontierRun):
    splits: int = 0
    subsplits: int = 0


def sssp_nearfar(off, col, w, source: int, delta: int, threshold: int, sub_delta: int = 0,
                 max_rounds: int = 1 << 24) -> NearFarRun:
    """Frontier rounds with the near-far split of width `delta` (0: no split)
    and, for vertices above the threshold, the sub-split of width `sub_delta`
    (0: none)."""
    off, col, w = _c(off, np.int32), _c(col, np.int32), _c(w, np.uint32)
    n = off.shape[0] - 1
    dist = np.empty(n, np.uint32)
    cap = min(max_rounds, 1 << 16)
    while True:
        fs = np.zeros(cap, np.int64)
        hv = np.zeros(cap, np.int64)
        relax, splits, subs = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        r = _load().oracle_sssp_nearfar(n, _p(off), _p(col), _p(w), source, int(delta), int(sub_delta), threshold,
                                        _p(dist), cap, _p(fs), _p(hv), ctypes.addressof(relax),
                                        ctypes.addressof(splits), ctypes.addressof(subs))
        if r >= 0 or cap >= max_rounds:
            break
        cap = min(max_rounds, cap * 16)  # more rounds than the arrays held: run again with room
    if r < 0:
        raise ValueError("oracle_sssp_nearfar failed")
    return NearFarRun(dist, fs[:r].copy(), hv[:r].copy(), int(relax.value), int(splits.value), int(subs.value))


def spmv_f64(off, col, val, x, ncols: int | None = None):
    """(y, absrow): y = A x in float64 and absrow[i] = sum_k |a_ik x_k|."""
    off, col = _c(off, np.int32), _c(col, np.int32)
    val, x = _c(val, np.float32), _c(x, np.float32)
    nrows = off.shape[0] - 1
    ncols = x.shape[0] if ncols is None else ncols
    y = np.empty(nrows, np.float64)
    a = np.empty(nrows, np.float64)
    rc = _load().oracle_spmv_f64(nrows, ncols, _p(off), _p(col), _p(val), _p(x), _p(y), _p(a))
    if rc != 0:
        raise ValueError("oracle_spmv_f64 failed")
    return y, a


def tree_descendants(coff, cidx, root: int = 0) -> np.ndarray:
    coff, cidx = _c(coff, np.int32), _c(cidx, np.int32)
    n = coff.shape[0] - 1
    out = np.zeros(n, np.uint32)
    if _load().oracle_tree_descendants(n, _p(coff), _p(cidx), root, _p(out)) != 0:
        raise ValueError("not a tree rooted at root spanning all nodes")
    return out


def tree_height(coff, cidx, root: int = 0) -> np.ndarray:
    coff, cidx = _c(coff, np.int32), _c(cidx, np.int32)
    n = coff.shape[0] - 1
    out = np.zeros(n, np.int32)
    if _load().oracle_tree_height(n, _p(coff), _p(cidx), root, _p(out)) != 0:
        raise ValueError("not a tree rooted at root spanning all nodes")
    return out


@dataclass
class TreeLevels:
    nodes: np.ndarray
    internal: np.ndarray
    edges: np.ndarray
    heavy: np.ndarray


def tree_levels(coff, cidx, root: int = 0, threshold: int = 32, max_levels: int = 1 << 16) -> TreeLevels:
    coff, cidx = _c(coff, np.int32), _c(cidx, np.int32)
    n = coff.shape[0] - 1
    cap = min(max_levels, n + 1)
    arrs = [np.zeros(cap, np.int64) for _ in range(4)]
    L = _load().oracle_tree_levels(n, _p(coff), _p(cidx), root, threshold, cap, *[_p(a) for a in arrs])
    if L < 0:
        raise ValueError("oracle_tree_levels failed")
    return TreeLevels(*[a[:L].copy() for a in arrs])


LEVELS = ("basic_dp", "flat", "warp", "block", "grid")


def pagerank(off, col, damping: float, iters: int) -> np.ndarray:
    """PageRank after `iters` power iterations from the uniform vector (float64),
    graph given by its out-edge CSR; see oracle_pagerank for the definition."""
    off, col = _c(off, np.int32), _c(col, np.int32)
    n = off.shape[0] - 1
    rank = np.empty(n, np.float64)
    if _load().oracle_pagerank(n, _p(off), _p(col), float(damping), int(iters), _p(rank)) != 0:
        raise ValueError("bad arguments")
    return rank


def bfs(off, col, source: int):
    """Breadth-first levels from `source` (uint32, unreachable = 0xFFFFFFFF) and
    the number of distinct levels."""
    off, col = _c(off, np.int32), _c(col, np.int32)
    n = off.shape[0] - 1
    level = np.empty(n, np.uint32)
    depth = _load().oracle_bfs(n, _p(off), _p(col), int(source), _p(level))
    if depth < 0:
        raise ValueError("bad arguments")
    return level, int(depth)


@dataclass
class Coloring:
    color: np.ndarray    # int32, colours 1..rounds
    rounds: int
    active: np.ndarray   # uncoloured vertices when each round began
    heavy: np.ndarray    # of those, the ones with more than `threshold` neighbours


def color_jp(off, col, prio, threshold: int = 32) -> Coloring:
    """Round-sweep colouring: the independent-set rounds of Jones-Plassmann with
    the given priorities (ties: larger id wins), the colour being the round."""
    off, col, prio = _c(off, np.int32), _c(col, np.int32), _c(prio, np.uint32)
    n = off.shape[0] - 1
    color = np.empty(n, np.int32)
    cap = n + 1
    active = np.zeros(cap, np.int64)
    heavy = np.zeros(cap, np.int64)
    r = _load().oracle_color_jp(n, _p(off), _p(col), _p(prio), int(threshold), _p(color), cap, _p(active),
                                _p(heavy))
    if r < 0:
        raise ValueError("bad arguments")
    return Coloring(color, int(r), active[:r].copy(), heavy[:r].copy())


def consolidation_launches(flags, blocks: int, threads: int) -> dict:
    """Child launches of one parent grid per consolidation granularity (Sec. IV.B)."""
    f = _c(np.asarray(flags).astype(np.uint8), np.uint8)
    out = np.zeros(5, np.int64)
    if _load().oracle_consolidation_launches(f.shape[0], _p(f), blocks, threads, _p(out)) != 0:
        raise ValueError("bad arguments")
    return dict(zip(LEVELS, (int(v) for v in out)))
