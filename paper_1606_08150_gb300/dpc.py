"""Python binding of libdpc.so (ctypes; argument marshalling only).

The functions mirror the C ABI in ``include/dpc.h`` one to one and take torch
CUDA tensors for every array. PyTorch supplies device memory and the current
stream; every step of the computation runs in the library's CUDA kernels. There
is no CPU fallback: if libdpc.so cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

from . import build as _build

BASIC_DP, FLAT, WARP, BLOCK, GRID, QUEUE = 0, 1, 2, 3, 4, 5
LEVELS = {"basic_dp": BASIC_DP, "flat": FLAT, "warp": WARP, "block": BLOCK, "grid": GRID, "queue": QUEUE}
LEVEL_NAMES = {v: k for k, v in LEVELS.items()}

OK, ERR_INVALID_ARG, ERR_WORKSPACE, ERR_CUDA, ERR_DEVICE, ERR_TIMEOUT, ERR_OVERFLOW, ERR_UNSUPPORTED, ERR_DEPTH = range(9)
FLAG_SYNC_CHECK = 0x1
FLAG_DEVICE_MALLOC = 0x2  # dpc_sssp warp/block buffers from device malloc (the allocator study)

INF = 0xFFFFFFFF

# entry points declared in include/dpc.h
EXPORTS = (
    "dpc_status_string", "dpc_abi_version", "dpc_device_init", "dpc_memory_device_accessible",
    "dpc_sssp_workspace_size", "dpc_sssp",
    "dpc_spmv_csr_workspace_size", "dpc_spmv_csr", "dpc_spmv_csr_noalloc",
    "dpc_tree_workspace_size", "dpc_tree_descendants", "dpc_tree_height",
    "dpc_pagerank_workspace_size", "dpc_pagerank",
    "dpc_bfs_rec_workspace_size", "dpc_bfs_rec",
    "dpc_graph_coloring_workspace_size", "dpc_graph_coloring",
    "dpc_engine_workspace_size", "dpc_engine_init", "dpc_engine_step", "dpc_engine_serve",
    "dpc_mailbox_init", "dpc_mailbox_post", "dpc_mailbox_stop", "dpc_mailbox_taken",
    "dpc_wait_selftest", "dpc_gather_rate",
)

JOB_SSSP, JOB_TREE_DESCENDANTS, JOB_TREE_HEIGHT = 0, 1, 2


class Tuning(ctypes.Structure):
    """dpc_tuning: zero fields select the defaults."""

    _fields_ = [("threshold", ctypes.c_int32), ("parent_blocks", ctypes.c_int32), ("parent_threads", ctypes.c_int32),
                ("child_blocks", ctypes.c_int32), ("child_threads", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("kc", ctypes.c_int32), ("flags", ctypes.c_uint32), ("delta", ctypes.c_int32),
                ("sub_delta", ctypes.c_int32)]


class Job(ctypes.Structure):
    """dpc_job: one problem for the batched engine (device pointers)."""

    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("source", ctypes.c_int32),
                ("off", ctypes.c_void_p), ("col", ctypes.c_void_p), ("w", ctypes.c_void_p), ("out", ctypes.c_void_p)]


MAILBOX_CAP = 1024  # DPC_MAILBOX_CAP


class MailboxLayout(ctypes.Structure):
    """dpc_mailbox: the resident engine's ring of posted jobs (host memory)."""

    _fields_ = [("posted", ctypes.c_uint64), ("stop", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
                ("taken", ctypes.c_uint64), ("reserved1", ctypes.c_uint64 * 5), ("jobs", Job * MAILBOX_CAP),
                ("slots", ctypes.c_int32 * MAILBOX_CAP)]


class Stats(ctypes.Structure):
    """Host copy of dpc_stats (the device struct is 56 bytes)."""

    _fields_ = [("child_launches", ctypes.c_uint64), ("aux_launches", ctypes.c_uint64),
                ("buffered_items", ctypes.c_uint64), ("inline_items", ctypes.c_uint64),
                ("relaxations", ctypes.c_uint64), ("launch_failures", ctypes.c_uint64),
                ("rounds", ctypes.c_uint32), ("status", ctypes.c_uint32)]


STATS_BYTES = ctypes.sizeof(Stats)


class DpcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


def _load_library() -> ctypes.CDLL:
    # DPC_LIBRARY=checked selects the bounds-checked build (built by
    # build.build(checked=True)), DPC_LIBRARY=<file>.so another build of the
    # library (to compare two builds); the default is the regular build
    sel = os.environ.get("DPC_LIBRARY", "")
    path = _build.LIB_CHECKED if sel == "checked" else (sel if sel.endswith(".so") else _build.LIB)
    if not os.path.exists(path):
        raise ImportError(f"libdpc.so is not built ({path}); run __graft_entry__.build() or python -m "
                          "paper_1606_08150_gb300.build")
    lib = ctypes.CDLL(path)
    P, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
    st = ctypes.c_int
    lib.dpc_status_string.argtypes = [st]
    lib.dpc_status_string.restype = ctypes.c_char_p
    lib.dpc_abi_version.argtypes = []
    lib.dpc_abi_version.restype = i32
    lib.dpc_device_init.argtypes = [ctypes.c_int, sz]
    lib.dpc_device_init.restype = st
    lib.dpc_memory_device_accessible.argtypes = [P, ctypes.POINTER(i32)]
    lib.dpc_memory_device_accessible.restype = st
    lib.dpc_spmv_csr_workspace_size.argtypes = [i32, i32, st, P, P]
    lib.dpc_spmv_csr_workspace_size.restype = st
    lib.dpc_spmv_csr.argtypes = [P, P, P, i32, i32, i32, P, P, st, P, P, sz, P, P]
    lib.dpc_spmv_csr.restype = st
    lib.dpc_spmv_csr_noalloc.argtypes = [P, P, P, i32, i32, i32, P, P, st, P, P, P]
    lib.dpc_spmv_csr_noalloc.restype = st
    if hasattr(lib, "dpc_sssp"):
        lib.dpc_sssp_workspace_size.argtypes = [i32, i32, st, P, P]
        lib.dpc_sssp_workspace_size.restype = st
        lib.dpc_sssp.argtypes = [P, P, P, i32, i32, i32, P, st, P, P, sz, P, P]
        lib.dpc_sssp.restype = st
    lib.dpc_pagerank_workspace_size.argtypes = [i32, i32, st, P, P]
    lib.dpc_pagerank_workspace_size.restype = st
    lib.dpc_pagerank.argtypes = [P, P, P, i32, i32, ctypes.c_float, i32, P, st, P, P, sz, P, P]
    lib.dpc_pagerank.restype = st
    lib.dpc_bfs_rec_workspace_size.argtypes = [i32, i32, st, P, P]
    lib.dpc_bfs_rec_workspace_size.restype = st
    lib.dpc_bfs_rec.argtypes = [P, P, i32, i32, i32, P, st, P, P, sz, P, P]
    lib.dpc_bfs_rec.restype = st
    lib.dpc_graph_coloring_workspace_size.argtypes = [i32, i32, st, P, P]
    lib.dpc_graph_coloring_workspace_size.restype = st
    lib.dpc_graph_coloring.argtypes = [P, P, i32, i32, P, P, st, P, P, sz, P, P]
    lib.dpc_graph_coloring.restype = st
    lib.dpc_engine_workspace_size.argtypes = [i32, i32, i32, P, P]
    lib.dpc_engine_workspace_size.restype = st
    lib.dpc_engine_init.argtypes = [P, sz, i32, i32, i32, P, P, P]
    lib.dpc_engine_init.restype = st
    lib.dpc_engine_step.argtypes = [P, sz, i32, i32, i32, P, P, P, P, i32, P, P, P]
    lib.dpc_engine_step.restype = st
    lib.dpc_engine_serve.argtypes = [P, sz, i32, i32, i32, P, P, ctypes.c_uint32, P, P, P]
    lib.dpc_engine_serve.restype = st
    lib.dpc_mailbox_init.argtypes = [P]
    lib.dpc_mailbox_init.restype = st
    lib.dpc_mailbox_post.argtypes = [P, P, i32]
    lib.dpc_mailbox_post.restype = st
    lib.dpc_mailbox_stop.argtypes = [P]
    lib.dpc_mailbox_stop.restype = st
    lib.dpc_mailbox_taken.argtypes = [P, P]
    lib.dpc_mailbox_taken.restype = st
    lib.dpc_gather_rate.argtypes = [P, i32, i32, P, P, P]
    lib.dpc_gather_rate.restype = st
    lib.dpc_wait_selftest.argtypes = [ctypes.c_uint32, P, P]
    lib.dpc_wait_selftest.restype = st
    if hasattr(lib, "dpc_tree_height"):
        lib.dpc_tree_workspace_size.argtypes = [i32, st, P, P]
        lib.dpc_tree_workspace_size.restype = st
        for fn in (lib.dpc_tree_descendants, lib.dpc_tree_height):
            fn.argtypes = [P, P, i32, i32, P, st, P, P, sz, P, P]
            fn.restype = st
    return lib


_lib = _load_library()


def library() -> ctypes.CDLL:
    return _lib


def status_string(status: int) -> str:
    return _lib.dpc_status_string(status).decode()


def abi_version() -> int:
    return int(_lib.dpc_abi_version())


def device_init(device: int = 0, pending_launch_limit: int = 0) -> int:
    return int(_lib.dpc_device_init(device, pending_launch_limit))


def _check(status: int, where: str) -> None:
    if status != OK:
        raise DpcError(status, where)


def _level(level) -> int:
    return LEVELS[level] if isinstance(level, str) else int(level)


def _tuning(tuning: Optional[Tuning]):
    return ctypes.byref(tuning) if tuning is not None else None


def device_accessible(t: torch.Tensor) -> bool:
    """dpc_memory_device_accessible: whether the current device can read the
    tensor's memory in place (device memory, or pinned host memory mapped into
    the device's address space)."""
    if t.numel() == 0:
        return True
    flag = ctypes.c_int32(0)
    _check(_lib.dpc_memory_device_accessible(t.data_ptr(), ctypes.byref(flag)), "dpc_memory_device_accessible")
    return bool(flag.value)


def _dptr(t: Optional[torch.Tensor], dtype: torch.dtype, name: str, host_ok: bool = False):
    if t is None:
        return None
    if not t.is_cuda and not (host_ok and t.is_pinned() and device_accessible(t)):
        raise ValueError(f"{name} must be a CUDA tensor" +
                         (" or pinned host memory the device can read" if host_ok else ""))
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr() if t.numel() else None


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def new_stats(device=None) -> torch.Tensor:
    """Device buffer for dpc_stats (pass to a call, read with read_stats after sync)."""
    return torch.zeros(STATS_BYTES, dtype=torch.uint8, device=device or "cuda")


def read_stats(buf: torch.Tensor) -> Stats:
    raw = bytes(buf.cpu().numpy().tobytes())
    return Stats.from_buffer_copy(raw)


def _ws_tensor(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ------------------------------------------------------------------ SpMV

def spmv_csr_workspace_size(nrows: int, nnz: int, level, tuning: Optional[Tuning] = None) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib.dpc_spmv_csr_workspace_size(nrows, nnz, _level(level), _tuning(tuning), ctypes.byref(out)),
           "dpc_spmv_csr_workspace_size")
    return int(out.value)


def spmv_csr(off: torch.Tensor, col: torch.Tensor, val: torch.Tensor, x: torch.Tensor, y: torch.Tensor,
             level, tuning: Optional[Tuning] = None, workspace: Optional[torch.Tensor] = None,
             stats: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None,
             ncols: Optional[int] = None) -> int:
    """y = A x (fp32) through dpc_spmv_csr; returns the status (raises on host-side errors).
    The matrix (off, col, val) may be pinned host memory the device reads in
    place; x and y are CUDA tensors."""
    nrows = off.numel() - 1
    nnz = col.numel()
    ncols = x.numel() if ncols is None else ncols
    lvl = _level(level)
    if workspace is None:
        workspace = _ws_tensor(spmv_csr_workspace_size(nrows, nnz, lvl, tuning), y.device)
    st = _lib.dpc_spmv_csr(_dptr(off, torch.int32, "off", True), _dptr(col, torch.int32, "col", True),
                           _dptr(val, torch.float32, "val", True), nrows, ncols, nnz, _dptr(x, torch.float32, "x"),
                           _dptr(y, torch.float32, "y"), lvl, _tuning(tuning), workspace.data_ptr(),
                           workspace.numel(), _dptr(stats, torch.uint8, "stats"), _stream(stream))
    if st not in (OK, ERR_DEVICE, ERR_OVERFLOW, ERR_DEPTH, ERR_TIMEOUT):
        raise DpcError(st, "dpc_spmv_csr")
    return int(st)


NOALLOC_SCRATCH_BYTES = 16 << 20  # DPC_NOALLOC_SCRATCH_BYTES


def wait_selftest(limit_us: int, status: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> None:
    """dpc_wait_selftest: one block waits `limit_us` microseconds for a word
    nothing sets, then writes DPC_ERR_TIMEOUT and the microseconds waited into
    status[0:2] (int32 device tensor of at least two elements)."""
    if status.numel() < 2:
        raise ValueError("status needs two elements")
    _check(_lib.dpc_wait_selftest(int(limit_us), _dptr(status, torch.int32, "status"), _stream(stream)),
           "dpc_wait_selftest")


def gather_rate(x: torch.Tensor, batches: int, out: torch.Tensor,
                stream: Optional[torch.cuda.Stream] = None) -> int:
    """dpc_gather_rate: random 4-byte gathers from x (float32, a power-of-two
    length) held in L2, summed into out[0]; returns the number of loads."""
    g = ctypes.c_int64(0)
    _check(_lib.dpc_gather_rate(_dptr(x, torch.float32, "x"), x.numel(), int(batches),
                                _dptr(out, torch.float32, "out"), ctypes.byref(g), _stream(stream)),
           "dpc_gather_rate")
    return int(g.value)


def spmv_csr_noalloc(off: torch.Tensor, col: torch.Tensor, val: torch.Tensor, x: torch.Tensor, y: torch.Tensor,
                     level, tuning: Optional[Tuning] = None, stats: Optional[torch.Tensor] = None,
                     stream: Optional[torch.cuda.Stream] = None, ncols: Optional[int] = None) -> int:
    """y = A x through dpc_spmv_csr_noalloc: no workspace, nothing allocated by the
    library; scratch comes from the array compiled into libdpc.so. Returns the
    status; raises on host-side errors (including a problem too large for the
    array, DPC_ERR_WORKSPACE)."""
    nrows = off.numel() - 1
    nnz = col.numel()
    ncols = x.numel() if ncols is None else ncols
    st = _lib.dpc_spmv_csr_noalloc(_dptr(off, torch.int32, "off"), _dptr(col, torch.int32, "col"),
                                   _dptr(val, torch.float32, "val"), nrows, ncols, nnz,
                                   _dptr(x, torch.float32, "x"), _dptr(y, torch.float32, "y"), _level(level),
                                   _tuning(tuning), _dptr(stats, torch.uint8, "stats"), _stream(stream))
    if st not in (OK, ERR_DEVICE, ERR_OVERFLOW, ERR_DEPTH, ERR_TIMEOUT):
        raise DpcError(st, "dpc_spmv_csr_noalloc")
    return int(st)


# ------------------------------------------------------------------ PageRank

def pagerank_workspace_size(n: int, m: int, level, tuning: Optional[Tuning] = None) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib.dpc_pagerank_workspace_size(n, m, _level(level), _tuning(tuning), ctypes.byref(out)),
           "dpc_pagerank_workspace_size")
    return int(out.value)


def pagerank(in_off: torch.Tensor, in_src: torch.Tensor, outdeg: torch.Tensor, rank: torch.Tensor, level,
             damping: float = 0.85, iterations: int = 20, tuning: Optional[Tuning] = None,
             workspace: Optional[torch.Tensor] = None, stats: Optional[torch.Tensor] = None,
             stream: Optional[torch.cuda.Stream] = None) -> int:
    """PageRank over the in-edge CSR (in_off, in_src) with out-degrees outdeg
    into rank (float32): `iterations` power iterations from the uniform vector."""
    n = in_off.numel() - 1
    m = in_src.numel()
    lvl = _level(level)
    if workspace is None:
        workspace = _ws_tensor(pagerank_workspace_size(n, m, lvl, tuning), in_off.device)
    st = _lib.dpc_pagerank(_dptr(in_off, torch.int32, "in_off"), _dptr(in_src, torch.int32, "in_src"),
                           _dptr(outdeg, torch.int32, "outdeg"), n, m, float(damping), int(iterations),
                           _dptr(rank, torch.float32, "rank"), lvl, _tuning(tuning), workspace.data_ptr(),
                           workspace.numel(), _dptr(stats, torch.uint8, "stats"), _stream(stream))
    if st not in (OK, ERR_DEVICE, ERR_OVERFLOW, ERR_DEPTH, ERR_TIMEOUT):
        raise DpcError(st, "dpc_pagerank")
    return int(st)


# ------------------------------------------------------------------ graph colouring

def graph_coloring_workspace_size(n: int, m: int, level, tuning: Optional[Tuning] = None) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib.dpc_graph_coloring_workspace_size(n, m, _level(level), _tuning(tuning), ctypes.byref(out)),
           "dpc_graph_coloring_workspace_size")
    return int(out.value)


def graph_coloring(off: torch.Tensor, col: torch.Tensor, priority: torch.Tensor, color: torch.Tensor, level,
                   tuning: Optional[Tuning] = None, workspace: Optional[torch.Tensor] = None,
                   stats: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None) -> int:
    """Jones-Plassmann colours into color (int32) for the symmetric CSR graph
    (off, col) with vertex priorities `priority` (uint32 stored in an int32 tensor)."""
    n = off.numel() - 1
    m = col.numel()
    lvl = _level(level)
    if workspace is None:
        workspace = _ws_tensor(graph_coloring_workspace_size(n, m, lvl, tuning), off.device)
    st = _lib.dpc_graph_coloring(_dptr(off, torch.int32, "off"), _dptr(col, torch.int32, "col"), n, m,
                                 _dptr(priority, torch.int32, "priority"), _dptr(color, torch.int32, "color"), lvl,
                                 _tuning(tuning), workspace.data_ptr(), workspace.numel(),
                                 _dptr(stats, torch.uint8, "stats"), _stream(stream))
    if st not in (OK, ERR_DEVICE, ERR_OVERFLOW, ERR_DEPTH, ERR_TIMEOUT):
        raise DpcError(st, "dpc_graph_coloring")
    return int(st)


# ------------------------------------------------------------------ recursive BFS

def bfs_rec_workspace_size(n: int, m: int, level, tuning: Optional[Tuning] = None) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib.dpc_bfs_rec_workspace_size(n, m, _level(level), _tuning(tuning), ctypes.byref(out)),
           "dpc_bfs_rec_workspace_size")
    return int(out.value)


def bfs_rec(off: torch.Tensor, col: torch.Tensor, source: int, bfs_level: torch.Tensor, level,
            tuning: Optional[Tuning] = None, workspace: Optional[torch.Tensor] = None,
            stats: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None) -> int:
    """Breadth-first levels from `source` into bfs_level (uint32 stored in an int32 tensor)."""
    n = off.numel() - 1
    m = col.numel()
    lvl = _level(level)
    if workspace is None:
        workspace = _ws_tensor(bfs_rec_workspace_size(n, m, lvl, tuning), off.device)
    st = _lib.dpc_bfs_rec(_dptr(off, torch.int32, "off"), _dptr(col, torch.int32, "col"), n, m, source,
                          _dptr(bfs_level, torch.int32, "bfs_level"), lvl, _tuning(tuning), workspace.data_ptr(),
                          workspace.numel(), _dptr(stats, torch.uint8, "stats"), _stream(stream))
    if st not in (OK, ERR_DEVICE, ERR_OVERFLOW, ERR_DEPTH, ERR_TIMEOUT):
        raise DpcError(st, "dpc_bfs_rec")
    return int(st)


# ------------------------------------------------------------------ SSSP

def sssp_workspace_size(n: int, m: int, level, tuning: Optional[Tuning] = None) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib.dpc_sssp_workspace_size(n, m, _level(level), _tuning(tuning), ctypes.byref(out)),
           "dpc_sssp_workspace_size")
    return int(out.value)


def sssp(off: torch.Tensor, col: torch.Tensor, w: torch.Tensor, source: int, dist: torch.Tensor, level,
         tuning: Optional[Tuning] = None, workspace: Optional[torch.Tensor] = None,
         stats: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None) -> int:
    """Shortest-path distances from `source` into dist (uint32 stored in an int32 tensor)."""
    n = off.numel() - 1
    m = col.numel()
    lvl = _level(level)
    if workspace is None:
        workspace = _ws_tensor(sssp_workspace_size(n, m, lvl, tuning), off.device)
    st = _lib.dpc_sssp(_dptr(off, torch.int32, "off"), _dptr(col, torch.int32, "col"), _dptr(w, torch.int32, "w"),
                       n, m, source, _dptr(dist, torch.int32, "dist"), lvl, _tuning(tuning), workspace.data_ptr(),
                       workspace.numel(), _dptr(stats, torch.uint8, "stats"), _stream(stream))
    if st not in (OK, ERR_DEVICE, ERR_OVERFLOW, ERR_DEPTH, ERR_TIMEOUT):
        raise DpcError(st, "dpc_sssp")
    return int(st)


# ------------------------------------------------------------------ trees

def tree_workspace_size(n: int, level, tuning: Optional[Tuning] = None) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib.dpc_tree_workspace_size(n, _level(level), _tuning(tuning), ctypes.byref(out)),
           "dpc_tree_workspace_size")
    return int(out.value)


def _tree(fn, name, coff, cidx, root, out, out_dtype, level, tuning, workspace, stats, stream):
    n = coff.numel() - 1
    lvl = _level(level)
    if workspace is None:
        workspace = _ws_tensor(tree_workspace_size(n, lvl, tuning), coff.device)
    st = fn(_dptr(coff, torch.int32, "coff"), _dptr(cidx, torch.int32, "cidx"), n, root,
            _dptr(out, out_dtype, "out"), lvl, _tuning(tuning), workspace.data_ptr(), workspace.numel(),
            _dptr(stats, torch.uint8, "stats"), _stream(stream))
    if st not in (OK, ERR_DEVICE, ERR_OVERFLOW, ERR_DEPTH, ERR_TIMEOUT):
        raise DpcError(st, name)
    return int(st)


def tree_descendants(coff, cidx, root, desc, level, tuning=None, workspace=None, stats=None, stream=None) -> int:
    """Proper-descendant counts (uint32 stored in an int32 tensor)."""
    return _tree(_lib.dpc_tree_descendants, "dpc_tree_descendants", coff, cidx, root, desc, torch.int32, level,
                 tuning, workspace, stats, stream)


def tree_height(coff, cidx, root, height, level, tuning=None, workspace=None, stats=None, stream=None) -> int:
    """Node heights (int32, leaves 0)."""
    return _tree(_lib.dpc_tree_height, "dpc_tree_height", coff, cidx, root, height, torch.int32, level, tuning,
                 workspace, stats, stream)


# ------------------------------------------------------------------ batched engine

def engine_workspace_size(slots: int, max_n: int, max_m: int, tuning: Optional[Tuning] = None) -> int:
    out = ctypes.c_size_t(0)
    _check(_lib.dpc_engine_workspace_size(slots, max_n, max_m, _tuning(tuning), ctypes.byref(out)),
           "dpc_engine_workspace_size")
    return int(out.value)


def _state_ptr(t: torch.Tensor):
    """slot_state: a CUDA tensor, or a pinned host tensor (the resident form's)."""
    if t.is_cuda:
        return _dptr(t, torch.int32, "slot_state")
    if not t.is_pinned() or t.dtype != torch.int32 or not t.is_contiguous():
        raise ValueError("slot_state must be a CUDA int32 tensor or a pinned, contiguous host int32 tensor")
    return t.data_ptr()


def engine_init(workspace: torch.Tensor, slots: int, max_n: int, max_m: int, slot_state: torch.Tensor,
                tuning: Optional[Tuning] = None, stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(_lib.dpc_engine_init(workspace.data_ptr(), workspace.numel(), slots, max_n, max_m, _tuning(tuning),
                                _state_ptr(slot_state), _stream(stream)), "dpc_engine_init")


def engine_step(workspace: torch.Tensor, slots: int, max_n: int, max_m: int, new_jobs: Optional[torch.Tensor],
                new_slots: Optional[torch.Tensor], new_count: Optional[torch.Tensor], max_waves: int,
                slot_state: torch.Tensor, tuning: Optional[Tuning] = None, stats: Optional[torch.Tensor] = None,
                stream: Optional[torch.cuda.Stream] = None) -> None:
    """One engine step. new_jobs: device uint8 tensor holding packed dpc_job
    records (see jobs_tensor); new_slots / new_count: device int32 tensors."""
    _check(_lib.dpc_engine_step(workspace.data_ptr(), workspace.numel(), slots, max_n, max_m, _tuning(tuning),
                                new_jobs.data_ptr() if new_jobs is not None else None,
                                _dptr(new_slots, torch.int32, "new_slots"), _dptr(new_count, torch.int32, "new_count"),
                                max_waves, _state_ptr(slot_state),
                                _dptr(stats, torch.uint8, "stats"), _stream(stream)), "dpc_engine_step")


class Mailbox:
    """The resident engine's mailbox (dpc_mailbox) in pinned host memory. One
    host thread posts; the running kernel admits what was posted at its next
    wave barrier."""

    def __init__(self):
        self.buf = torch.zeros(ctypes.sizeof(MailboxLayout), dtype=torch.uint8).pin_memory()
        self.ptr = self.buf.data_ptr()
        _check(_lib.dpc_mailbox_init(self.ptr), "dpc_mailbox_init")

    def post(self, job: Job, slot: int) -> None:
        _check(_lib.dpc_mailbox_post(self.ptr, ctypes.byref(job), int(slot)), "dpc_mailbox_post")

    def stop(self) -> None:
        _check(_lib.dpc_mailbox_stop(self.ptr), "dpc_mailbox_stop")

    def clear_stop(self) -> None:
        """Undo stop(); only while no resident kernel runs on this mailbox."""
        MailboxLayout.from_address(self.ptr).stop = 0

    def taken(self) -> int:
        out = ctypes.c_uint64(0)
        _check(_lib.dpc_mailbox_taken(self.ptr, ctypes.byref(out)), "dpc_mailbox_taken")
        return int(out.value)


def engine_serve(workspace: torch.Tensor, slots: int, max_n: int, max_m: int, mailbox: Mailbox, limit_us: int,
                 slot_state: torch.Tensor, tuning: Optional[Tuning] = None, stats: Optional[torch.Tensor] = None,
                 stream: Optional[torch.cuda.Stream] = None) -> None:
    """Launch the resident engine (returns at once); slot_state: pinned host int32."""
    if slot_state.is_cuda:
        raise ValueError("the resident engine reports in pinned host memory: slot_state must be a pinned host tensor")
    _check(_lib.dpc_engine_serve(workspace.data_ptr(), workspace.numel(), slots, max_n, max_m, _tuning(tuning),
                                 mailbox.ptr, int(limit_us), _state_ptr(slot_state), _dptr(stats, torch.uint8, "stats"),
                                 _stream(stream)), "dpc_engine_serve")


def pack_jobs(jobs) -> bytes:
    """Pack a sequence of Job records into the dpc_job array layout."""
    arr = (Job * len(jobs))(*jobs)
    return bytes(memoryview(arr).cast("B"))
