"""Continuous-batching request loop over the persistent engine.

Requests are SSSP queries (graph, source) and tree queries (tree, descendants
or heights) on problems kept resident in device memory. The loop admits
arrived requests into free engine slots (the number of slots is chosen from
the free device memory), runs one engine step of a bounded number of waves,
and retires the requests whose slot reports completion. New arrivals join the
work already on the GPU at the next step: their tasks share the waves of the
running ones. The engine step is a CUDA graph replayed every step, between an
asynchronous copy of the admissions in and of the slot states out.

ResidentServer keeps the engine on the GPU instead (dpc_engine_serve): an
arrival is posted to the running kernel's mailbox in pinned host memory and
joins the waves at the kernel's next wave barrier, with no step boundary and
no launch in between; completions are read from pinned host memory while the
kernel runs.

The one-at-a-time baseline serves the same stream with one library call per
request (grid-level consolidation), each waited for before the next.

Host-side scheduling only: every step of the computation runs in libdpc.so.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import dpc, gen


@dataclass
class Request:
    kind: int        # dpc.JOB_SSSP / JOB_TREE_DESCENDANTS / JOB_TREE_HEIGHT
    problem: int     # index into the resident problem pool of that kind
    source: int      # SSSP source / tree root
    arrival: float   # seconds after the start of the stream


@dataclass
class Resident:
    """A graph or tree uploaded once and kept on the device."""

    n: int
    m: int
    off: torch.Tensor
    col: torch.Tensor
    w: Optional[torch.Tensor] = None


def upload_graph(g: gen.Graph) -> Resident:
    return Resident(g.n, g.m, torch.from_numpy(g.off).cuda(), torch.from_numpy(g.col).cuda(),
                    torch.from_numpy(g.w.view(np.int32)).cuda())


def upload_tree(t: gen.Tree) -> Resident:
    cidx = t.cidx if t.n > 1 else np.zeros(1, np.int32)
    return Resident(t.n, max(t.n - 1, 0), torch.from_numpy(t.coff).cuda(), torch.from_numpy(cidx).cuda())


def slots_for_memory(max_n: int, max_m: int, budget_bytes: int, max_slots: int = 256,
                     tuning: Optional[dpc.Tuning] = None) -> int:
    """Largest slot count whose engine workspace plus per-slot outputs fit the budget."""
    lo, hi = 1, max_slots
    per_out = 4 * max_n
    if dpc.engine_workspace_size(1, max_n, max_m, tuning) + per_out > budget_bytes:
        return 0
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if dpc.engine_workspace_size(mid, max_n, max_m, tuning) + mid * per_out <= budget_bytes:
            lo = mid
        else:
            hi = mid - 1
    return lo


@dataclass
class ServeResult:
    admitted: np.ndarray   # seconds, per request
    finished: np.ndarray   # seconds, per request
    steps: int
    slots: int
    makespan: float
    status: int = 0
    slot_of: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))

    def latencies(self, arrivals: np.ndarray) -> np.ndarray:
        return self.finished - arrivals


class Server:
    """Persistent-engine server with continuous batching."""

    def __init__(self, graphs: Sequence[Resident], trees: Sequence[Resident], slots: Optional[int] = None,
                 waves_per_step: int = 32, tuning: Optional[dpc.Tuning] = None, memory_fraction: float = 0.5,
                 max_slots: int = 128, use_graph: bool = True):
        self.graphs, self.trees = list(graphs), list(trees)
        self.max_n = max([r.n for r in self.graphs + self.trees] + [1])
        self.max_m = max([r.m for r in self.graphs] + [r.n for r in self.trees] + [1])
        self.tuning = tuning
        if slots is None:  # admission by free device memory
            free, _ = torch.cuda.mem_get_info()
            slots = slots_for_memory(self.max_n, self.max_m, int(free * memory_fraction), max_slots, tuning)
            if slots < 1:
                raise MemoryError("not enough free device memory for one engine slot")
        self.slots = slots
        self.waves = waves_per_step
        self.ws = torch.empty(dpc.engine_workspace_size(slots, self.max_n, self.max_m, tuning), dtype=torch.uint8,
                              device="cuda")
        self.state = torch.zeros(slots, dtype=torch.int32, device="cuda")
        self.out = torch.empty((slots, self.max_n), dtype=torch.int32, device="cuda")
        self.stats = dpc.new_stats()
        # staging: pinned host -> device inside the step graph
        self.h_jobs = torch.zeros(48 * slots, dtype=torch.uint8).pin_memory()
        self.h_slots = torch.zeros(slots, dtype=torch.int32).pin_memory()
        self.h_count = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.h_state = torch.zeros(slots, dtype=torch.int32).pin_memory()
        self.d_jobs = torch.zeros(48 * slots, dtype=torch.uint8, device="cuda")
        self.d_slots = torch.zeros(slots, dtype=torch.int32, device="cuda")
        self.d_count = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.stream = torch.cuda.Stream()
        self.graph = None
        self.use_graph = use_graph
        self.reset()

    def reset(self) -> None:
        with torch.cuda.stream(self.stream):
            dpc.engine_init(self.ws, self.slots, self.max_n, self.max_m, self.state, self.tuning)
        self.stream.synchronize()

    def _engine_step(self) -> None:
        dpc.engine_step(self.ws, self.slots, self.max_n, self.max_m, self.d_jobs, self.d_slots, self.d_count,
                        self.waves, self.state, self.tuning, self.stats)

    def _capture(self) -> None:
        # the graph holds the engine step only; the small admission / state
        # copies are plain asynchronous copies on the same stream around it
        with torch.cuda.stream(self.stream):
            self.d_count.zero_()
            self._engine_step()  # warm-up outside capture (module load, occupancy)
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._engine_step()

    def step(self) -> None:
        if self.use_graph and self.graph is None:
            self._capture()
        with torch.cuda.stream(self.stream):
            self.d_jobs.copy_(self.h_jobs, non_blocking=True)
            self.d_slots.copy_(self.h_slots, non_blocking=True)
            self.d_count.copy_(self.h_count, non_blocking=True)
            if self.use_graph:
                self.graph.replay()
            else:
                self._engine_step()
            self.h_state.copy_(self.state, non_blocking=True)
        self.stream.synchronize()

    def job_for(self, r: Request, slot: int) -> dpc.Job:
        out = self.out[slot].data_ptr()
        if r.kind == dpc.JOB_SSSP:
            g = self.graphs[r.problem]
            return dpc.Job(dpc.JOB_SSSP, g.n, g.m, r.source, g.off.data_ptr(), g.col.data_ptr() if g.m else 0,
                           g.w.data_ptr() if g.m else 0, out)
        t = self.trees[r.problem]
        return dpc.Job(r.kind, t.n, t.m, r.source, t.off.data_ptr(), t.col.data_ptr(), 0, out)

    def run(self, requests: Sequence[Request], on_done=None) -> ServeResult:
        """Serve a request stream in arrival order; `on_done(i, slot)` is called
        when request i's results sit in self.out[slot] (before the slot is reused)."""
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        n = len(requests)
        admitted = np.zeros(n)
        finished = np.zeros(n)
        slot_of = np.full(n, -1, np.int64)
        free = list(range(self.slots))
        running = {}
        nxt = 0
        steps = 0
        jobs_view = self.h_jobs.numpy()
        t0 = time.perf_counter()
        while nxt < n or running:
            now = time.perf_counter() - t0
            if not running and nxt < n and requests[order[nxt]].arrival > now:
                time.sleep(min(requests[order[nxt]].arrival - now, 0.001))
                continue
            new = []
            while nxt < n and free and requests[order[nxt]].arrival <= now:
                i = order[nxt]
                s = free.pop()
                new.append((i, s))
                nxt += 1
            if new:
                raw = dpc.pack_jobs([self.job_for(requests[i], s) for i, s in new])
                jobs_view[:len(raw)] = np.frombuffer(raw, dtype=np.uint8)
                self.h_slots[:len(new)] = torch.tensor([s for _, s in new], dtype=torch.int32)
                for i, s in new:
                    running[s] = i
                    admitted[i] = now
                    slot_of[i] = s
            self.h_count[0] = len(new)
            self.step()
            steps += 1
            t_done = time.perf_counter() - t0
            state = self.h_state.numpy()
            for s in [s for s in running if state[s] == 2]:
                i = running.pop(s)
                finished[i] = t_done
                if on_done is not None:
                    on_done(i, s)
                free.append(s)
        makespan = time.perf_counter() - t0
        return ServeResult(admitted, finished, steps, self.slots, makespan, dpc.read_stats(self.stats).status, slot_of)


class ResidentServer(Server):
    """Server whose engine stays resident: arrivals are folded into the running
    kernel through its mailbox (dpc_engine_serve). The kernel returns when it
    has been idle for `limit_us` (or is asked to stop at the end of a stream);
    the loop launches it again when work arrives after that."""

    def __init__(self, graphs: Sequence[Resident], trees: Sequence[Resident], slots: Optional[int] = None,
                 tuning: Optional[dpc.Tuning] = None, memory_fraction: float = 0.5, max_slots: int = 128,
                 limit_us: int = 100_000):
        self.limit_us = int(limit_us)
        super().__init__(graphs, trees, slots=slots, waves_per_step=1, tuning=tuning,
                         memory_fraction=memory_fraction, max_slots=max_slots, use_graph=False)
        self.launches = 0

    def reset(self) -> None:
        # the kernel reports admissions and completions here, in pinned host memory
        self.state_host = torch.zeros(self.slots, dtype=torch.int32).pin_memory()
        self.mailbox = dpc.Mailbox()
        # result reads while the kernel runs: a side stream and a pinned buffer, made
        # here because allocating page-locked memory can serialise streams
        self.side = torch.cuda.Stream()
        self.read_buf = torch.empty(self.max_n, dtype=torch.int32).pin_memory()
        with torch.cuda.stream(self.stream):
            dpc.engine_init(self.ws, self.slots, self.max_n, self.max_m, self.state_host, self.tuning)
        self.stream.synchronize()

    def _launch(self) -> None:
        dpc.engine_serve(self.ws, self.slots, self.max_n, self.max_m, self.mailbox, self.limit_us, self.state_host,
                         self.tuning, self.stats, self.stream)
        self.launches += 1

    def read_out(self, slot: int, n: int) -> np.ndarray:
        """A copy of slot `slot`'s first n results (int32), read on the side
        stream (the kernel's stream is busy while it runs)."""
        with torch.cuda.stream(self.side):
            self.read_buf[:n].copy_(self.out[slot, :n], non_blocking=True)
        self.side.synchronize()
        return self.read_buf[:n].numpy().copy()

    def run(self, requests: Sequence[Request], on_done=None) -> ServeResult:
        """Serve a request stream in arrival order; `on_done(i, slot)` is called
        when request i's results sit in self.out[slot] (read them with
        read_out: the kernel may still be running)."""
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        n = len(requests)
        admitted = np.zeros(n)
        finished = np.zeros(n)
        slot_of = np.full(n, -1, np.int64)
        free = list(range(self.slots))
        running = {}
        state = self.state_host.numpy()
        nxt = 0
        polls = 0
        self.stream.synchronize()  # no kernel of an earlier run is still on the mailbox
        self.mailbox.clear_stop()
        t0 = time.perf_counter()
        self._launch()
        while nxt < n or running:
            now = time.perf_counter() - t0
            posted = False
            while nxt < n and free and requests[order[nxt]].arrival <= now:
                i = order[nxt]
                s = free.pop()
                state[s] = 0  # before the post, whose release store orders it
                self.mailbox.post(self.job_for(requests[i], s), s)
                running[s] = i
                admitted[i] = now
                slot_of[i] = s
                nxt += 1
                posted = True
            if running:
                done = [s for s in np.nonzero(state == 2)[0].tolist() if s in running]
                if done:
                    t_done = time.perf_counter() - t0
                    for s in done:
                        i = running.pop(s)
                        finished[i] = t_done
                        if on_done is not None:
                            on_done(i, s)
                        free.append(s)
            polls += 1
            if (posted or (running and polls % 64 == 0)) and self.stream.query():
                # the kernel returned (its lifetime passed, or a device error): check, then relaunch
                st = dpc.read_stats(self.stats).status
                if st != dpc.OK:
                    raise dpc.DpcError(st, "resident engine")
                if any(state[s] != 2 for s in running) or nxt < n:
                    self._launch()
        self.mailbox.stop()
        self.stream.synchronize()
        makespan = time.perf_counter() - t0
        return ServeResult(admitted, finished, self.launches, self.slots, makespan,
                           dpc.read_stats(self.stats).status, slot_of)


def server_from_cache(cache, graphs: Sequence[Resident], trees: Sequence[Resident], sssp_fraction: float = 0.6,
                      resident: bool = False, **kw) -> "Server":
    """A Server (or, with resident=True, a ResidentServer, which has no steps)
    configured by the autotuner's entry for this request mix
    (autotune.tune_engine, stored under autotune.mix_key); the engine's
    default configuration when the cache holds none."""
    from . import autotune

    p = cache.lookup(autotune.mix_key(graphs, trees, sssp_fraction)) or dict(autotune.ENGINE_DEFAULT)
    if resident:
        return ResidentServer(graphs, trees, tuning=autotune.engine_tuning(p), **kw)
    return Server(graphs, trees, waves_per_step=p["waves"], tuning=autotune.engine_tuning(p), **kw)


def one_at_a_time(graphs: Sequence[Resident], trees: Sequence[Resident], requests: Sequence[Request],
                  level="grid", on_done=None) -> ServeResult:
    """Baseline: each request is one library call, waited for before the next."""
    max_n = max([r.n for r in list(graphs) + list(trees)] + [1])
    max_m = max([r.m for r in graphs] + [1])
    out = torch.empty(max_n, dtype=torch.int32, device="cuda")
    ws_sssp = torch.empty(dpc.sssp_workspace_size(max_n, max_m, level), dtype=torch.uint8, device="cuda")
    ws_tree = torch.empty(dpc.tree_workspace_size(max_n, level), dtype=torch.uint8, device="cuda")
    order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
    n = len(requests)
    admitted = np.zeros(n)
    finished = np.zeros(n)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for i in order:
        r = requests[i]
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        admitted[i] = time.perf_counter() - t0
        if r.kind == dpc.JOB_SSSP:
            g = graphs[r.problem]
            dpc.sssp(g.off, g.col, g.w, r.source, out[:g.n], level, workspace=ws_sssp)
        else:
            t = trees[r.problem]
            fn = dpc.tree_descendants if r.kind == dpc.JOB_TREE_DESCENDANTS else dpc.tree_height
            fn(t.off, t.col, r.source, out[:t.n], level, workspace=ws_tree)
        stream.synchronize()
        finished[i] = time.perf_counter() - t0
        if on_done is not None:
            on_done(i, out)
    return ServeResult(admitted, finished, len(order), 1, time.perf_counter() - t0)


def poisson_stream(rng: np.random.Generator, count: int, rate: float, n_graphs: int, n_trees: int,
                   graph_sources: Sequence[np.ndarray], sssp_fraction: float = 0.6) -> List[Request]:
    """Poisson arrivals (mean `rate` per second); SSSP with probability
    sssp_fraction, else tree descendants / heights half and half."""
    gaps = rng.exponential(1.0 / rate, size=count) if rate > 0 else np.zeros(count)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(count):
        if rng.random() < sssp_fraction and n_graphs:
            p = int(rng.integers(0, n_graphs))
            src = int(rng.choice(graph_sources[p]))
            reqs.append(Request(dpc.JOB_SSSP, p, src, float(t[i])))
        else:
            p = int(rng.integers(0, n_trees))
            kind = dpc.JOB_TREE_DESCENDANTS if rng.random() < 0.5 else dpc.JOB_TREE_HEIGHT
            reqs.append(Request(kind, p, 0, float(t[i])))
    return reqs
