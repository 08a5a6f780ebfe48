"""Autotuning of launch configuration and consolidation knobs.

The paper configures consolidated child kernels by the KC_X rule: take the
occupancy-maximising grid of B blocks and launch ceil(B/X) of them, with
X = 1 for grid-level, 16 for block-level and 32 for warp-level consolidation
(Sec. IV.E), and compares that rule with an exhaustive search over
configurations (Sec. V.B, Fig. 6). This module is the systematic form of that
search: it times every candidate of a search space on the device (CUDA
events on the calling stream, median of several runs) and returns the best,
and `kc_study` reports how close the KC_X rule comes to the searched optimum.

Results can be cached per workload key (application, level, size class) in
memory and in a JSON file.
"""
from __future__ import annotations

import itertools
import json
import os
from dataclasses import dataclass
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import dpc

KC_RULE = {"grid": 1, "block": 16, "warp": 32}


@dataclass
class Trial:
    params: Dict[str, int]
    ms: float


def time_call(fn: Callable[[], None], reps: int = 5, warmup: int = 2) -> float:
    """Median device time of fn() in ms, CUDA events on the current stream."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def grid_space(**axes: Sequence[int]) -> List[Dict[str, int]]:
    """Cartesian product of named axes (values of dpc.Tuning fields)."""
    names = list(axes)
    return [dict(zip(names, vals)) for vals in itertools.product(*(axes[n] for n in names))]


def search(run: Callable[[dpc.Tuning], None], space: Iterable[Dict[str, int]], reps: int = 5
           ) -> Tuple[Dict[str, int], List[Trial]]:
    """Time run(Tuning(**params)) for every candidate; return the fastest and all trials."""
    trials = []
    for params in space:
        t = dpc.Tuning(**params)
        trials.append(Trial(dict(params), time_call(lambda: run(t), reps)))
    best = min(trials, key=lambda tr: tr.ms)
    return best.params, trials


# child_blocks that no buffer reaches: the child grid is then sized by the
# buffer alone, one warp per buffered unit (the paper's "1-1 mapping", Sec. V.B)
ONE_TO_ONE_BLOCKS = 1 << 30
DEFAULT_CHILD_THREADS = 256


def kc_study(run_level: Callable[[str, dpc.Tuning], None], levels: Sequence[str] = ("grid", "block", "warp"),
             kcs: Sequence[int] = (1, 2, 4, 8, 16, 32, 64), child_threads: Sequence[int] = (128, 256, 512),
             reps: int = 5, passes: int = 2) -> Dict[str, Dict[str, float]]:
    """Fig. 6's comparison, in kind, for every level: the KC_X rule's
    configuration (X of the level, default child blocks of 256 threads), the
    1-1 mapping (as many child warps as buffered units, whatever the
    occupancy) and the best configuration of an exhaustive search over (X,
    child threads). All candidates are timed in the same sweep, `passes` times
    in interleaved order, keeping each one's fastest median; the rule is one of
    the searched candidates, so the search never reports worse than the rule."""
    out = {}
    for level in levels:
        rule = {"kc": KC_RULE[level], "child_threads": DEFAULT_CHILD_THREADS}
        space = grid_space(kc=kcs, child_threads=child_threads)
        if rule not in space:
            space.append(rule)
        one = {"child_blocks": ONE_TO_ONE_BLOCKS, "child_threads": DEFAULT_CHILD_THREADS}
        cands = space + [one]
        best_ms = [float("inf")] * len(cands)
        for k in range(passes):
            order = range(len(cands)) if k % 2 == 0 else reversed(range(len(cands)))
            for i in order:
                t = dpc.Tuning(**cands[i])
                best_ms[i] = min(best_ms[i], time_call(lambda: run_level(level, t), reps))
        searched = best_ms[:len(space)]
        ib = int(np.argmin(searched))
        t_rule = searched[space.index(rule)]
        t_best = searched[ib]
        t_one = best_ms[-1]
        out[level] = {"rule_kc": KC_RULE[level], "rule_ms": round(t_rule, 4), "best_ms": round(t_best, 4),
                      "best": space[ib], "rule_fraction_of_best": round(t_best / t_rule, 4),
                      "one_to_one_ms": round(t_one, 4), "one_to_one_fraction_of_best": round(t_best / t_one, 4)}
    return out


class Cache:
    """Best parameters per workload key, kept in memory and optionally in a JSON file."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.table: Dict[str, Dict[str, int]] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    @staticmethod
    def key(app: str, level: str, size: int) -> str:
        return f"{app}/{level}/2^{max(0, int(size).bit_length() - 1)}"

    def lookup(self, key: str) -> Optional[Dict[str, int]]:
        """The raw parameters stored under `key` (any workload key), or None."""
        p = self.table.get(key)
        return dict(p) if p is not None else None

    def store(self, key: str, params: Dict[str, int]) -> None:
        self.table[key] = dict(params)
        if self.path:
            with open(self.path, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)

    def get(self, app: str, level: str, size: int) -> Optional[dpc.Tuning]:
        p = self.table.get(self.key(app, level, size))
        return dpc.Tuning(**p) if p is not None else None

    def tune(self, app: str, level: str, size: int, run: Callable[[dpc.Tuning], None],
             space: Iterable[Dict[str, int]], reps: int = 5) -> dpc.Tuning:
        k = self.key(app, level, size)
        if k not in self.table:
            best, _ = search(run, space, reps)
            self.table[k] = best
            if self.path:
                with open(self.path, "w") as f:
                    json.dump(self.table, f, indent=1, sort_keys=True)
        return dpc.Tuning(**self.table[k])


def default_space(app: str, level: str) -> List[Dict[str, int]]:
    """Search space per application and level (threshold, chunk, child shape)."""
    if app == "spmv":
        return grid_space(chunk=(512, 1024, 2048, 4096, 8192), child_threads=(128, 256, 512),
                          kc=(KC_RULE.get(level, 1), max(1, KC_RULE.get(level, 1) // 4)))
    if app == "sssp":
        return grid_space(threshold=(16, 32, 64), chunk=(128, 256, 1024), kc=(KC_RULE.get(level, 1),))
    return grid_space(chunk=(8, 32, 128), child_threads=(128, 256), kc=(KC_RULE.get(level, 1),))


# ---------------------------------------------------------------- the batched engine

# The engine's knobs: threshold and chunk (how a large SSSP frontier vertex is
# split into EDGES tasks), the cooperative grid (parent_blocks, 0 = every
# resident block) and the waves an engine step runs before it returns to the
# request loop (waves). The default is the engine's own configuration.
ENGINE_DEFAULT = {"threshold": 32, "chunk": 512, "parent_blocks": 0, "waves": 32}


def engine_axes(sms: int) -> Dict[str, Sequence[int]]:
    """Values tried per knob (coordinate search around the default)."""
    return {"threshold": (16, 32, 64), "chunk": (256, 512, 1024), "parent_blocks": (0, 2 * sms, sms),
            "waves": (16, 32, 64)}


def engine_tuning(params: Dict[str, int]) -> dpc.Tuning:
    return dpc.Tuning(threshold=params["threshold"], chunk=params["chunk"], parent_blocks=params["parent_blocks"])


def mix_key(graphs, trees, sssp_fraction: float) -> str:
    """Cache key of a request mix: the SSSP share and the size classes of the
    resident graphs and trees."""
    gs = sorted({max(0, int(g.n).bit_length() - 1) for g in graphs})
    ts = sorted({max(0, int(t.n).bit_length() - 1) for t in trees})
    return (f"engine/sssp{int(round(100 * sssp_fraction))}/graphs2^{gs[0]}-2^{gs[-1]}/"
            f"trees2^{ts[0]}-2^{ts[-1]}" if gs and ts else "engine/empty")


def engine_throughput(graphs, trees, requests, params: Dict[str, int], slots: Optional[int] = None) -> float:
    """Requests per second of the engine serving `requests` with `params`
    (the arrivals as given; all at time 0 measures saturated throughput)."""
    from . import serve

    srv = serve.Server(graphs, trees, slots=slots, waves_per_step=params["waves"], tuning=engine_tuning(params))
    srv.run(requests[: min(32, len(requests))])  # warm-up: graph capture, module load
    srv.reset()
    res = srv.run(requests)
    if res.status != 0:
        raise RuntimeError(f"engine status {res.status} with {params}")
    return len(requests) / res.makespan


def tune_engine(graphs, trees, requests, sms: int, slots: Optional[int] = None, sweeps: int = 2
                ) -> Tuple[Dict[str, int], List[Trial]]:
    """Coordinate search over the engine's knobs on a request sample: starting
    from the default, each knob in turn takes the value with the highest
    throughput, the others fixed, for `sweeps` sweeps (or until nothing
    changes). Returns the best parameters and every trial (ms per request)."""
    best = dict(ENGINE_DEFAULT)
    seen: Dict[Tuple, float] = {}
    trials: List[Trial] = []

    def measure(p):
        k = tuple(sorted(p.items()))
        if k not in seen:
            seen[k] = engine_throughput(graphs, trees, requests, p, slots)
            trials.append(Trial(dict(p), 1e3 / seen[k]))
        return seen[k]

    best_rate = measure(best)
    axes = engine_axes(sms)
    for _ in range(sweeps):
        changed = False
        for knob, values in axes.items():
            for v in values:
                cand = dict(best, **{knob: v})
                rate = measure(cand)
                if rate > best_rate * 1.02:  # a clear gain only: the rates carry a few % of noise
                    best, best_rate, changed = cand, rate, True
        if not changed:
            break
    return best, trials
