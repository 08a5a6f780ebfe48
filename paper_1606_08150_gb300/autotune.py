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
        return grid_space(chunk=(1024, 2048, 4096, 8192), child_threads=(128, 256, 512),
                          kc=(KC_RULE.get(level, 1), max(1, KC_RULE.get(level, 1) // 4)))
    if app == "sssp":
        return grid_space(threshold=(16, 32, 64), chunk=(128, 256, 1024), kc=(KC_RULE.get(level, 1),))
    return grid_space(chunk=(8, 32, 128), child_threads=(128, 256), kc=(KC_RULE.get(level, 1),))
