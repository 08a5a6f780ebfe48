"""Do the oracle's pins catch plausible mistakes? Each case rebuilds
dpc_oracle.c with one slip planted (a dropped term, a comparison off by one, a
Gauss-Seidel read where the round is Jacobi, a wrong modulus, a LIFO where the
search is FIFO, a split that is not aligned to its bucket), binds the broken
copy in place of the real oracle and runs the CPU pins of the function it
touches: at least one pin must fail. The unmodified oracle passes every one of
them (the regular CPU tests). Every planted slip keeps the oracle's memory
accesses in bounds, so a broken copy fails a pin instead of the process."""
import inspect
import os
import subprocess

import pytest

import oracle
from tests import (test_oracle_bfs, test_oracle_launches, test_oracle_pagerank, test_oracle_spmv, test_oracle_sssp,
                   test_oracle_tree)

# name: (text in dpc_oracle.c, planted replacement, pin modules)
MUTANTS = {
    # per-depth recursion counts (Sec. IV.B): the counts the tree launch tests rely on
    "tree_levels_internal_counts_leaves": ("if (k > 0) internal[L]++;", "if (k >= 0) internal[L]++;",
                                           [test_oracle_tree]),
    "tree_levels_heavy_at_threshold": ("if (k > threshold) heavy[L]++;", "if (k >= threshold) heavy[L]++;",
                                       [test_oracle_tree]),
    "tree_levels_edges_once_per_node": ("edges[L] += k;", "edges[L] += (k > 0);", [test_oracle_tree]),
    "tree_descendants_drop_child_itself": ("s += 1 + (uint64_t)desc[cidx[k]];", "s += (uint64_t)desc[cidx[k]];",
                                           [test_oracle_tree]),
    "tree_height_drop_plus_one": ("int32_t hc = 1 + height[cidx[k]];", "int32_t hc = height[cidx[k]];",
                                  [test_oracle_tree]),
    # SSSP
    "dijkstra_max_heap": ("if (h[p].d <= h[i].d) break;", "if (h[p].d >= h[i].d) break;", [test_oracle_sssp]),
    "frontier_reads_live_distance": ("int32_t u = F[i];\n      for (int64_t e = off[u]; e < off[u + 1]; ++e) {\n"
                                     "        int32_t v = col[e];\n        uint64_t nd = dprev[u] + (uint64_t)w[e];",
                                     "int32_t u = F[i];\n      for (int64_t e = off[u]; e < off[u + 1]; ++e) {\n"
                                     "        int32_t v = col[e];\n        uint64_t nd = d[u] + (uint64_t)w[e];",
                                     [test_oracle_sssp]),
    "nearfar_reads_live_distance": ("int32_t u = act[i];\n      for (int64_t e = off[u]; e < off[u + 1]; ++e) {\n"
                                    "        int32_t v = col[e];\n        uint64_t nd = dprev[u] + (uint64_t)w[e];",
                                    "int32_t u = act[i];\n      for (int64_t e = off[u]; e < off[u + 1]; ++e) {\n"
                                    "        int32_t v = col[e];\n        uint64_t nd = d[u] + (uint64_t)w[e];",
                                    [test_oracle_sssp]),
    "frontier_heavy_at_threshold": ("off[F[i] + 1] - off[F[i]] > threshold) hv++;",
                                    "off[F[i] + 1] - off[F[i]] >= threshold) hv++;", [test_oracle_sssp]),
    # the near-far split and the sub-split
    "nearfar_live_far_vertex_dropped": ("if (d[v] < S_old) { in_far[v] = 0; continue; }",
                                        "if (d[v] <= S_old) { in_far[v] = 0; continue; }", [test_oracle_sssp]),
    "nearfar_split_not_bucket_aligned": ("S = (dmin / delta + 1) * (uint64_t)delta;", "S = dmin + delta;",
                                         [test_oracle_sssp]),
    "subsplit_light_bound": ("if (off[v + 1] - off[v] <= threshold || d[v] < s) act[na++] = v;",
                             "if (off[v + 1] - off[v] < threshold || d[v] < s) act[na++] = v;", [test_oracle_sssp]),
    "subsplit_not_bucket_aligned": ("s = (hmin / sub_delta + 1) * (uint64_t)sub_delta;", "s = hmin + sub_delta;",
                                    [test_oracle_sssp]),
    # SpMV
    "spmv_signed_row_scale": ("a += p < 0 ? -p : p;", "a += p;", [test_oracle_spmv]),
    "spmv_single_precision_sum": ("double s = 0.0, a = 0.0;", "float s = 0.0f; double a = 0.0;",
                                  [test_oracle_spmv]),
    # launch counts of one parent grid (Sec. IV.B)
    "launches_items_wrapped_by_block": ("int64_t g = i % G;", "int64_t g = i % threads;", [test_oracle_launches]),
    # PageRank
    "pagerank_damping_swapped": ("(1.0 - d) / (double)n + d * (", "d / (double)n + (1.0 - d) * (",
                                 [test_oracle_pagerank]),
    "pagerank_dangling_dropped": ("d * (dangling / (double)n + next[v])", "d * (next[v])", [test_oracle_pagerank]),
    # BFS
    "bfs_lifo": ("const int32_t u = queue[head++];", "const int32_t u = queue[--tail];", [test_oracle_bfs]),
}


def pin_calls(module):
    """Every test function of `module` with each parameter set of its
    parametrize marks (the oracle pin tests take no fixtures)."""
    for name, fn in inspect.getmembers(module, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != module.__name__:
            continue
        params = inspect.signature(fn).parameters
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        if not params:
            yield name, fn, {}
            continue
        assert len(marks) == 1, name
        argnames, values = marks[0].args[0], marks[0].args[1]
        names = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
        for v in values:
            yield name, fn, dict(zip(names, v if len(names) > 1 else (v,)))


def build_mutant(tmp_path, key, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"{key}: the planted text must occur exactly once"
    c = tmp_path / f"{key}.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / f"lib{key}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(c), "-o", str(so)])
    return str(so)


@pytest.mark.parametrize("key", sorted(MUTANTS))
def test_pins_catch_planted_mistake(tmp_path, key):
    old, new, modules = MUTANTS[key]
    lib = oracle.load_variant(build_mutant(tmp_path, key, old, new))
    oracle._load()
    saved, oracle._lib = oracle._lib, lib
    failed = []
    try:
        for module in modules:
            for name, fn, kw in pin_calls(module):
                try:
                    fn(**kw)
                except (AssertionError, ValueError) as e:  # a pin failed, or the oracle refused its own input
                    failed.append((name, kw, type(e).__name__))
    finally:
        oracle._lib = saved
    assert failed, f"no pin caught the planted mistake {key!r}"


def test_pin_runner_passes_on_the_real_oracle():
    for module in (test_oracle_tree, test_oracle_launches):
        calls = list(pin_calls(module))
        assert calls
        for name, fn, kw in calls:
            fn(**kw)
    assert os.path.exists(oracle._LIB)
