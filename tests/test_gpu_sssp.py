"""GPU parity of dpc_sssp against the oracle (bit-exact distances) at every level."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1606_08150_gb300 import gen
from tests.gpu_util import dev, level_names_with_queue, u32

pytestmark = pytest.mark.gpu
LEVELS = level_names_with_queue()
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run(dpc, g, source, level, tuning=None, stats=False, offset=0):
    off = dev(g.off)
    if offset:
        col = dev(np.concatenate([np.zeros(offset, np.int32), g.col]))[offset:]
        w = dev(np.concatenate([np.zeros(offset, np.uint32), g.w]))[offset:]
    else:
        col, w = dev(g.col), dev(g.w)
    dist = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    st = dpc.new_stats() if stats else None
    status = dpc.sssp(off, col, w, source, dist, level, tuning=tuning, stats=st)
    torch.cuda.synchronize()
    return u32(dist), status, (dpc.read_stats(st) if stats else None)


def graph_from_edges(n, edges):
    edges = sorted(edges)
    off = np.zeros(n + 1, np.int64)
    for u, _, _ in edges:
        off[u + 1] += 1
    return gen.Graph(np.cumsum(off).astype(np.int32), np.array([e[1] for e in edges], np.int32),
                     np.array([e[2] for e in edges], np.uint32))


@pytest.mark.parametrize("level", LEVELS)
def test_hand_worked_instance(dpc, level):
    d = json.load(open(os.path.join(GOLDEN, "sssp_hand.json")))
    g = graph_from_edges(d["n"], d["edges"])
    dist, status, st = run(dpc, g, d["source"], level, tuning=dpc.Tuning(threshold=d["threshold"]), stats=True)
    assert status == dpc.OK
    assert dist.tolist() == d["dist"]
    assert st.rounds == len(d["frontier_size"])
    assert st.relaxations == d["relaxations"]


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_multigraphs(dpc, level, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 3000))
    g = gen.random_graph(n, int(rng.integers(0, 20 * n)), 1, 1000, seed=seed)
    src = int(rng.integers(0, n))
    want = oracle.sssp_dijkstra(g.off, g.col, g.w, src)
    dist, status, _ = run(dpc, g, src, level, tuning=dpc.Tuning(threshold=8))
    assert status == dpc.OK
    assert np.array_equal(dist, want)


@pytest.mark.parametrize("level", LEVELS)
def test_rmat_scale12_stats_match_oracle_rounds(dpc, level):
    """R-MAT scale 12, edge factor 16, weights in [1,100], source 0."""
    g = gen.rmat(12, seed=1)
    thr = 32
    fr = oracle.sssp_frontier(g.off, g.col, g.w, 0, thr)
    dist, status, st = run(dpc, g, 0, level, tuning=dpc.Tuning(threshold=thr), stats=True)
    assert status == dpc.OK and st.status == 0
    assert np.array_equal(dist, oracle.sssp_dijkstra(g.off, g.col, g.w, 0))
    assert st.rounds == fr.rounds
    assert st.relaxations == fr.relaxations
    assert st.launch_failures == 0
    if level in ("flat", "queue"):
        assert st.child_launches == 0  # flat: no device launches; queue: queue tasks instead
    elif level == "basic_dp":
        assert st.child_launches == int(fr.heavy.sum())
    elif level == "grid":
        assert st.child_launches == int((fr.heavy > 0).sum())
    else:
        assert int((fr.heavy > 0).sum()) <= st.child_launches <= int(fr.heavy.sum())
    if level not in ("flat", "queue"):
        assert st.buffered_items == int(fr.heavy.sum())


@pytest.mark.parametrize("level", LEVELS)
def test_edge_cases(dpc, level):
    # single vertex, no edges
    g = gen.Graph(np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    dist, status, _ = run(dpc, g, 0, level)
    assert status == dpc.OK and dist.tolist() == [0]
    # isolated source amid edges elsewhere
    g = graph_from_edges(4, [(1, 2, 3), (2, 3, 4), (3, 1, 1)])
    dist, _, _ = run(dpc, g, 0, level)
    assert dist.tolist() == [0, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]
    # a hub with every edge duplicated and self-loops, thresholds at both extremes, tiny chunks
    n = 2000
    edges = [(0, v, 1 + (v * 7) % 50) for v in range(1, n)] * 2 + [(v, v, 1) for v in range(n)]
    edges += [(v, v + 1, 3) for v in range(1, n - 1)]
    g = graph_from_edges(n, edges)
    want = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
    for t in (dpc.Tuning(threshold=-1), dpc.Tuning(threshold=2**31 - 1), dpc.Tuning(chunk=5, threshold=3)):
        dist, status, _ = run(dpc, g, 0, level, tuning=t)
        assert status == dpc.OK and np.array_equal(dist, want)


@pytest.mark.parametrize("level", LEVELS)
def test_unaligned_and_small_blocks(dpc, level):
    g = gen.rmat(10, seed=4)
    want = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
    dist, status, _ = run(dpc, g, 0, level, offset=1,
                          tuning=dpc.Tuning(parent_threads=32, child_threads=64, threshold=4))
    assert status == dpc.OK and np.array_equal(dist, want)


@pytest.mark.parametrize("level", ["warp", "block", "grid"])
def test_device_heap_buffers(dpc, level):
    """FLAG_DEVICE_MALLOC, the allocator study of Sec. V.A (Fig. 5): the warp
    and block levels take every consolidation buffer from device malloc(), the
    grid level ignores the flag. Distances, rounds, relaxations and buffered
    items are those of the pool; 300 calls in a row would exhaust the 8 MB
    device heap if the children did not free their buffers."""
    g = gen.rmat(13, seed=1)
    thr = 32
    fr = oracle.sssp_frontier(g.off, g.col, g.w, 0, thr)
    want = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
    off, col, w = dev(g.off), dev(g.col), dev(g.w)
    dist = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    t = dpc.Tuning(threshold=thr, flags=dpc.FLAG_DEVICE_MALLOC)
    ws = torch.empty(dpc.sssp_workspace_size(g.n, g.m, level, t), dtype=torch.uint8, device="cuda")
    sts = [dpc.new_stats() for _ in range(300)]
    for st in sts:
        assert dpc.sssp(off, col, w, 0, dist, level, tuning=t, workspace=ws, stats=st) == dpc.OK
    torch.cuda.synchronize()
    assert np.array_equal(u32(dist), want)
    for st in sts:
        s = dpc.read_stats(st)
        assert s.status == 0 and s.launch_failures == 0
        assert (s.rounds, s.relaxations, s.buffered_items) == (fr.rounds, fr.relaxations, int(fr.heavy.sum()))
        if level == "grid":
            assert s.child_launches == int((fr.heavy > 0).sum())
        else:
            assert int((fr.heavy > 0).sum()) <= s.child_launches <= int(fr.heavy.sum())


def test_deterministic_stats(dpc):
    g = gen.rmat(11, seed=7)
    for level in ("grid", "basic_dp"):
        a = run(dpc, g, 0, level, stats=True)[2]
        b = run(dpc, g, 0, level, stats=True)[2]
        assert (a.rounds, a.relaxations, a.child_launches, a.buffered_items) == \
               (b.rounds, b.relaxations, b.child_launches, b.buffered_items)


@pytest.mark.parametrize("level", ["grid", "block", "warp", "flat", "basic_dp", "queue"])
def test_full_size_rmat22(dpc, level, rmat22):
    """R-MAT scale 22 (4,194,304 vertices, 67,108,864 edges, weights in [1,1000]),
    all 8 sources of the configuration, the graph loaded once."""
    g, sources, wants = rmat22
    off, col, w = dev(g.off), dev(g.col), dev(g.w)
    dist = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    ws = torch.empty(dpc.sssp_workspace_size(g.n, g.m, level), dtype=torch.uint8, device="cuda")
    for src, want in zip(sources, wants):
        st = dpc.new_stats()
        dist.fill_(-7)
        assert dpc.sssp(off, col, w, src, dist, level, workspace=ws, stats=st) == dpc.OK
        torch.cuda.synchronize()
        assert np.array_equal(u32(dist), want), src
        assert dpc.read_stats(st).status == 0


@pytest.fixture(scope="module")
def rmat22():
    from concurrent.futures import ThreadPoolExecutor

    g = gen.rmat(22, whi=1000, seed=2)
    deg = np.diff(g.off)
    rng = np.random.default_rng(2)
    sources = [int(s) for s in rng.choice(np.nonzero(deg > 0)[0], 8, replace=False)]
    # the oracle is one C call per source; ctypes releases the GIL, so threads run them side by side
    with ThreadPoolExecutor(8) as ex:
        wants = list(ex.map(lambda s: oracle.sssp_dijkstra(g.off, g.col, g.w, s), sources))
    return g, sources, wants


# ---------------------------------------------------------------- near-far split

NEARFAR = [(10, 0), (10, 2), (0, 3), (1, 0)]  # (delta, sub_delta)


@pytest.mark.parametrize("level", LEVELS)
def test_hand_worked_near_far(dpc, level):
    d = json.load(open(os.path.join(GOLDEN, "sssp_hand.json")))
    g = graph_from_edges(d["n"], d["edges"])
    for delta, want in d["nearfar"].items():
        t = dpc.Tuning(threshold=d["threshold"], delta=int(delta))
        dist, status, st = run(dpc, g, d["source"], level, tuning=t, stats=True)
        assert status == dpc.OK and st.status == 0
        assert dist.tolist() == d["dist"]
        assert st.rounds == len(want["frontier_size"]), delta
        assert st.relaxations == want["relaxations"], delta


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("scale,whi,delta,sub", [(12, 100, 20, 2), (12, 100, 7, 0), (13, 1000, 150, 8),
                                                 (12, 100, 0, 4)])
def test_rmat_near_far_stats_match_oracle(dpc, level, scale, whi, delta, sub):
    """Rounds, relaxations and launch counts of the near-far rounds equal the
    oracle's (Davidson et al.'s split, with the sub-split for heavy vertices)."""
    g = gen.rmat(scale, whi=whi, seed=scale)
    thr = 32
    fr = oracle.sssp_nearfar(g.off, g.col, g.w, 0, delta, thr, sub)
    t = dpc.Tuning(threshold=thr, delta=delta, sub_delta=sub)
    dist, status, st = run(dpc, g, 0, level, tuning=t, stats=True)
    assert status == dpc.OK and st.status == 0
    assert np.array_equal(dist, oracle.sssp_dijkstra(g.off, g.col, g.w, 0))
    assert np.array_equal(dist, fr.dist)
    assert st.rounds == fr.rounds
    assert st.relaxations == fr.relaxations
    assert st.launch_failures == 0
    if level in ("flat", "queue"):
        assert st.child_launches == 0
    elif level == "basic_dp":
        assert st.child_launches == int(fr.heavy.sum())
    elif level == "grid":
        assert st.child_launches == int((fr.heavy > 0).sum())
    else:
        assert int((fr.heavy > 0).sum()) <= st.child_launches <= int(fr.heavy.sum())
    if level not in ("flat", "queue"):
        assert st.buffered_items == int(fr.heavy.sum())


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("seed", [3, 4])
def test_random_multigraphs_near_far(dpc, level, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 3000))
    g = gen.random_graph(n, int(rng.integers(0, 20 * n)), 0, 1000, seed=seed)  # zero weights allowed
    src = int(rng.integers(0, n))
    want = oracle.sssp_dijkstra(g.off, g.col, g.w, src)
    for delta, sub in NEARFAR:
        t = dpc.Tuning(threshold=8, delta=delta, sub_delta=sub)
        fr = oracle.sssp_nearfar(g.off, g.col, g.w, src, delta, 8, sub)
        dist, status, st = run(dpc, g, src, level, tuning=t, stats=True)
        assert status == dpc.OK and st.status == 0
        assert np.array_equal(dist, want), (delta, sub)
        assert (st.rounds, st.relaxations) == (fr.rounds, fr.relaxations), (delta, sub)


@pytest.mark.parametrize("level", LEVELS)
def test_near_far_edge_cases(dpc, level):
    t = dpc.Tuning(delta=5, sub_delta=1, threshold=2)
    g = gen.Graph(np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    dist, status, _ = run(dpc, g, 0, level, tuning=t)
    assert status == dpc.OK and dist.tolist() == [0]
    g = graph_from_edges(4, [(1, 2, 3), (2, 3, 4), (3, 1, 1)])
    dist, _, _ = run(dpc, g, 0, level, tuning=t)
    assert dist.tolist() == [0, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]
    # a hub with duplicated edges and self-loops; widths of one, far above every distance, tiny chunks
    n = 2000
    edges = [(0, v, 1 + (v * 7) % 50) for v in range(1, n)] * 2 + [(v, v, 1) for v in range(n)]
    edges += [(v, v + 1, 3) for v in range(1, n - 1)]
    g = graph_from_edges(n, edges)
    want = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
    for tu in (dpc.Tuning(delta=1, sub_delta=1, threshold=-1), dpc.Tuning(delta=1 << 30, threshold=3, chunk=5),
               dpc.Tuning(delta=3, sub_delta=2, threshold=2**31 - 1)):
        dist, status, st = run(dpc, g, 0, level, tuning=tu, stats=True)
        assert status == dpc.OK and np.array_equal(dist, want)
        fr = oracle.sssp_nearfar(g.off, g.col, g.w, 0, tu.delta, max(tu.threshold, 0), tu.sub_delta)
        assert (st.rounds, st.relaxations) == (fr.rounds, fr.relaxations)
    # unaligned arrays and small blocks
    g = gen.rmat(10, seed=4)
    dist, status, _ = run(dpc, g, 0, level, offset=1,
                          tuning=dpc.Tuning(parent_threads=32, child_threads=64, threshold=4, delta=9, sub_delta=2))
    assert status == dpc.OK and np.array_equal(dist, oracle.sssp_dijkstra(g.off, g.col, g.w, 0))


@pytest.mark.parametrize("level", ["grid", "block", "warp", "flat", "basic_dp", "queue"])
def test_full_size_rmat22_near_far(dpc, level, rmat22):
    """R-MAT scale 22 on all 8 sources with the near-far split of width 200 and
    the heavy-vertex sub-split of width 8: the same distances as Dijkstra."""
    g, sources, wants = rmat22
    off, col, w = dev(g.off), dev(g.col), dev(g.w)
    dist = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    t = dpc.Tuning(delta=200, sub_delta=8)
    ws = torch.empty(dpc.sssp_workspace_size(g.n, g.m, level, t), dtype=torch.uint8, device="cuda")
    for src, want in zip(sources, wants):
        st = dpc.new_stats()
        dist.fill_(-7)
        assert dpc.sssp(off, col, w, src, dist, level, tuning=t, workspace=ws, stats=st) == dpc.OK
        torch.cuda.synchronize()
        assert np.array_equal(u32(dist), want), src
        s = dpc.read_stats(st)
        assert s.status == 0
        reach = int(np.diff(g.off)[want != 0xFFFFFFFF].sum())
        assert s.relaxations <= 1.5 * reach, (src, s.relaxations / reach)
