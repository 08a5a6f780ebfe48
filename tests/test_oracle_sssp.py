"""Pins for the SSSP oracle (Dijkstra and frontier rounds) against facts that do
not come from the oracle itself: Floyd-Warshall on small random multigraphs, a
hand-worked instance, and the shortest-path optimality conditions."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1606_08150_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.INF


def csr_from_edges(n, edges):
    edges = sorted(edges, key=lambda e: (e[0], e[1], e[2]))
    off = np.zeros(n + 1, np.int32)
    for u, _, _ in edges:
        off[u + 1] += 1
    off = np.cumsum(off).astype(np.int32)
    col = np.array([e[1] for e in edges], np.int32)
    w = np.array([e[2] for e in edges], np.uint32)
    return off, col, w


def floyd_warshall(n, off, col, w):
    d = np.full((n, n), np.inf)
    np.fill_diagonal(d, 0.0)
    for u in range(n):
        for e in range(off[u], off[u + 1]):
            d[u, col[e]] = min(d[u, col[e]], float(w[e]))
    for k in range(n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return d


def as_u32(row):
    return np.array([INF if np.isinf(v) else int(v) for v in row], np.uint32)


@pytest.mark.parametrize("seed", range(12))
def test_dijkstra_and_frontier_match_floyd_warshall(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 65))
    m = int(rng.integers(0, 4 * n + 1))
    g = gen.random_graph(n, m, 1, int(rng.integers(1, 1000)), seed=seed)
    fw = floyd_warshall(n, g.off, g.col, g.w)
    for s in range(n):
        want = as_u32(fw[s])
        np.testing.assert_array_equal(oracle.sssp_dijkstra(g.off, g.col, g.w, s), want)
        np.testing.assert_array_equal(oracle.sssp_frontier(g.off, g.col, g.w, s, threshold=2).dist, want)


def test_hand_worked_instance():
    d = json.load(open(os.path.join(GOLDEN, "sssp_hand.json")))
    off, col, w = csr_from_edges(d["n"], d["edges"])
    np.testing.assert_array_equal(oracle.sssp_dijkstra(off, col, w, d["source"]), np.array(d["dist"], np.uint32))
    fr = oracle.sssp_frontier(off, col, w, d["source"], d["threshold"])
    np.testing.assert_array_equal(fr.dist, np.array(d["dist"], np.uint32))
    assert fr.frontier_size.tolist() == d["frontier_size"]
    assert fr.heavy.tolist() == d["heavy"]
    assert fr.relaxations == d["relaxations"]


def test_hand_worked_near_far():
    d = json.load(open(os.path.join(GOLDEN, "sssp_hand.json")))
    off, col, w = csr_from_edges(d["n"], d["edges"])
    for delta, want in d["nearfar"].items():
        r = oracle.sssp_nearfar(off, col, w, d["source"], int(delta), d["threshold"])
        np.testing.assert_array_equal(r.dist, np.array(d["dist"], np.uint32))
        assert r.frontier_size.tolist() == want["frontier_size"], delta
        assert r.heavy.tolist() == want["heavy"], delta
        assert (r.relaxations, r.splits) == (want["relaxations"], want["splits"]), delta


def test_hand_worked_sub_split():
    d = json.load(open(os.path.join(GOLDEN, "sssp_hand.json")))
    off, col, w = csr_from_edges(d["n"], d["edges"])
    for want in d["subsplit"]:
        r = oracle.sssp_nearfar(off, col, w, d["source"], want["delta"], d["threshold"], want["sub_delta"])
        np.testing.assert_array_equal(r.dist, np.array(d["dist"], np.uint32))
        assert r.frontier_size.tolist() == want["frontier_size"]
        assert r.heavy.tolist() == want["heavy"]
        assert (r.relaxations, r.splits, r.subsplits) == (want["relaxations"], want["splits"], want["subsplits"])


@pytest.mark.parametrize("scale,seed", [(8, 1), (11, 2)])
def test_sub_split_width_one_on_heavy_vertices_relaxes_each_once(scale, seed):
    """Every vertex heavy (threshold -1), no split, sub-split width 1, weights
    >= 1: a round relaxes exactly the vertices of the smallest pending
    distance, which are final, so the rounds are the distinct distances in
    increasing order and each sub-split advance opens the next one."""
    g = gen.rmat(scale, seed=seed)
    d = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
    deg = np.diff(g.off)
    reached = d != INF
    values, counts = np.unique(d[reached], return_counts=True)
    r = oracle.sssp_nearfar(g.off, g.col, g.w, 0, 0, -1, 1)
    np.testing.assert_array_equal(r.dist, d)
    assert r.frontier_size.tolist() == counts.tolist()
    assert r.heavy.tolist() == counts.tolist()
    assert r.relaxations == int(deg[reached].sum())
    assert (r.splits, r.subsplits) == (0, r.rounds - 1)


@pytest.mark.parametrize("scale,seed", [(10, 2), (12, 1)])
def test_sub_split_without_heavy_vertices_changes_nothing(scale, seed):
    """With a threshold above every out-degree no vertex is heavy: the runs with
    and without the sub-split are the same."""
    g = gen.rmat(scale, whi=1000, seed=seed)
    top = int(np.diff(g.off).max())
    for delta in (0, 60):
        a = oracle.sssp_nearfar(g.off, g.col, g.w, 0, delta, top, 0)
        b = oracle.sssp_nearfar(g.off, g.col, g.w, 0, delta, top, 7)
        assert a.frontier_size.tolist() == b.frontier_size.tolist()
        assert (a.relaxations, a.splits, b.subsplits) == (b.relaxations, b.splits, 0)


def test_sub_split_path_closed_form():
    # the path of test_near_far_path_closed_form with every vertex heavy: one vertex per round, and a
    # sub-split advance each time the next vertex lies above the current sub-bucket
    k = 40
    off, col, w = csr_from_edges(k, [(i, i + 1, i + 1) for i in range(k - 1)])
    want = np.array([j * (j + 1) // 2 for j in range(k)], np.uint32)
    for sub in (1, 3, 10, 100):
        r = oracle.sssp_nearfar(off, col, w, 0, 0, -1, sub)
        np.testing.assert_array_equal(r.dist, want)
        assert r.frontier_size.tolist() == [1] * k and r.relaxations == k - 1
        buckets = [int(x) // sub for x in want]
        assert r.subsplits == sum(1 for j in range(1, k) if buckets[j] != buckets[j - 1])


@pytest.mark.parametrize("seed", range(8))
def test_near_far_matches_floyd_warshall(seed):
    rng = np.random.default_rng(50 + seed)
    n = int(rng.integers(1, 65))
    g = gen.random_graph(n, int(rng.integers(0, 4 * n + 1)), 0 if seed % 3 == 0 else 1, int(rng.integers(1, 300)),
                         seed=seed)
    fw = floyd_warshall(n, g.off, g.col, g.w)
    for s in range(0, n, 3):
        for delta, sub in ((1, 0), (7, 0), (50, 3), (1 << 30, 0), (0, 2), (9, 1)):
            np.testing.assert_array_equal(oracle.sssp_nearfar(g.off, g.col, g.w, s, delta, 2, sub).dist,
                                          as_u32(fw[s]))


@pytest.mark.parametrize("scale,seed", [(8, 1), (10, 2), (12, 1)])
def test_near_far_width_one_relaxes_each_vertex_once(scale, seed):
    """Width 1 with weights >= 1: a bucket holds one distance value, whose
    vertices are final when it is relaxed (Dijkstra's argument), so each
    reached vertex is relaxed exactly once and the rounds are the distinct
    distances in increasing order."""
    g = gen.rmat(scale, seed=seed)
    assert g.w.min() >= 1
    d = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
    deg = np.diff(g.off)
    reached = d != INF
    values, counts = np.unique(d[reached], return_counts=True)
    thr = 20
    heavy = [int(((d == v) & (deg > thr)).sum()) for v in values]
    r = oracle.sssp_nearfar(g.off, g.col, g.w, 0, 1, thr)
    np.testing.assert_array_equal(r.dist, d)
    assert r.frontier_size.tolist() == counts.tolist()
    assert r.heavy.tolist() == heavy
    assert r.relaxations == int(deg[reached].sum())
    assert r.splits == r.rounds - 1


@pytest.mark.parametrize("scale,seed", [(9, 3), (12, 1)])
def test_near_far_without_a_split_is_the_plain_rounds(scale, seed):
    """delta = 0 (no split) and a width above every distance both leave the far
    pile empty: the frontier rounds exactly."""
    g = gen.rmat(scale, whi=1000, seed=seed)
    fr = oracle.sssp_frontier(g.off, g.col, g.w, 0, 32)
    for delta in (0, 1 << 31):
        r = oracle.sssp_nearfar(g.off, g.col, g.w, 0, delta, 32)
        np.testing.assert_array_equal(r.dist, fr.dist)
        assert r.frontier_size.tolist() == fr.frontier_size.tolist()
        assert r.heavy.tolist() == fr.heavy.tolist()
        assert (r.relaxations, r.splits) == (fr.relaxations, 0)


def test_near_far_path_closed_form():
    # path with weight i+1 on edge i: d(j) = j(j+1)/2, one vertex per round whatever the width
    k = 40
    off, col, w = csr_from_edges(k, [(i, i + 1, i + 1) for i in range(k - 1)])
    want = np.array([j * (j + 1) // 2 for j in range(k)], np.uint32)
    for delta in (1, 3, 10, 100):
        r = oracle.sssp_nearfar(off, col, w, 0, delta, 0)
        np.testing.assert_array_equal(r.dist, want)
        assert r.frontier_size.tolist() == [1] * k and r.relaxations == k - 1
        # a split each time the next vertex lies above the current bucket: the buckets of d(1)..d(k-1)
        # that differ from the bucket before them
        buckets = [int(x) // delta for x in want]
        assert r.splits == sum(1 for j in range(1, k) if buckets[j] != buckets[j - 1])


def check_optimality(off, col, w, src, dist):
    """d(src)=0; d(v) <= d(u)+w on every edge out of a reached u; every reached
    v != src has an in-edge with equality; unreached vertices have no edge from a
    reached vertex."""
    n = off.shape[0] - 1
    src_of = np.repeat(np.arange(n), np.diff(off))
    du = dist[src_of].astype(np.uint64)
    dv = dist[col].astype(np.uint64)
    reached = dist[src_of] != INF
    assert dist[src] == 0
    assert np.all(dv[reached] <= du[reached] + w[reached].astype(np.uint64))
    tight = reached & (dv == du + w.astype(np.uint64))
    has_tight = np.zeros(n, bool)
    has_tight[col[tight]] = True
    reach_v = (dist != INF)
    reach_v[src] = False
    assert np.all(has_tight[reach_v])
    assert np.all(dist[col[reached]] != INF)


@pytest.mark.parametrize("scale,seed", [(8, 1), (10, 2), (12, 1)])
def test_optimality_conditions_rmat(scale, seed):
    g = gen.rmat(scale, seed=seed)
    d = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
    check_optimality(g.off, g.col, g.w, 0, d)
    fr = oracle.sssp_frontier(g.off, g.col, g.w, 0, 32)
    np.testing.assert_array_equal(fr.dist, d)
    # the frontier run ends when a round improves nothing, and round 0 is {source}
    assert fr.frontier_size[0] == 1
    assert fr.relaxations >= int(np.diff(g.off)[d != INF].sum())


def test_optimality_check_catches_planted_error():
    g = gen.rmat(8, seed=3)
    d = oracle.sssp_dijkstra(g.off, g.col, g.w, 0).copy()
    v = int(np.nonzero((d != INF) & (d > 0))[0][0])
    d[v] += 1
    with pytest.raises(AssertionError):
        check_optimality(g.off, g.col, g.w, 0, d)


def test_path_closed_form():
    # path 0->1->...->k-1 with weight i+1 on edge i: d(j) = j(j+1)/2; one vertex per round
    k = 50
    edges = [(i, i + 1, i + 1) for i in range(k - 1)]
    off, col, w = csr_from_edges(k, edges)
    want = np.array([j * (j + 1) // 2 for j in range(k)], np.uint32)
    np.testing.assert_array_equal(oracle.sssp_dijkstra(off, col, w, 0), want)
    fr = oracle.sssp_frontier(off, col, w, 0, 0)
    np.testing.assert_array_equal(fr.dist, want)
    assert fr.rounds == k and fr.frontier_size.tolist() == [1] * k


def test_isolated_source_and_single_vertex():
    off, col, w = csr_from_edges(3, [(1, 2, 5)])
    np.testing.assert_array_equal(oracle.sssp_dijkstra(off, col, w, 0), np.array([0, INF, INF], np.uint32))
    off1 = np.zeros(2, np.int32)
    e = np.zeros(0, np.int32)
    np.testing.assert_array_equal(oracle.sssp_dijkstra(off1, e, e.astype(np.uint32), 0), np.array([0], np.uint32))


def test_distance_overflow_is_reported():
    off, col, w = csr_from_edges(3, [(0, 1, 0xFFFFFFF0), (1, 2, 0x20)])
    with pytest.raises(ValueError):
        oracle.sssp_dijkstra(off, col, w, 0)
    with pytest.raises(ValueError):
        oracle.sssp_frontier(off, col, w, 0, 0)
