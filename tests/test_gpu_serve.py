"""The continuous-batching request loop (paper_1606_08150_gb300.serve): every
request's result in the mixed, overlapping stream equals the oracle and the
result of serving it alone (one library call per request)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_08150_gb300 import dpc, gen, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    rng = np.random.default_rng(5)
    graphs, graphs_h, sources = [], [], []
    for i, scale in enumerate([8, 10, 11, 12, 13]):
        g = gen.rmat(scale, seed=100 + i)
        graphs_h.append(g)
        graphs.append(serve.upload_graph(g))
        sources.append(np.nonzero(np.diff(g.off) > 0)[0])
    trees, trees_h = [], []
    for i, n in enumerate([1000, 5000, 30000, 120000]):
        t = gen.tree(n, seed=200 + i, permute=bool(i % 2))
        trees_h.append(t)
        trees.append(serve.upload_tree(t))
    return graphs, graphs_h, sources, trees, trees_h


def expected(r, graphs_h, trees_h):
    if r.kind == dpc.JOB_SSSP:
        g = graphs_h[r.problem]
        return oracle.sssp_dijkstra(g.off, g.col, g.w, r.source).view(np.int32)
    t = trees_h[r.problem]
    if r.kind == dpc.JOB_TREE_DESCENDANTS:
        return oracle.tree_descendants(t.coff, t.cidx, 0).view(np.int32)
    return oracle.tree_height(t.coff, t.cidx, 0)


@pytest.mark.parametrize("rate,slots,waves,use_graph", [(20000.0, 6, 8, False), (20000.0, 6, 8, True),
                                                        (0.0, 16, 64, True)])
def test_mixed_stream_matches_alone_and_oracle(dpc, pool, rate, slots, waves, use_graph):
    graphs, graphs_h, sources, trees, trees_h = pool
    rng = np.random.default_rng(9)
    reqs = serve.poisson_stream(rng, 120, rate, len(graphs), len(trees), sources)
    srv = serve.Server(graphs, trees, slots=slots, waves_per_step=waves, use_graph=use_graph)
    got = {}

    def keep(i, s):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        got[i] = srv.out[s, :n].cpu().numpy().copy()

    res = srv.run(reqs, on_done=keep)
    assert res.status == 0
    assert len(got) == len(reqs)
    assert np.all(res.finished >= res.admitted)
    alone = {}

    def keep_alone(i, out):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        alone[i] = out[:n].cpu().numpy().copy()

    serve.one_at_a_time(graphs, trees, [serve.Request(r.kind, r.problem, r.source, 0.0) for r in reqs],
                        on_done=keep_alone)
    for i, r in enumerate(reqs):
        want = expected(r, graphs_h, trees_h)
        assert np.array_equal(got[i], want), i
        assert np.array_equal(alone[i], got[i]), i


@pytest.fixture(scope="module")
def pool_upper():
    """The served stream's size range up to its top (R-MAT 2^18, trees of 10^6 nodes)."""
    graphs, graphs_h, sources = [], [], []
    for i, scale in enumerate([10, 14, 18]):
        g = gen.rmat(scale, seed=300 + i)
        graphs_h.append(g)
        graphs.append(serve.upload_graph(g))
        sources.append(np.nonzero(np.diff(g.off) > 0)[0])
    trees, trees_h = [], []
    for i, n in enumerate([1000, 100_000, 1_000_000]):
        t = gen.tree(n, seed=400 + i, permute=bool(i % 2))
        trees_h.append(t)
        trees.append(serve.upload_tree(t))
    return graphs, graphs_h, sources, trees, trees_h


def test_upper_sizes_in_the_stream_match_alone_and_oracle(dpc, pool_upper):
    graphs, graphs_h, sources, trees, trees_h = pool_upper
    rng = np.random.default_rng(19)
    reqs = serve.poisson_stream(rng, 48, 5000.0, len(graphs), len(trees), sources)
    # every request on the largest graph and the largest tree is in the stream at least once
    reqs += [serve.Request(dpc.JOB_SSSP, 2, int(sources[2][7]), reqs[-1].arrival),
             serve.Request(dpc.JOB_TREE_DESCENDANTS, 2, 0, reqs[-1].arrival),
             serve.Request(dpc.JOB_TREE_HEIGHT, 2, 0, reqs[-1].arrival)]
    srv = serve.Server(graphs, trees, slots=8, waves_per_step=16)
    got = {}

    def keep(i, s):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        got[i] = srv.out[s, :n].cpu().numpy().copy()

    res = srv.run(reqs, on_done=keep)
    assert res.status == 0 and len(got) == len(reqs)
    alone = {}

    def keep_alone(i, out):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        alone[i] = out[:n].cpu().numpy().copy()

    serve.one_at_a_time(graphs, trees, [serve.Request(r.kind, r.problem, r.source, 0.0) for r in reqs],
                        on_done=keep_alone)
    for i, r in enumerate(reqs):
        want = expected(r, graphs_h, trees_h)
        assert np.array_equal(got[i], want), i
        assert np.array_equal(alone[i], got[i]), i


def test_slots_follow_free_memory(dpc):
    small = serve.slots_for_memory(1000, 16000, 64 << 20)
    big = serve.slots_for_memory(1000, 16000, 512 << 20)
    assert 1 <= small <= big
    assert serve.slots_for_memory(1 << 22, 1 << 26, 1 << 20) == 0


@pytest.mark.parametrize("rate,slots", [(20000.0, 6), (0.0, 16)])
def test_resident_engine_folds_arrivals_into_the_running_kernel(dpc, pool, rate, slots):
    """ResidentServer: one kernel launch serves the whole stream (arrivals are
    admitted from the mailbox while it runs), and every result equals the
    oracle's and the one served alone."""
    graphs, graphs_h, sources, trees, trees_h = pool
    rng = np.random.default_rng(9)
    reqs = serve.poisson_stream(rng, 120, rate, len(graphs), len(trees), sources)
    srv = serve.ResidentServer(graphs, trees, slots=slots, limit_us=2_000_000)
    got = {}

    def keep(i, s):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        got[i] = srv.read_out(s, n)

    res = srv.run(reqs, on_done=keep)
    assert res.status == 0
    assert res.steps == 1  # kernel launches: the stream never waited for a new one
    assert len(got) == len(reqs) and np.all(res.finished >= res.admitted)
    assert srv.mailbox.taken() == len(reqs)
    alone = {}

    def keep_alone(i, out):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        alone[i] = out[:n].cpu().numpy().copy()

    serve.one_at_a_time(graphs, trees, [serve.Request(r.kind, r.problem, r.source, 0.0) for r in reqs],
                        on_done=keep_alone)
    for i, r in enumerate(reqs):
        want = expected(r, graphs_h, trees_h)
        assert np.array_equal(got[i], want), i
        assert np.array_equal(alone[i], got[i]), i


def test_resident_engine_returns_when_idle_and_resumes(dpc, pool):
    """With a short lifetime and arrivals far apart the resident kernel returns
    while idle; the loop launches it again for the next arrival, and the
    engine's state carries over: results stay exact."""
    graphs, graphs_h, sources, trees, trees_h = pool
    reqs = [serve.Request(dpc.JOB_TREE_HEIGHT, 1, 0, 0.0), serve.Request(dpc.JOB_SSSP, 2, int(sources[2][3]), 0.03),
            serve.Request(dpc.JOB_TREE_DESCENDANTS, 3, 0, 0.06), serve.Request(dpc.JOB_SSSP, 4, int(sources[4][5]), 0.09)]
    srv = serve.ResidentServer(graphs, trees, slots=4, limit_us=2000)
    got = {}

    def keep(i, s):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        got[i] = srv.read_out(s, n)

    res = srv.run(reqs, on_done=keep)
    assert res.status == 0 and len(got) == len(reqs)
    assert res.steps >= 2  # relaunched after idle returns
    for i, r in enumerate(reqs):
        assert np.array_equal(got[i], expected(r, graphs_h, trees_h)), i


def test_resident_engine_rejects_device_memory_for_the_mailbox_side(dpc, pool):
    graphs, _, _, trees, _ = pool
    srv = serve.ResidentServer(graphs[:1], trees[:1], slots=2)
    with pytest.raises(ValueError):
        dpc.engine_serve(srv.ws, srv.slots, srv.max_n, srv.max_m, srv.mailbox, 1000, srv.state, stream=srv.stream)
