"""The autotuner on the GPU: exhaustive search picks a configuration no slower
than the KC_X rule and the tuned configuration still computes exact results."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_08150_gb300 import autotune, gen
from tests.gpu_util import dev, u32

pytestmark = pytest.mark.gpu


def test_kc_study_and_tuned_result_on_tree_descendants(dpc):
    t = gen.tree(200_000, seed=4)
    coff, cidx = dev(t.coff), dev(t.cidx)
    out = torch.empty(t.n, dtype=torch.int32, device="cuda")

    def run(level, tuning):
        dpc.tree_descendants(coff, cidx, 0, out, level, tuning=tuning)

    study = autotune.kc_study(run, kcs=(1, 16, 32), child_threads=(128, 256), reps=3)
    for level, r in study.items():
        # the rule is one of the searched candidates, timed in the same sweep
        assert r["best_ms"] <= r["rule_ms"]
        assert 0 < r["rule_fraction_of_best"] <= 1.0
        assert r["one_to_one_ms"] > 0 and r["one_to_one_fraction_of_best"] > 0
    # the 1-1 mapping (one child warp per buffered unit) computes the same result
    for level in ("grid", "block", "warp"):
        out.fill_(-1)
        run(level, dpc.Tuning(child_blocks=autotune.ONE_TO_ONE_BLOCKS))
        torch.cuda.synchronize()
        assert np.array_equal(u32(out), oracle.tree_descendants(t.coff, t.cidx, 0)), level
    cache = autotune.Cache()
    tuned = cache.tune("tree", "grid", t.n, lambda tu: run("grid", tu), autotune.default_space("tree", "grid"), reps=3)
    out.fill_(-1)
    run("grid", tuned)
    torch.cuda.synchronize()
    assert np.array_equal(u32(out), oracle.tree_descendants(t.coff, t.cidx, 0))


def test_tuned_engine_serves_the_mix_bit_exact(dpc):
    """The autotuner's coordinate search over the engine's knobs (threshold,
    chunk, grid size, waves per step) on a saturated sample, stored under the
    mix's key; the server built from that entry gives every request the
    oracle's result."""
    from paper_1606_08150_gb300 import serve

    rng = np.random.default_rng(31)
    graphs_h = [gen.rmat(s, seed=500 + s) for s in (9, 11, 13)]
    trees_h = [gen.tree(n, seed=600 + i) for i, n in enumerate((2000, 40000))]
    graphs = [serve.upload_graph(g) for g in graphs_h]
    trees = [serve.upload_tree(t) for t in trees_h]
    sources = [np.nonzero(np.diff(g.off) > 0)[0] for g in graphs_h]
    sample = serve.poisson_stream(rng, 96, 0.0, len(graphs), len(trees), sources)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    best, trials = autotune.tune_engine(graphs, trees, sample, sms, slots=8, sweeps=1)
    assert set(best) == set(autotune.ENGINE_DEFAULT) and len(trials) >= 4
    assert min(t.ms for t in trials) <= [t.ms for t in trials if t.params == autotune.ENGINE_DEFAULT][0]
    cache = autotune.Cache()
    cache.store(autotune.mix_key(graphs, trees, 0.6), best)
    srv = serve.server_from_cache(cache, graphs, trees, slots=8)
    assert srv.waves == best["waves"]
    reqs = serve.poisson_stream(rng, 80, 20000.0, len(graphs), len(trees), sources)
    got = {}

    def keep(i, s):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        got[i] = srv.out[s, :n].cpu().numpy().copy()

    assert srv.run(reqs, on_done=keep).status == 0
    for i, r in enumerate(reqs):
        if r.kind == dpc.JOB_SSSP:
            g = graphs_h[r.problem]
            want = oracle.sssp_dijkstra(g.off, g.col, g.w, r.source).view(np.int32)
        elif r.kind == dpc.JOB_TREE_DESCENDANTS:
            want = oracle.tree_descendants(trees_h[r.problem].coff, trees_h[r.problem].cidx, 0).view(np.int32)
        else:
            want = oracle.tree_height(trees_h[r.problem].coff, trees_h[r.problem].cidx, 0)
        assert np.array_equal(got[i], want), i
    # the resident server from the same entry: the same results
    rsrv = serve.server_from_cache(cache, graphs, trees, resident=True, slots=8, limit_us=2_000_000)
    assert isinstance(rsrv, serve.ResidentServer)
    got_r = {}

    def keep_r(i, s):
        n = graphs[reqs[i].problem].n if reqs[i].kind == dpc.JOB_SSSP else trees[reqs[i].problem].n
        got_r[i] = rsrv.read_out(s, n)

    assert rsrv.run(reqs, on_done=keep_r).status == 0
    for i in range(len(reqs)):
        assert np.array_equal(got_r[i], got[i]), i


def test_engine_grid_size_from_tuning(dpc):
    """A smaller cooperative engine grid (tuning.parent_blocks) runs the same problems to the same results."""
    from tests.test_gpu_engine import Eng, make_problems, to_jobs, check

    probs = make_problems(5, 10)
    jobs, keep, outs = to_jobs(dpc, probs)
    max_n = max(p[1].n for p in probs)
    max_m = max(p[1].m if p[0] == "sssp" else p[1].n for p in probs)
    for blocks in (1, 7, 152):
        for o in outs:
            o.fill_(-5)
        e = Eng(dpc, len(jobs), max_n, max_m, tuning=dpc.Tuning(parent_blocks=blocks))
        e.stage(jobs, list(range(len(jobs))))
        e.step(1 << 30)
        torch.cuda.synchronize()
        assert dpc.read_stats(e.stats).status == 0
        check(probs, outs)
