"""GPU parity of the persistent batched engine (dpc_engine_*): many SSSP and
tree problems of uneven sizes in one resident kernel, bit-exact against the
oracle, the same result alone and in a mix, admitted all at once or arriving
between steps, and replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_08150_gb300 import gen
from tests.gpu_util import dev, u32

pytestmark = pytest.mark.gpu


def make_problems(seed, count, max_n=20000):
    """Mixed SSSP (R-MAT / random graphs) and tree problems with their expected results."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            scale = int(rng.integers(5, 14))
            g = gen.rmat(scale, seed=seed * 1000 + i) if rng.random() < 0.7 else \
                gen.random_graph(int(rng.integers(1, 3000)), int(rng.integers(0, 30000)), 1, 100, seed=i)
            src = int(rng.integers(0, g.n))
            probs.append(("sssp", g, src, oracle.sssp_dijkstra(g.off, g.col, g.w, src)))
        else:
            n = int(np.exp(rng.uniform(np.log(2), np.log(max_n))))
            t = gen.tree(n, heavy_p=0.01, hlo=50, hhi=2000, seed=seed * 1000 + i, permute=bool(i % 2))
            want = oracle.tree_descendants(t.coff, t.cidx, 0) if kind == 1 else oracle.tree_height(t.coff, t.cidx, 0)
            probs.append(("desc" if kind == 1 else "height", t, 0, want))
    return probs


def to_jobs(dpc, probs):
    jobs, keep, outs = [], [], []
    for kind, obj, src, _ in probs:
        if kind == "sssp":
            off, col, w = dev(obj.off), dev(obj.col), dev(obj.w)
            out = torch.full((obj.n,), -5, dtype=torch.int32, device="cuda")
            jobs.append(dpc.Job(dpc.JOB_SSSP, obj.n, obj.m, src, off.data_ptr(),
                                col.data_ptr() if obj.m else 0, w.data_ptr() if obj.m else 0, out.data_ptr()))
            keep += [off, col, w]
        else:
            off, col = dev(obj.coff), dev(obj.cidx if obj.n > 1 else np.zeros(1, np.int32))
            out = torch.full((obj.n,), -5, dtype=torch.int32, device="cuda")
            k = dpc.JOB_TREE_DESCENDANTS if kind == "desc" else dpc.JOB_TREE_HEIGHT
            jobs.append(dpc.Job(k, obj.n, max(obj.n - 1, 0), src, off.data_ptr(), col.data_ptr(), 0, out.data_ptr()))
            keep += [off, col]
        outs.append(out)
    return jobs, keep, outs


def check(probs, outs):
    for (kind, _, _, want), out in zip(probs, outs):
        got = u32(out) if kind in ("sssp", "desc") else out.cpu().numpy()
        assert np.array_equal(got, want), kind


class Eng:
    def __init__(self, dpc, slots, max_n, max_m, tuning=None):
        self.dpc, self.slots, self.max_n, self.max_m, self.tuning = dpc, slots, max_n, max_m, tuning
        self.ws = torch.empty(dpc.engine_workspace_size(slots, max_n, max_m, tuning), dtype=torch.uint8, device="cuda")
        self.state = torch.zeros(slots, dtype=torch.int32, device="cuda")
        self.jobs = torch.zeros(48 * slots, dtype=torch.uint8, device="cuda")
        self.slot_ids = torch.zeros(slots, dtype=torch.int32, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.stats = dpc.new_stats()
        dpc.engine_init(self.ws, slots, max_n, max_m, self.state, tuning)

    def stage(self, jobs, slot_ids):
        raw = self.dpc.pack_jobs(jobs)
        if raw:
            self.jobs[:len(raw)].copy_(torch.frombuffer(bytearray(raw), dtype=torch.uint8))
            self.slot_ids[:len(slot_ids)].copy_(torch.tensor(slot_ids, dtype=torch.int32))
        self.count.fill_(len(jobs))

    def step(self, max_waves):
        self.dpc.engine_step(self.ws, self.slots, self.max_n, self.max_m, self.jobs, self.slot_ids, self.count,
                             max_waves, self.state, self.tuning, self.stats)


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_to_completion(dpc, seed):
    probs = make_problems(seed, 24)
    jobs, keep, outs = to_jobs(dpc, probs)
    max_n = max(p[1].n for p in probs)
    max_m = max(p[1].m if p[0] == "sssp" else p[1].n for p in probs)
    e = Eng(dpc, len(jobs), max_n, max_m)
    e.stage(jobs, list(range(len(jobs))))
    e.step(1 << 30)
    torch.cuda.synchronize()
    assert dpc.read_stats(e.stats).status == 0
    assert (e.state.cpu().numpy() == 2).all()
    check(probs, outs)


def test_same_result_alone_and_in_the_mix(dpc):
    probs = make_problems(7, 12)
    max_n = max(p[1].n for p in probs)
    max_m = max(p[1].m if p[0] == "sssp" else p[1].n for p in probs)
    jobs, keep, outs = to_jobs(dpc, probs)
    e = Eng(dpc, len(jobs), max_n, max_m)
    e.stage(jobs, list(range(len(jobs))))
    e.step(1 << 30)
    torch.cuda.synchronize()
    mixed = [o.clone() for o in outs]
    for i, job in enumerate(jobs):  # each problem alone, through the same engine
        outs[i].fill_(-5)
        e2 = Eng(dpc, 1, max_n, max_m)
        e2.stage([job], [0])
        e2.step(1 << 30)
        torch.cuda.synchronize()
        assert torch.equal(outs[i], mixed[i])
    check(probs, outs)


def test_arrivals_between_steps(dpc):
    """Continuous batching: problems arrive while others run; few waves per step."""
    probs = make_problems(3, 30)
    jobs, keep, outs = to_jobs(dpc, probs)
    slots = 8
    max_n = max(p[1].n for p in probs)
    max_m = max(p[1].m if p[0] == "sssp" else p[1].n for p in probs)
    e = Eng(dpc, slots, max_n, max_m, dpc.Tuning(threshold=16))
    free = list(range(slots))
    waiting = list(range(len(jobs)))
    running = {}
    steps = 0
    while waiting or running:
        admit_ids = []
        admit_slots = []
        while waiting and free and len(admit_ids) < 3:  # at most three arrivals per step
            admit_ids.append(waiting.pop(0))
            admit_slots.append(free.pop(0))
        e.stage([jobs[i] for i in admit_ids], admit_slots)
        for i, s in zip(admit_ids, admit_slots):
            running[s] = i
        e.step(4)
        torch.cuda.synchronize()
        state = e.state.cpu().numpy()
        for s in list(running):
            if state[s] == 2:
                del running[s]
                free.append(s)
        steps += 1
        assert steps < 100000
    assert dpc.read_stats(e.stats).status == 0
    check(probs, outs)


def test_graph_capture_and_replay(dpc):
    probs = make_problems(11, 10)
    jobs, keep, outs = to_jobs(dpc, probs)
    max_n = max(p[1].n for p in probs)
    max_m = max(p[1].m if p[0] == "sssp" else p[1].n for p in probs)
    e = Eng(dpc, len(jobs), max_n, max_m)
    e.stage(jobs, list(range(len(jobs))))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        # first step outside capture (module load, occupancy query)
        e.count.fill_(0)
        e.step(1)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        e.step(1 << 30)
    for rep in range(2):
        for o in outs:
            o.fill_(-5)
        dpc.engine_init(e.ws, e.slots, e.max_n, e.max_m, e.state)
        e.stage(jobs, list(range(len(jobs))))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        check(probs, outs)


def test_upper_sizes_of_the_served_mix(dpc):
    """The largest problems of the served stream (an R-MAT 2^18 graph, edge
    factor 16, weights in [1,100]; a 10^6-node heavy-tailed tree for
    descendants and for heights) inside a mixed batch with small problems:
    bit-exact against the oracle, and the same alone as in the mix."""
    g = gen.rmat(18, seed=1018)
    src = int(np.nonzero(np.diff(g.off) > 0)[0][3])
    t = gen.tree(1_000_000, seed=2018)
    big = [("sssp", g, src, oracle.sssp_dijkstra(g.off, g.col, g.w, src)),
           ("desc", t, 0, oracle.tree_descendants(t.coff, t.cidx, 0)),
           ("height", t, 0, oracle.tree_height(t.coff, t.cidx, 0))]
    probs = big + make_problems(3, 9)
    jobs, keep, outs = to_jobs(dpc, probs)
    max_n = max(p[1].n for p in probs)
    max_m = max(p[1].m if p[0] == "sssp" else p[1].n for p in probs)
    e = Eng(dpc, len(jobs), max_n, max_m)
    e.stage(jobs, list(range(len(jobs))))
    e.step(1 << 30)
    torch.cuda.synchronize()
    assert dpc.read_stats(e.stats).status == 0
    assert (e.state.cpu().numpy() == 2).all()
    check(probs, outs)
    mixed = [o.clone() for o in outs[:len(big)]]
    e1 = Eng(dpc, 1, max_n, max_m)
    for i in range(len(big)):
        outs[i].fill_(-5)
        dpc.engine_init(e1.ws, 1, max_n, max_m, e1.state, None)
        e1.stage([jobs[i]], [0])
        e1.step(1 << 30)
        torch.cuda.synchronize()
        assert dpc.read_stats(e1.stats).status == 0
        assert torch.equal(outs[i], mixed[i]), probs[i][0]
