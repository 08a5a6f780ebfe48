"""Run in a fresh process by test_gpu_checked.py with DPC_LIBRARY=checked: the
bounds-checked build of the library (every index read from the caller's
arrays and every append into a bounded buffer checked on the device) runs
every application at every level on small inputs, and reports the largest
error and every status. It then gives SSSP and SpMV a column index past the
end of the arrays, which the checked build skips and reports as
DPC_ERR_OVERFLOW; that part runs only after the loaded library is confirmed to
be the checked build."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_1606_08150_gb300 import build, dpc, gen  # noqa: E402

LEVELS = ["basic_dp", "flat", "warp", "block", "grid", "queue"]
dpc.device_init(0, 1 << 16)


def d(a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a).cuda()


res = {"library": dpc._lib._name, "checked": os.path.samefile(dpc._lib._name, build.LIB_CHECKED), "cases": []}


def case(name, level, ok, status):
    res["cases"].append({"case": name, "level": level, "ok": bool(ok), "status": int(status)})


g = gen.rmat(10, seed=3)
want = oracle.sssp_dijkstra(g.off, g.col, g.w, 0)
for tuning, tag in ((None, "plain"), (dpc.Tuning(delta=20, sub_delta=2), "nearfar")):
    for lv in LEVELS:
        dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
        st = dpc.new_stats()
        dpc.sssp(d(g.off), d(g.col), d(g.w), 0, dist, lv, tuning=tuning, stats=st)
        torch.cuda.synchronize()
        case("sssp_" + tag, lv, np.array_equal(dist.cpu().numpy().view(np.uint32), want), dpc.read_stats(st).status)

A = gen.zipf_csr(5000, 4000, s=1.5, lmax=4000, seed=4)
x = gen.vector(4000, 4)
y_ref, absrow = oracle.spmv_f64(A.off, A.col, A.val, x)
for lv in LEVELS:
    y = torch.empty(A.nrows, device="cuda")
    st = dpc.new_stats()
    dpc.spmv_csr(d(A.off), d(A.col), d(A.val), d(x), y, lv, stats=st)
    torch.cuda.synchronize()
    err = float(np.max(np.abs(y.cpu().numpy().astype(np.float64) - y_ref) / (absrow + 1e-30)))
    case("spmv", lv, err <= 1e-5, dpc.read_stats(st).status)

t = gen.tree(20000, heavy_p=0.01, hlo=50, hhi=2000, seed=5)
wd, wh = oracle.tree_descendants(t.coff, t.cidx, 0), oracle.tree_height(t.coff, t.cidx, 0)
for lv in LEVELS:
    for name, fn, want_t in (("tree_desc", dpc.tree_descendants, wd.view(np.int32)),
                             ("tree_height", dpc.tree_height, wh)):
        out = torch.empty(t.n, dtype=torch.int32, device="cuda")
        st = dpc.new_stats()
        fn(d(t.coff), d(t.cidx), 0, out, lv, stats=st)
        torch.cuda.synchronize()
        case(name, lv, np.array_equal(out.cpu().numpy(), want_t), dpc.read_stats(st).status)

g9 = gen.rmat(9, seed=6)
ie = gen.in_edges(g9.off, g9.col)
pr = oracle.pagerank(g9.off, g9.col, 0.85, 5)
for lv in LEVELS:
    rank = torch.empty(g9.n, device="cuda")
    st = dpc.new_stats()
    dpc.pagerank(d(ie.off), d(ie.src), d(ie.outdeg), rank, lv, iterations=5, stats=st)
    torch.cuda.synchronize()
    case("pagerank", lv, float(np.max(np.abs(rank.cpu().numpy() - pr) / pr)) < 1e-4, dpc.read_stats(st).status)

lvl_want, _ = oracle.bfs(g.off, g.col, 0)
for lv in LEVELS:
    lvl = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = dpc.new_stats()
    dpc.bfs_rec(d(g.off), d(g.col), 0, lvl, lv, stats=st)
    torch.cuda.synchronize()
    case("bfs_rec", lv, np.array_equal(lvl.cpu().numpy().view(np.uint32), lvl_want), dpc.read_stats(st).status)

s_off, s_col = gen.symmetrize(g9.off, g9.col)
prio = gen.priorities(g9.n, 6)
cw = oracle.color_jp(s_off, s_col, prio).color
for lv in LEVELS:
    color = torch.empty(g9.n, dtype=torch.int32, device="cuda")
    st = dpc.new_stats()
    dpc.graph_coloring(d(s_off), d(s_col), d(prio), color, lv, stats=st)
    torch.cuda.synchronize()
    case("graph_coloring", lv, np.array_equal(color.cpu().numpy(), cw), dpc.read_stats(st).status)

y = torch.empty(A.nrows, device="cuda")
st = dpc.new_stats()
dpc.spmv_csr_noalloc(d(A.off), d(A.col), d(A.val), d(x), y, "grid", stats=st)
torch.cuda.synchronize()
err = float(np.max(np.abs(y.cpu().numpy().astype(np.float64) - y_ref) / (absrow + 1e-30)))
case("spmv_noalloc", "grid", err <= 1e-5, dpc.read_stats(st).status)

# the batched engine: SSSP and tree problems in one resident kernel
jobs, keep, outs, wants = [], [], [], []
for kind, obj, w_ in (("sssp", g, want), ("desc", t, wd), ("height", t, wh)):
    out = torch.full((obj.n,), -5, dtype=torch.int32, device="cuda")
    if kind == "sssp":
        a = [d(obj.off), d(obj.col), d(obj.w)]
        jobs.append(dpc.Job(dpc.JOB_SSSP, obj.n, obj.m, 0, a[0].data_ptr(), a[1].data_ptr(), a[2].data_ptr(),
                            out.data_ptr()))
    else:
        a = [d(obj.coff), d(obj.cidx)]
        jobs.append(dpc.Job(dpc.JOB_TREE_DESCENDANTS if kind == "desc" else dpc.JOB_TREE_HEIGHT, obj.n, obj.n - 1, 0,
                            a[0].data_ptr(), a[1].data_ptr(), 0, out.data_ptr()))
    keep += a
    outs.append(out)
    wants.append(w_.view(np.int32))
max_n, max_m = max(g.n, t.n), max(g.m, t.n)
ws = torch.empty(dpc.engine_workspace_size(3, max_n, max_m), dtype=torch.uint8, device="cuda")
state = torch.zeros(3, dtype=torch.int32, device="cuda")
dpc.engine_init(ws, 3, max_n, max_m, state)
raw = torch.frombuffer(bytearray(dpc.pack_jobs(jobs)), dtype=torch.uint8).cuda()
slots = torch.arange(3, dtype=torch.int32, device="cuda")
count = torch.full((1,), 3, dtype=torch.int32, device="cuda")
st = dpc.new_stats()
dpc.engine_step(ws, 3, max_n, max_m, raw, slots, count, 1 << 30, state, None, st)
torch.cuda.synchronize()
case("engine", "queue", all(np.array_equal(o.cpu().numpy(), w_) for o, w_ in zip(outs, wants)),
     dpc.read_stats(st).status)

# malformed input: a column index past the end, which only the checked build may be given
if res["checked"]:
    bad = g.col.copy()
    bad[len(bad) // 2] = g.n + 3
    for lv in LEVELS:
        dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
        s_ = dpc.sssp(d(g.off), d(bad), d(g.w), 0, dist, lv, tuning=dpc.Tuning(flags=dpc.FLAG_SYNC_CHECK))
        res["cases"].append({"case": "sssp_bad_column", "level": lv, "status": int(s_)})
    badc = A.col.copy()
    badc[len(badc) // 3] = A.ncols + 7
    for lv in LEVELS:
        y = torch.empty(A.nrows, device="cuda")
        s_ = dpc.spmv_csr(d(A.off), d(badc), d(A.val), d(x), y, lv, tuning=dpc.Tuning(flags=dpc.FLAG_SYNC_CHECK))
        res["cases"].append({"case": "spmv_bad_column", "level": lv, "status": int(s_)})
print(json.dumps(res))
