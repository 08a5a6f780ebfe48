"""GPU parity of dpc_spmv_csr against the fp64 oracle at every consolidation level."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_08150_gb300 import gen
from tests.gpu_util import SPMV_TOL, dev, level_names_with_queue, row_relative_error

pytestmark = pytest.mark.gpu
LEVELS = level_names_with_queue()


def run(dpc, A, x, level, tuning=None, stats=False, offset=0):
    """Run through the C ABI; `offset` shifts col/val by that many elements to
    break 16-byte alignment."""
    off = dev(A.off)
    if offset:
        col_b = dev(np.concatenate([np.zeros(offset, np.int32), A.col]))
        val_b = dev(np.concatenate([np.zeros(offset, np.float32), A.val]))
        col, val = col_b[offset:], val_b[offset:]
    else:
        col, val = dev(A.col), dev(A.val)
    xd = dev(x)
    y = torch.full((A.nrows,), float("nan"), dtype=torch.float32, device="cuda")
    st = dpc.new_stats() if stats else None
    status = dpc.spmv_csr(off, col, val, xd, y, level, tuning=tuning, stats=st, ncols=A.ncols)
    torch.cuda.synchronize()
    return y.cpu().numpy(), status, (dpc.read_stats(st) if stats else None)


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("seed", [0, 1])
def test_random_zipf_matrix(dpc, level, seed):
    A = gen.zipf_csr(5000 + seed * 777, 6000, s=1.5, lmax=6000, seed=seed)
    x = gen.vector(6000, seed)
    y_ref, absrow = oracle.spmv_f64(A.off, A.col, A.val, x)
    y, status, _ = run(dpc, A, x, level)
    assert status == dpc.OK
    assert row_relative_error(y, y_ref, absrow) <= SPMV_TOL


@pytest.mark.parametrize("level", LEVELS)
def test_integer_matrix_is_exact_and_deterministic(dpc, level):
    A = gen.zipf_csr(3000, 4000, s=1.3, lmax=4000, seed=5, normal_values=False)
    x = gen.vector(4000, 5, integer_values=True)
    y_ref, _ = oracle.spmv_f64(A.off, A.col, A.val, x)
    y1, _, _ = run(dpc, A, x, level, tuning=dpc.Tuning(chunk=64))
    y2, _, _ = run(dpc, A, x, level, tuning=dpc.Tuning(chunk=64))
    assert np.array_equal(y1.astype(np.float64), y_ref)
    assert np.array_equal(y1.view(np.int32), y2.view(np.int32))


@pytest.mark.parametrize("level", LEVELS)
def test_repeat_runs_bitwise_identical(dpc, level):
    A = gen.zipf_csr(20000, 20000, s=1.5, lmax=20000, seed=9)
    x = gen.vector(20000, 9)
    y1, _, _ = run(dpc, A, x, level, tuning=dpc.Tuning(chunk=256))
    y2, _, _ = run(dpc, A, x, level, tuning=dpc.Tuning(chunk=256))
    assert np.array_equal(y1.view(np.int32), y2.view(np.int32))


@pytest.mark.parametrize("chunk", [64, 2048])
def test_consolidated_levels_bitwise_identical(dpc, chunk):
    """Warp, block, grid and queue levels cut long rows into the same units and
    add unit partials in unit order, so their results agree bit for bit."""
    A = gen.zipf_csr(30000, 30000, s=1.5, lmax=30000, seed=12)
    x = gen.vector(30000, 12)
    t = dpc.Tuning(chunk=chunk)
    ys = {lv: run(dpc, A, x, lv, tuning=t)[0].view(np.int32) for lv in ("warp", "block", "grid", "queue")}
    for lv in ("warp", "block", "queue"):
        assert np.array_equal(ys[lv], ys["grid"]), lv


@pytest.mark.parametrize("level", LEVELS)
@pytest.mark.parametrize("blocks,threads", [(3, 64), (7, 256), (1, 1024)])
def test_launch_counts_match_oracle(dpc, level, blocks, threads):
    A = gen.zipf_csr(9000, 9000, s=1.6, lmax=9000, seed=2)
    x = gen.vector(9000, 2)
    thr = 40
    t = dpc.Tuning(threshold=thr, parent_blocks=blocks, parent_threads=threads)
    y_ref, absrow = oracle.spmv_f64(A.off, A.col, A.val, x)
    y, status, st = run(dpc, A, x, level, tuning=t, stats=True)
    assert status == dpc.OK and st.status == 0
    assert row_relative_error(y, y_ref, absrow) <= SPMV_TOL
    heavy = np.diff(A.off) > thr
    want = oracle.consolidation_launches(heavy, blocks, threads)
    assert st.launch_failures == 0
    # the queue level runs the child's loop inside the parent grid: no launch
    assert st.child_launches == (0 if level == "queue" else want[level])
    if level != "flat":
        assert st.buffered_items == int(heavy.sum())
        assert st.inline_items == int((~heavy).sum())


@pytest.mark.parametrize("level", LEVELS)
def test_edge_cases(dpc, level):
    # every row empty
    off = np.zeros(101, np.int32)
    A = gen.Csr(off, np.zeros(0, np.int32), np.zeros(0, np.float32), 50)
    y, status, _ = run(dpc, A, gen.vector(50, 1), level)
    assert status == dpc.OK and np.all(y == 0.0)
    # one row of 200,000 non-zeros amid empty and short rows
    L = np.array([0, 3, 200_000, 0, 40, 1], np.int64)
    off = np.concatenate([[0], np.cumsum(L)]).astype(np.int32)
    A = gen.csr_from_offsets(off, 250_000, seed=4)
    x = gen.vector(250_000, 4)
    y_ref, absrow = oracle.spmv_f64(A.off, A.col, A.val, x)
    for t in (None, dpc.Tuning(threshold=-1), dpc.Tuning(threshold=2**31 - 1), dpc.Tuning(chunk=7)):
        y, status, _ = run(dpc, A, x, level, tuning=t)
        assert status == dpc.OK
        assert row_relative_error(y, y_ref, absrow) <= SPMV_TOL
        assert y[0] == 0.0 and y[3] == 0.0


@pytest.mark.parametrize("level", LEVELS)
def test_unaligned_arrays_and_small_blocks(dpc, level):
    A = gen.zipf_csr(4000, 5000, s=1.4, lmax=5000, seed=8)
    x = gen.vector(5000, 8)
    y_ref, absrow = oracle.spmv_f64(A.off, A.col, A.val, x)
    y, status, _ = run(dpc, A, x, level, offset=1, tuning=dpc.Tuning(child_threads=32, parent_threads=32))
    assert status == dpc.OK
    assert row_relative_error(y, y_ref, absrow) <= SPMV_TOL


def test_zero_rows(dpc):
    for level in LEVELS:
        off = torch.zeros(1, dtype=torch.int32, device="cuda")
        e = torch.zeros(0, dtype=torch.int32, device="cuda")
        ev = torch.zeros(0, dtype=torch.float32, device="cuda")
        y = torch.zeros(0, dtype=torch.float32, device="cuda")
        assert dpc.spmv_csr(off, e, ev, torch.zeros(4, device="cuda"), y, level) == dpc.OK


def test_too_small_workspace_is_rejected(dpc):
    A = gen.zipf_csr(1000, 1000, seed=1)
    need = dpc.spmv_csr_workspace_size(A.nrows, A.nnz, "grid")
    ws = torch.empty(need - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(dpc.DpcError):
        dpc.spmv_csr(dev(A.off), dev(A.col), dev(A.val), dev(gen.vector(1000, 1)),
                     torch.empty(A.nrows, device="cuda"), "grid", workspace=ws)


@pytest.mark.parametrize("law", ["calibrated", "literal"])
def test_full_size_zipf_1m(dpc, law):
    """1,048,576 x 1,048,576, Zipf row lengths in [1, 200,000]: the mean-16
    calibrated law (s=1.8795) and the literal s=1.5 law, every level, every row
    checked against the oracle."""
    s = 1.8795 if law == "calibrated" else 1.5
    n = 1 << 20
    A = gen.zipf_csr(n, n, s=s, lmax=200_000, seed=3)
    x = gen.vector(n, 3)
    y_ref, absrow = oracle.spmv_f64(A.off, A.col, A.val, x)
    off, col, val, xd = dev(A.off), dev(A.col), dev(A.val), dev(x)
    for level in LEVELS:
        y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        st = dpc.new_stats()
        assert dpc.spmv_csr(off, col, val, xd, y, level, stats=st) == dpc.OK
        torch.cuda.synchronize()
        err = row_relative_error(y.cpu().numpy(), y_ref, absrow)
        assert err <= SPMV_TOL, (level, err)
        stats = dpc.read_stats(st)
        assert stats.status == 0
        if level != "flat":
            assert stats.buffered_items == int((np.diff(A.off) > 32).sum())


@pytest.mark.parametrize("level", LEVELS)
def test_host_resident_matrix_read_in_place(dpc, level):
    """The matrix in pinned host memory, read by the kernels in place over the
    host link: y is bitwise the y of the same matrix in device memory; host
    memory the device cannot read is refused before any launch."""
    A = gen.zipf_csr(20000, 20000, s=1.5, lmax=20000, seed=11)
    x = gen.vector(20000, 11)
    h = [torch.from_numpy(a).pin_memory() for a in (A.off, A.col, A.val)]
    assert all(dpc.device_accessible(t) for t in h)
    y_dev, status, _ = run(dpc, A, x, level)
    assert status == dpc.OK
    xd = dev(x)
    y = torch.full((A.nrows,), float("nan"), dtype=torch.float32, device="cuda")
    assert dpc.spmv_csr(h[0], h[1], h[2], xd, y, level) == dpc.OK
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy().view(np.int32), y_dev.view(np.int32))
    with pytest.raises(ValueError):
        dpc.spmv_csr(torch.from_numpy(A.off), h[1], h[2], xd, y, level)  # pageable host memory
    with pytest.raises(ValueError):
        dpc.spmv_csr(h[0], h[1], h[2], torch.from_numpy(x).pin_memory(), y, level)  # x must be on the device
