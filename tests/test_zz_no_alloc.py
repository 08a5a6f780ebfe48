"""The allocation-free SpMV entry point (dpc_spmv_csr_noalloc).

It serves callers that may not allocate device memory: code whose device heap
is owned by another memory manager, services with a fixed memory budget that
forbids allocation after start-up, and latency-critical paths on which
cudaMalloc/cudaFree would synchronise the device. It takes its scratch space
from an array compiled into the library instead of a workspace and runs the
kernels and units of the regular entry point, so its y must be the regular
entry point's bit for bit, call after call (the launch pool is the same for
both here, so basic-DP inlines the same rows).

This file is collected last on purpose; it passes alone in a fresh process and
after the rest of the suite.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_1606_08150_gb300 import gen
from tests.gpu_util import SPMV_TOL, dev, row_relative_error

pytestmark = pytest.mark.gpu


def problem(seed, nrows, ncols, s):
    A = gen.zipf_csr(nrows, ncols, s=s, lmax=ncols, seed=seed)
    x = gen.vector(ncols, seed)
    return A, x, dev(A.off), dev(A.col), dev(A.val), dev(x)


@pytest.mark.parametrize("level", ["grid", "block", "warp", "basic_dp", "flat"])
def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(dpc, level):
    # two different problems back to back: the shared scratch keeps the first
    # call's contents, which must not leak into the second
    for seed, (nrows, ncols, s) in ((11, (30000, 40000, 1.5)), (12, (50000, 20000, 1.7))):
        A, x, off, col, val, xd = problem(seed, nrows, ncols, s)
        assert dpc.spmv_csr_workspace_size(A.nrows, A.nnz, level) <= dpc.NOALLOC_SCRATCH_BYTES
        y_ref_gpu = torch.full((A.nrows,), float("nan"), device="cuda")
        y_noalloc = torch.full((A.nrows,), float("nan"), device="cuda")
        st_ref = dpc.new_stats()
        assert dpc.spmv_csr(off, col, val, xd, y_ref_gpu, level, stats=st_ref) == dpc.OK
        st = dpc.new_stats()
        assert dpc.spmv_csr_noalloc(off, col, val, xd, y_noalloc, level, stats=st) == dpc.OK
        torch.cuda.synchronize()
        a, b = y_ref_gpu.cpu().numpy(), y_noalloc.cpu().numpy()
        s_ref, s_na = dpc.read_stats(st_ref), dpc.read_stats(st)
        assert s_ref.status == 0 and s_na.status == 0
        assert s_ref.launch_failures == 0 and s_na.launch_failures == 0  # no row inlined by a refused launch
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        y_o, absrow = oracle.spmv_f64(A.off, A.col, A.val, x)
        assert row_relative_error(b, y_o, absrow) <= SPMV_TOL


def test_noalloc_rejects_problems_larger_than_its_array(dpc):
    # 1,048,576 rows of 64 non-zeros: the grid-level workspace is far above 16 MiB
    n = 1 << 20
    off = torch.arange(0, 64 * (n + 1), 64, dtype=torch.int32, device="cuda")
    col = torch.zeros(64 * n, dtype=torch.int32, device="cuda")
    val = torch.zeros(64 * n, dtype=torch.float32, device="cuda")
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    assert dpc.spmv_csr_workspace_size(n, 64 * n, "grid") > dpc.NOALLOC_SCRATCH_BYTES
    with pytest.raises(dpc.DpcError) as e:
        dpc.spmv_csr_noalloc(off, col, val, x, y, "grid")
    assert e.value.status == dpc.ERR_WORKSPACE
    with pytest.raises(dpc.DpcError) as e:
        dpc.spmv_csr_noalloc(off[:2], col[:64], val[:64], x, y[:1], "queue")
    assert e.value.status == dpc.ERR_INVALID_ARG


def test_noalloc_as_the_first_call_of_a_process():
    # the array's address is looked up by the first call, under the launch pool
    # CUDA starts with (this entry point never sets it): results within the
    # SpMV tolerance at basic-DP, the regular entry point's bits at the grid level
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "noalloc_child.py")
    out = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    for i in (0, 1):
        for level in ("grid", "basic_dp"):
            assert res[f"status_{i}_{level}"] == 0 and res[f"device_status_{i}_{level}"] == 0
            assert res[f"err_{i}_{level}"] <= SPMV_TOL, (i, level)
    assert res["regular_status"] == 0 and res["grid_bitwise_equal"]
