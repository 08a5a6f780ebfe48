"""The bounded device-side waits: a wait on a word that nothing sets runs out,
reports DPC_ERR_TIMEOUT and leaves the context usable (no GPU fault, no hang).
Every grid barrier of the queue levels and of the engine waits the same way."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_08150_gb300 import gen
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_us", [1000, 20000])
def test_wait_runs_out_and_reports_timeout(dpc, limit_us):
    status = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    dpc.wait_selftest(limit_us, status)
    torch.cuda.synchronize()
    code, waited = status.cpu().tolist()
    assert code == dpc.ERR_TIMEOUT
    assert limit_us <= waited < limit_us + 500_000
    # the context is still usable: an ordinary call right after
    A = gen.zipf_csr(3000, 4000, s=1.3, lmax=4000, seed=5, normal_values=False)
    x = gen.vector(4000, 5, integer_values=True)
    y = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
    assert dpc.spmv_csr(dev(A.off), dev(A.col), dev(A.val), dev(x), y, "queue") == dpc.OK
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy().astype(np.float64), oracle.spmv_f64(A.off, A.col, A.val, x)[0])


def test_gather_rate_probe_counts_every_load(dpc):
    """dpc_gather_rate (the ceiling of the SpMV gathers): over an array of ones
    the sum it returns is the number of loads it reports, exactly (every
    partial sum is an integer below 2^24)."""
    x = torch.ones(1 << 20, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    n = dpc.gather_rate(x, 1, out)
    torch.cuda.synchronize()
    assert n > 0 and n % 16 == 0 and n < (1 << 24)
    assert float(out.item()) == float(n)
