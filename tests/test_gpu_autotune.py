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
