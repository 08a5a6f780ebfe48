"""Host-side logic of the autotuner (no GPU): search spaces and the cache."""
import json

from paper_1606_08150_gb300 import autotune


def test_grid_space_is_the_cartesian_product():
    sp = autotune.grid_space(kc=(1, 16), chunk=(8, 32, 128))
    assert len(sp) == 6 and {"kc": 16, "chunk": 32} in sp


def test_cache_keys_by_size_class_and_persists(tmp_path):
    p = tmp_path / "tune.json"
    c = autotune.Cache(str(p))
    assert c.key("spmv", "grid", 1 << 20) == c.key("spmv", "grid", (1 << 21) - 1) == "spmv/grid/2^20"
    calls = []
    c.table[c.key("tree", "block", 1000)] = {"chunk": 32}
    assert c.get("tree", "block", 1000).chunk == 32
    assert c.get("tree", "block", 5000) is None
    c2 = autotune.Cache(str(p))  # nothing written yet: tune() writes
    assert c2.get("tree", "block", 1000) is None
    json.dump(c.table, open(p, "w"))
    assert autotune.Cache(str(p)).get("tree", "block", 1000).chunk == 32
    assert not calls


def test_default_spaces_use_the_kc_rule():
    for level, x in autotune.KC_RULE.items():
        assert any(cfg.get("kc") == x for cfg in autotune.default_space("spmv", level))


def test_cache_lookup_and_store_raw_params(tmp_path):
    p = tmp_path / "t.json"
    c = autotune.Cache(str(p))
    assert c.lookup("engine/x") is None
    c.store("engine/x", {"threshold": 16, "chunk": 512, "parent_blocks": 0, "waves": 64})
    assert autotune.Cache(str(p)).lookup("engine/x")["waves"] == 64


def test_mix_key_and_engine_tuning():
    from types import SimpleNamespace

    graphs = [SimpleNamespace(n=1 << 10), SimpleNamespace(n=(1 << 18) + 5)]
    trees = [SimpleNamespace(n=1000), SimpleNamespace(n=1_000_000)]
    assert autotune.mix_key(graphs, trees, 0.6) == "engine/sssp60/graphs2^10-2^18/trees2^9-2^19"
    t = autotune.engine_tuning(dict(autotune.ENGINE_DEFAULT, parent_blocks=304))
    assert (t.threshold, t.chunk, t.parent_blocks) == (32, 512, 304)
    axes = autotune.engine_axes(152)
    assert all(autotune.ENGINE_DEFAULT[k] in v for k, v in axes.items())
