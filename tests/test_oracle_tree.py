"""Pins for the tree oracle: brute-force ancestor walks, closed forms (chains,
stars), the identity sum(desc) = sum(depth), and a hand-worked tree."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1606_08150_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def parents_of(tree):
    n = tree.n
    parent = np.full(n, -1, np.int64)
    for v in range(n):
        for k in range(tree.coff[v], tree.coff[v + 1]):
            parent[tree.cidx[k]] = v
    return parent


def brute_force(parent, root):
    """Walk from every node up to the root: each ancestor at distance k gains one
    descendant and a height candidate k."""
    n = parent.shape[0]
    desc = np.zeros(n, np.int64)
    height = np.zeros(n, np.int64)
    depth = np.zeros(n, np.int64)
    for v in range(n):
        u, k = v, 0
        while u != root:
            u = parent[u]
            k += 1
            desc[u] += 1
            height[u] = max(height[u], k)
        depth[v] = k
    return desc, height, depth


def test_hand_worked():
    d = json.load(open(os.path.join(GOLDEN, "tree_hand.json")))
    parent = np.zeros(d["n"], np.int64)
    for p, kids in d["children"].items():
        for c in kids:
            parent[c] = int(p)
    t = gen.tree_from_parents(parent, d["root"])
    assert oracle.tree_descendants(t.coff, t.cidx, d["root"]).tolist() == d["desc"]
    assert oracle.tree_height(t.coff, t.cidx, d["root"]).tolist() == d["height"]
    lv = oracle.tree_levels(t.coff, t.cidx, d["root"], threshold=2)
    assert lv.nodes.tolist() == np.bincount(d["depth"]).tolist()
    hand = d["levels"]
    assert lv.nodes.tolist() == hand["nodes"]
    assert lv.internal.tolist() == hand["internal"]
    assert lv.edges.tolist() == hand["edges"]
    for thr, heavy in hand["heavy_by_threshold"].items():
        assert oracle.tree_levels(t.coff, t.cidx, d["root"], threshold=int(thr)).heavy.tolist() == heavy, thr


def levels_brute_force(parent, root, threshold):
    """Per-depth counts from the parent array alone (no child lists): a node's
    child count is how often it appears as a parent, its depth the length of
    its walk to the root."""
    n = parent.shape[0]
    kids = np.bincount(parent[parent >= 0], minlength=n)
    _, _, depth = brute_force(parent, root)
    L = int(depth.max()) + 1
    nodes = np.bincount(depth, minlength=L)
    internal = np.bincount(depth, weights=(kids > 0), minlength=L).astype(np.int64)
    edges = np.bincount(depth, weights=kids, minlength=L).astype(np.int64)
    heavy = np.bincount(depth, weights=(kids > threshold), minlength=L).astype(np.int64)
    return nodes, internal, edges, heavy


def check_levels_against_brute_force(parent, root, thresholds=(0, 1, 2, 5, 32)):
    t = gen.tree_from_parents(parent, root)
    n_with_children = np.unique(parent[parent >= 0]).shape[0]
    for thr in thresholds:
        lv = oracle.tree_levels(t.coff, t.cidx, root, threshold=thr)
        nodes, internal, edges, heavy = levels_brute_force(parent, root, thr)
        assert lv.nodes.tolist() == nodes.tolist()
        assert lv.internal.tolist() == internal.tolist()
        assert lv.edges.tolist() == edges.tolist()
        assert lv.heavy.tolist() == heavy.tolist()
        # one recursive launch per node with children (Sec. IV.B): summed over depths
        assert int(lv.internal.sum()) == n_with_children
        assert int(lv.heavy.sum()) == int((np.bincount(parent[parent >= 0], minlength=t.n) > thr).sum())


@pytest.mark.parametrize("seed", range(6))
def test_tree_levels_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 600))
    # random recursive trees with a few wide nodes, so that every threshold splits somewhere
    parent = np.array([-1] + [int(rng.integers(0, max(1, i // 4))) if rng.random() < 0.5 else int(rng.integers(0, i))
                              for i in range(1, n)], np.int64)
    check_levels_against_brute_force(parent, 0)


def test_tree_levels_generated_and_non_zero_root():
    t = gen.tree(3000, heavy_p=0.02, hlo=5, hhi=60, seed=7, permute=True)
    check_levels_against_brute_force(parents_of(t), t.root)
    parent = np.array([2, 2, -1, 1, 1, 3, 3, 3], np.int64)  # root 2, node 3 has three children
    check_levels_against_brute_force(parent, 2, thresholds=(0, 1, 2, 3))


@pytest.mark.parametrize("seed", range(8))
def test_random_recursive_trees_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 800))
    parent = np.array([-1] + [int(rng.integers(0, i)) for i in range(1, n)], np.int64)
    t = gen.tree_from_parents(parent, 0)
    desc, height, depth = brute_force(parent, 0)
    assert np.array_equal(oracle.tree_descendants(t.coff, t.cidx, 0), desc)
    assert np.array_equal(oracle.tree_height(t.coff, t.cidx, 0), height)
    assert int(desc.sum()) == int(depth.sum())


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_generated_heavy_tail_trees_brute_force(seed):
    t = gen.tree(3000, heavy_p=0.02, hlo=50, hhi=400, seed=seed, permute=(seed % 2 == 1))
    parent = parents_of(t)
    desc, height, depth = brute_force(parent, t.root)
    d = oracle.tree_descendants(t.coff, t.cidx, t.root)
    h = oracle.tree_height(t.coff, t.cidx, t.root)
    assert np.array_equal(d, desc) and np.array_equal(h, height)
    assert d[t.root] == t.n - 1
    assert h[t.root] == depth.max()
    lv = oracle.tree_levels(t.coff, t.cidx, t.root)
    assert lv.nodes.sum() == t.n and lv.edges.sum() == t.n - 1
    assert lv.edges[:-1].tolist() == lv.nodes[1:].tolist()


def test_chain_and_star_closed_forms():
    n = 100
    c = gen.chain(n)
    assert oracle.tree_descendants(c.coff, c.cidx, 0).tolist() == list(range(n - 1, -1, -1))
    assert oracle.tree_height(c.coff, c.cidx, 0).tolist() == list(range(n - 1, -1, -1))
    star = gen.tree_from_parents(np.zeros(n, np.int64), 0)
    d = oracle.tree_descendants(star.coff, star.cidx, 0)
    h = oracle.tree_height(star.coff, star.cidx, 0)
    assert d[0] == n - 1 and h[0] == 1 and not d[1:].any() and not h[1:].any()
    one = gen.chain(1)
    assert oracle.tree_descendants(one.coff, one.cidx, 0).tolist() == [0]
    assert oracle.tree_height(one.coff, one.cidx, 0).tolist() == [0]


def test_non_root_zero_root():
    parent = np.array([2, 2, -1, 1, 1], np.int64)
    t = gen.tree_from_parents(parent, 2)
    assert oracle.tree_descendants(t.coff, t.cidx, 2).tolist() == [0, 2, 4, 0, 0]
    assert oracle.tree_height(t.coff, t.cidx, 2).tolist() == [0, 1, 2, 0, 0]


def test_malformed_trees_rejected():
    # right edge count but node 2 listed twice and node 3 never reached (a DAG)
    with pytest.raises(ValueError):
        oracle.tree_descendants(np.array([0, 2, 3, 3, 3], np.int32), np.array([1, 2, 2], np.int32), 0)
    # right edge count but a cycle 2 <-> 3 outside the root's subtree
    with pytest.raises(ValueError):
        oracle.tree_height(np.array([0, 1, 1, 2, 3], np.int32), np.array([1, 3, 2], np.int32), 0)
    # wrong edge count
    with pytest.raises(ValueError):
        oracle.tree_height(np.array([0, 1, 2, 3], np.int32), np.array([1, 2, 0], np.int32), 0)


def test_planted_off_by_one_is_caught():
    t = gen.tree(500, heavy_p=0.0, seed=9)
    desc, _, _ = brute_force(parents_of(t), 0)
    wrong = desc + (desc > 0)  # "including self" for internal nodes
    assert not np.array_equal(oracle.tree_descendants(t.coff, t.cidx, 0), wrong)
