"""Pins for the oracle's tree (Sec. 3.1): the node set against the paper's own
one-by-one insertion algorithm (brute force), key/permutation invariants,
exact mass bookkeeping, the root placement and the depth limit."""
import numpy as np
import pytest

import workloads as W


def clustered(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (4, 3))
    pos = c[rng.integers(0, 4, n)] + 0.05 * rng.standard_normal((n, 3)) ** 3
    return pos, np.full(n, 1.0 / n, np.float32)


def node_cells(oracle_mod, ex):
    return {oracle_mod.prefix_to_cell(int(l), int(p)): int(c)
            for l, p, c in zip(ex["level"], ex["prefix"], ex["count"])}


@pytest.mark.parametrize("bucket", [1, 3, 8])
@pytest.mark.parametrize("kind", ["uniform", "clustered", "plummer"])
def test_node_set_equals_sequential_insertion(oracle_mod, bucket, kind):
    n = 256
    if kind == "uniform":
        pos = np.random.default_rng(5).uniform(-3, 7, (n, 3))
        mass = np.full(n, 1.0 / n, np.float32)
    elif kind == "clustered":
        pos, mass = clustered(n, 6)
    else:
        pos, mass = W.plummer(n, 77)
    tree = oracle_mod.Tree(pos, mass, bucket=bucket, shift=W.root_shift(11))
    ex = tree.export()
    got = node_cells(oracle_mod, ex)
    for order_seed in (None, 1, 2):
        order = None if order_seed is None else np.random.default_rng(order_seed).permutation(n)
        ref = oracle_mod.insertion_tree(pos, tree.x0, tree.L0, bucket=bucket, order=order)
        assert got == ref


def test_root_placement(oracle_mod):
    pos, mass = W.hernquist(4096, 3)
    for s in range(5):
        tree = oracle_mod.Tree(pos, mass, bucket=8, shift=W.root_shift(100 + s))
        L0, x0 = tree.L0, tree.x0
        ext = (pos.max(0) - pos.min(0)).max()
        assert L0 >= 1.25 * ext and L0 < 2.5 * ext
        assert np.log2(L0) == np.round(np.log2(L0))
        unit = L0 / 2 ** 21
        assert np.all(np.floor(x0 / unit) * unit == x0)
        assert np.all(x0 <= pos.min(0))
    # different shifts give different roots (the randomised domain centre)
    t1 = oracle_mod.Tree(pos, mass, shift=(0.1, 0.2, 0.3))
    t2 = oracle_mod.Tree(pos, mass, shift=(0.7, 0.2, 0.3))
    assert t1.x0[0] != t2.x0[0]


def decode(key):
    q = np.zeros((len(key), 3), np.int64)
    k = key.astype(np.uint64)
    for b in range(21):
        for a in range(3):
            q[:, a] |= ((k >> np.uint64(3 * b + a)) & np.uint64(1)).astype(np.int64) << b
    return q


def test_keys_perm_and_cells(oracle_mod):
    pos, mass = W.plummer(3000, 8)
    tree = oracle_mod.Tree(pos, mass, bucket=4, shift=W.root_shift(12))
    ex = tree.export()
    key, perm = ex["key"], ex["perm"]
    assert sorted(perm.tolist()) == list(range(len(pos)))
    assert np.all(np.diff(key.astype(np.float64)) >= 0) or np.all(key[1:] >= key[:-1])
    same = key[1:] == key[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])  # ties in index order
    # each particle lies in the level-21 cell its key names
    q = decode(key)
    unit = tree.L0 / 2 ** 21
    x = pos[perm]
    lo = tree.x0 + q * unit
    assert np.all(lo <= x) and np.all(x < lo + unit)


def test_node_table_invariants(oracle_mod):
    pos, mass = clustered(5000, 9)
    B = 6
    tree = oracle_mod.Tree(pos, mass, bucket=B, shift=W.root_shift(13))
    ex = tree.export()
    lvl, first, count, skip = (ex[k].astype(np.int64) for k in ("level", "first", "count", "skip"))
    m = tree.nnodes
    key = ex["key"]
    leaf = skip == np.arange(m) + 1
    assert np.all(count[~leaf] > B)
    assert np.all((count[leaf] <= B) | (lvl[leaf] == 21))
    # count is the number of sorted keys carrying the prefix
    for i in np.random.default_rng(0).choice(m, 300, replace=False):
        sh = np.uint64(3 * (21 - lvl[i]))
        has = (key >> sh) == ex["prefix"][i]
        idx = np.nonzero(has)[0]
        assert idx[0] == first[i] and len(idx) == count[i] and idx[-1] == first[i] + count[i] - 1
    # children of an internal node tile its particle range, in ascending octant order
    for i in np.nonzero(~leaf)[0][:400]:
        c = i + 1
        pos_ = first[i]
        prev_oct = -1
        while c < skip[i]:
            assert lvl[c] == lvl[i] + 1 and first[c] == pos_
            oct_ = int(ex["prefix"][c]) & 7
            assert oct_ > prev_oct
            prev_oct = oct_
            pos_ += count[c]
            c = skip[c]
        assert pos_ == first[i] + count[i]


def test_masses_and_root_com(oracle_mod):
    pos, mass = W.plummer(8192, 1)
    tree = oracle_mod.Tree(pos, mass, bucket=1, shift=W.root_shift(1))
    ex = tree.export()
    # dyadic masses: every node mass is exact
    assert ex["mass"][0] == 1.0
    np.testing.assert_array_equal(ex["mass"], ex["count"] / 8192.0)
    com = (pos * mass[:, None].astype(np.float64)).sum(0) / mass.astype(np.float64).sum()
    np.testing.assert_allclose(ex["com"][0], com, rtol=0, atol=1e-14 * np.abs(pos).max())
    # every node's COM lies inside its cell
    lvl = ex["level"].astype(np.int64)
    side = tree.L0 / 2.0 ** lvl
    cells = np.array([oracle_mod.prefix_to_cell(int(l), int(p))[1:] for l, p in zip(ex["level"], ex["prefix"])])
    lo = tree.x0 + cells * side[:, None]
    assert np.all(ex["com"] >= lo - 1e-12) and np.all(ex["com"] <= lo + side[:, None] + 1e-12)


def test_depth_limit_coincident_particles(oracle_mod):
    pos = np.zeros((5, 3))
    pos[:3] = 0.25  # three identical positions
    pos[3] = [1.0, 1.0, 1.0]
    pos[4] = [-1.0, 0.5, 0.0]
    mass = np.full(5, 0.2, np.float32)
    tree = oracle_mod.Tree(pos, mass, bucket=1)
    ex = tree.export()
    deep = np.nonzero(ex["level"] == 21)[0]
    assert len(deep) == 1 and ex["count"][deep[0]] == 3
    ref = oracle_mod.insertion_tree(pos, tree.x0, tree.L0, bucket=1)
    assert node_cells(oracle_mod, ex) == ref


def test_periodic_shift_and_wrap(oracle_mod):
    pos, mass = W.zeldovich(16, 3)
    shift = np.array([0.3, 0.9, 0.05])
    tree = oracle_mod.Tree(pos, mass, bucket=4, periodic=True, box=1.0, shift=shift)
    ex = tree.export()
    xt = ex["xtree"]
    assert np.all(xt >= 0) and np.all(xt < 1.0)
    d = (xt - pos - shift) % 1.0
    d[d > 0.5] -= 1.0
    assert np.abs(d).max() < 1e-15
    assert tree.L0 == 1.0 and np.all(tree.x0 == 0)
