"""Pins of per-particle softening in the oracle (Sec. 3.2): a pair interacts
with the larger of its two spline supports (closed form, Newton's third law
exactly); equal supports reduce to the uniform walk bit for bit; the walk
converges to the direct sum; a node of mixed supports is opened for a target
of smaller support inside the node's largest support, and used as a monopole
with the larger support otherwise."""
import numpy as np
import pytest

import workloads as W


def test_pair_uses_the_larger_support(oracle_mod):
    pos = np.array([[0.0, 0.0, 0.0], [0.05, 0.0, 0.0]])
    mass = np.array([0.5, 0.25], np.float32)
    hs = np.array([0.1, 0.02], np.float32)
    acc, pot = oracle_mod.direct_soft(pos, mass, hs, np.array([0, 1]), 2.0)
    kf = oracle_mod.kforce(0.05, float(hs[0]))
    kp = oracle_mod.kpot(0.05, float(hs[0]))
    np.testing.assert_allclose(acc[0], [2.0 * 0.25 * 0.05 * kf, 0, 0], rtol=1e-14)
    np.testing.assert_allclose(acc[1], [-2.0 * 0.5 * 0.05 * kf, 0, 0], rtol=1e-14)
    assert pot[0] == pytest.approx(2.0 * 0.25 * kp, rel=1e-14) and pot[1] == pytest.approx(2.0 * 0.5 * kp, rel=1e-14)


def test_two_species_direct_sum_conserves_momentum(oracle_mod):
    pos, mass, hs, _ = W.two_species(1500, 500, 3)
    acc, _ = oracle_mod.direct_soft(pos, mass, hs, np.arange(len(pos)), 1.0)
    p = (mass[:, None].astype(np.float64) * acc).sum(0)
    assert np.abs(p).max() < 1e-13 * (mass[:, None] * np.abs(acc)).sum(0).max()


def test_equal_supports_reduce_to_the_uniform_walk(oracle_mod):
    pos, mass = W.plummer(3000, 4)
    hs = np.full(len(pos), 0.01, np.float32)
    tg = np.arange(0, 3000, 3)
    a0, p0, n0 = oracle_mod.Tree(pos, mass, bucket=4).walk(tg, 1.0, float(hs[0]), theta=0.6)
    a1, p1, n1 = oracle_mod.Tree(pos, mass, bucket=4, hsoft=hs).walk(tg, 1.0, 123.0, theta=0.6)
    np.testing.assert_array_equal(a0, a1)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(n0, n1)


def test_two_species_walk_converges_to_the_direct_sum(oracle_mod):
    pos, mass, hs, _ = W.two_species(3000, 1000, 5)
    tg = np.arange(0, len(pos), 5)
    ad, pd = oracle_mod.direct_soft(pos, mass, hs, tg, 1.0)
    tree = oracle_mod.Tree(pos, mass, bucket=4, hsoft=hs)
    errs = []
    for theta in (0.8, 0.4, 0.02):
        a, _, _ = tree.walk(tg, 1.0, 0.0, theta=theta)
        errs.append(np.percentile(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1), 99))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5, errs


def mixed_cluster(h_target):
    # a compact cluster far from the origin, with one particle of a large
    # support; the target at 0.3 from the cluster, inside that support
    rng = np.random.default_rng(1)
    cl = np.array([1.0, 0.0, 0.0]) + 0.004 * rng.standard_normal((12, 3))
    pos = np.vstack([[[0.7, 0.0, 0.0]], cl, [[-3.0, 2.0, 1.0], [3.0, -2.0, -1.0]]])
    mass = np.full(len(pos), 1.0 / len(pos), np.float32)
    hs = np.full(len(pos), 0.01, np.float32)
    hs[1] = 0.5
    hs[0] = h_target
    return pos, mass, hs


def test_mixed_node_is_opened_for_a_smaller_target_inside_its_support(oracle_mod):
    pos, mass, hs = mixed_cluster(0.01)
    tree = oracle_mod.Tree(pos, mass, bucket=1, hsoft=hs)
    a, p, n = tree.walk([0], 1.0, 0.0, theta=0.9, box_guard=False)
    ad, pd = oracle_mod.direct_soft(pos, mass, hs, [0], 1.0)
    # opened: sub-nodes of uniform small support may stay monopoles, the
    # large-support particle interacts on its own -- more interactions than a
    # target of large support makes with the same cluster
    pos6, mass6, hs6 = mixed_cluster(0.6)
    _, _, n6 = oracle_mod.Tree(pos6, mass6, bucket=1, hsoft=hs6).walk([0], 1.0, 0.0, theta=0.9, box_guard=False)
    assert n[0] > n6[0]
    assert np.linalg.norm(a[0] - ad[0]) <= 2e-3 * np.linalg.norm(ad[0])
    # without the rule the cluster would count as one monopole softened at 0.5
    tree_u = oracle_mod.Tree(pos, mass, bucket=1)
    au, _, _ = tree_u.walk([0], 1.0, 0.5, theta=0.9, box_guard=False)
    assert np.linalg.norm(au[0] - ad[0]) > 0.1 * np.linalg.norm(ad[0])


def test_mixed_node_is_a_monopole_for_a_target_of_larger_support(oracle_mod):
    pos, mass, hs = mixed_cluster(0.6)
    tree = oracle_mod.Tree(pos, mass, bucket=1, hsoft=hs)
    a, _, _ = tree.walk([0], 1.0, 0.0, theta=0.9, box_guard=False)
    ad, _ = oracle_mod.direct_soft(pos, mass, hs, [0], 1.0)
    # the mixed node is not forced open; every pair is softened at 0.6 anyway
    assert np.linalg.norm(a[0] - ad[0]) <= 2e-3 * np.linalg.norm(ad[0])
