"""The oracle against the constants the paper prints (tests/golden/
gravity_constants.txt): the softened potential at zero lag, the radius from
which the force is Newtonian, and the size of the box guard."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "gravity_constants.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_softening_constants(oracle_mod):
    g = golden()
    eps = 0.013
    h = g["newtonian_from_radius_over_eps"] * eps  # the spline support
    assert oracle_mod.kpot(0.0, h) * eps == pytest.approx(g["zero_lag_potential_times_eps_over_Gm"], rel=1e-12)
    r = g["newtonian_from_radius_over_eps"] * eps
    for x in (r, 1.0001 * r, 3 * r):
        assert oracle_mod.kforce(x, h) * x ** 3 == pytest.approx(1.0, rel=1e-12)
        assert oracle_mod.kpot(x, h) * x == pytest.approx(-1.0, rel=1e-12)
    assert oracle_mod.kforce(0.99 * r, h) * (0.99 * r) ** 3 < 1.0  # softened just inside


def test_box_guard_size(oracle_mod):
    # Root: the frame points fix lo = -4 and L0 = 16 (x0 = -4).  A tight pair
    # sits in the level-6 cell [0.25, 0.5)^3 (side L = 0.25, centre 0.375);
    # the probe sits on the -x axis of that cell, in its level-6 sibling, so
    # the level-5 parent holds three particles and the pair's cell is a leaf
    # node of its own.  With a huge opening angle only the box guard opens it.
    g = golden()
    half = g["box_guard_cube_over_node_side"] / 2
    L, c = 0.25, np.array([0.375, 0.375, 0.375])
    base = np.array([[0.30, 0.30, 0.30], [0.32, 0.31, 0.30], [4.0, 4.0, 4.0], [-4.0, -4.0, -4.0]])
    counts = []
    for f in (0.999 * half, 1.001 * half):
        pos = np.vstack([base, c - np.array([f * L, 0.0, 0.0])])
        mass = np.array([0.5, 0.5, 1e-30, 1e-30, 1e-30], np.float32)
        tree = oracle_mod.Tree(pos, mass, bucket=2)
        assert tree.L0 == 16.0 and np.all(tree.x0 == -4.0)
        ex = tree.export()
        leaf = [k for k in range(tree.nnodes) if ex["count"][k] == 2 and ex["level"][k] == 6]
        assert len(leaf) == 1  # the pair's node is the cell described above
        _, ix, iy, iz = oracle_mod.prefix_to_cell(6, int(ex["prefix"][leaf[0]]))
        np.testing.assert_allclose(tree.x0 + (np.array([ix, iy, iz]) + 0.5) * L, c)
        _, _, n = tree.walk([4], 1.0, 1e-6, theta=1e6)
        counts.append(int(n[0]))
    # inside the cube of 1.2 L the pair's node is opened (two pair terms),
    # outside it is one monopole; the frame points add one term each
    assert counts == [4, 3], counts
