"""Pins of the nonperiodic (isolated) PM oracle (Sec. 3.3: zero padding and
the isolated Green's function; Sec. 3.4: the Gaussian split) against closed
forms: the long-range pair force of one mass, the far field with no periodic
images and no background, and TreePM with open boundaries converging to the
direct sum as the split is resolved."""
import math

import numpy as np

import workloads as W


def frame(pos, half):
    """Two massless corner points that fix the mesh region around the origin."""
    return np.vstack([pos, [[half, half, half], [-half, -half, -half]]])


def test_region_is_the_root_cube_centred_on_the_particles(oracle_mod):
    pos, _ = W.plummer(500, 3)
    corner, side = oracle_mod.pm_region_isolated(pos)
    tree = oracle_mod.Tree(pos, np.ones(len(pos), np.float32), bucket=8)
    assert side == tree.L0
    lo, hi = pos.min(0), pos.max(0)
    np.testing.assert_allclose(corner + side / 2, (lo + hi) / 2, rtol=0, atol=1e-12)
    assert (lo - corner).min() >= 0.1 * side and (corner + side - hi).min() >= 0.1 * side


def test_isolated_pair_force_matches_long_range_closed_form(oracle_mod):
    # one unit mass: the mesh force at r = 2..4 r_s follows g_l(r) / r^2,
    # g_l = erf(x) - 2x/sqrt(pi) e^{-x^2}, x = r / 2 r_s (no background term:
    # open boundaries); CIC anisotropy leaves a few per cent of scatter
    ng = 32
    rng = np.random.default_rng(2)
    for mult in (2, 3, 4):
        ratios = []
        for _ in range(6):
            src = rng.uniform(-0.5, 0.5, (1, 3))
            d = rng.standard_normal((40, 3))
            d /= np.linalg.norm(d, axis=1)[:, None]
            pos = frame(np.vstack([src, src]), 2.0)  # the region: side 8, dx = 0.25
            corner, side = oracle_mod.pm_region_isolated(pos)
            rs = 1.25 * side / ng
            r = mult * rs
            probes = src + r * d
            pos = np.vstack([pos, probes])
            mass = np.zeros(len(pos), np.float32)
            mass[0] = 1.0
            phi = oracle_mod.pm_potential_isolated(pos, mass, corner, side, ng, rs)
            a, _ = oracle_mod.pm_interpolate_isolated(phi, probes, corner, side, ng)
            x = r / (2 * rs)
            gl = math.erf(x) - 2 * x / math.sqrt(math.pi) * math.exp(-x * x)
            ratios.append(-(a * d).sum(1) / (gl / r ** 2))
        ratios = np.concatenate(ratios)
        assert abs(ratios.mean() - 1.0) < 0.02 and ratios.std() < 0.03 and np.abs(ratios - 1).max() < 0.1


def test_isolated_far_field_is_newtonian_without_images(oracle_mod):
    # far from the split scale the long-range part is the whole force and
    # potential, G m / r^2 and -G m / r, out to 0.3 of the region: a periodic
    # mesh would add image forces of order 10% there
    ng = 64
    rng = np.random.default_rng(5)
    pos = frame(np.zeros((1, 3)), 4.0)  # side 16, dx = 0.25, r_s = 0.3125
    corner, side = oracle_mod.pm_region_isolated(pos)
    rs = 1.25 * side / ng
    d = rng.standard_normal((60, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = rng.uniform(8 * rs, 0.3 * side, 60)
    probes = d * r[:, None]
    pos = np.vstack([pos, probes])
    mass = np.zeros(len(pos), np.float32)
    mass[0] = 1.0
    phi = oracle_mod.pm_potential_isolated(pos, mass, corner, side, ng, rs)
    a, p = oracle_mod.pm_interpolate_isolated(phi, probes, corner, side, ng)
    fr = -(a * d).sum(1) * r ** 2
    assert np.abs(fr - 1).max() < 0.01
    assert np.abs(-p * r - 1).max() < 0.01
    assert np.abs(a - (a * d).sum(1)[:, None] * d).max() < 0.01 / (8 * rs) ** 2  # radial


def test_treepm_isolated_converges_to_direct_sum(oracle_mod):
    # short-range tree (small opening angle) plus isolated PM against the FP64
    # direct sum: the error comes from the mesh at the split scale, so it
    # shrinks as r_s covers more mesh cells
    n = 3000
    pos, mass = W.plummer(n, 12)
    tg = np.arange(0, n, 7)
    exact, _ = oracle_mod.direct(pos, mass, tg, 1.0, 0.01)
    med = []
    for asmth in (1.25, 2.5):
        a, _, _ = oracle_mod.treepm_isolated(pos, mass, tg, 64, asmth, 4.5, 1.0, 0.01, theta=0.2)
        e = np.linalg.norm(a - exact, axis=1) / np.linalg.norm(exact, axis=1)
        med.append(np.median(e))
    assert med[1] < 0.5 * med[0]
    assert med[1] < 2e-3
