"""Pins of the Ewald-corrected periodic tree oracle (Sec. 3.1: the mirrored
images summed by the Ewald technique, no mesh): the correction's closed-form
limits, its agreement with the independent Ewald sum of orc_ewald (another
splitting, another code path), the table interpolation error, and the whole
walk converging to the Ewald-summed force as the opening angle shrinks."""
import math

import numpy as np
import pytest

import workloads as W


def test_correction_small_separation_is_the_background_pull(oracle_mod):
    # the lattice images cancel to first order; the neutralising background
    # (-1/V around the source) pushes the target away: -(4 pi / 3 V) d
    for d in ([0.003, 0.004, -0.002], [0.0, 0.0, 0.005], [-0.004, 0.001, 0.0]):
        c = oracle_mod.ewald_correction(1.0, d)
        np.testing.assert_allclose(c[:3], -4 * math.pi / 3 * np.array(d), rtol=2e-3, atol=1e-12)


def test_correction_cancels_the_nearest_image_at_half_box(oracle_mod):
    # a target half a box from the source feels no net periodic force
    for box in (1.0, 3.0):
        c = oracle_mod.ewald_correction(box, [0.5 * box, 0.0, 0.0])
        assert c[0] == pytest.approx(-1.0 / (0.5 * box) ** 2, rel=1e-12)
        assert abs(c[1]) < 1e-12 and abs(c[2]) < 1e-12
        c = oracle_mod.ewald_correction(box, [0.5 * box] * 3)
        np.testing.assert_allclose(c[:3], -np.full(3, 0.5 * box) / (0.75 * box * box) ** 1.5, rtol=1e-12)


def test_correction_matches_the_ewald_sum(oracle_mod):
    rng = np.random.default_rng(3)
    for box in (1.0, 2.0):
        for _ in range(12):
            src = rng.uniform(0, box, 3)
            d = rng.uniform(-0.5, 0.5, 3) * box
            pos = np.array([src, (src - d) % box])
            mass = np.array([1.0, 0.0], np.float32)
            a, p = oracle_mod.ewald(pos, mass, np.array([1], np.uint32), 1.0, box)
            r = np.linalg.norm(d)
            c = oracle_mod.ewald_correction(box, d)
            np.testing.assert_allclose(a[0], d / r ** 3 + c[:3], rtol=0, atol=1e-6 * np.abs(a[0]).max() + 1e-12)
            assert p[0] == pytest.approx(-1.0 / r + c[3], abs=1e-6 / box)


def test_correction_is_odd_in_its_component(oracle_mod):
    d = np.array([0.21, -0.13, 0.37])
    c = oracle_mod.ewald_correction(1.0, d)
    for flip in ([-1, 1, 1], [1, -1, 1], [1, 1, -1]):
        f = np.array(flip)
        cf = oracle_mod.ewald_correction(1.0, d * f)
        np.testing.assert_allclose(cf[:3], c[:3] * f, rtol=1e-12, atol=1e-14)
        assert cf[3] == pytest.approx(c[3], rel=1e-12)


def test_pair_through_the_table_matches_the_ewald_sum(oracle_mod):
    # two particles: the walk's nearest image plus the interpolated correction
    rng = np.random.default_rng(8)
    for _ in range(20):
        pos = rng.uniform(0, 1, (2, 3))
        mass = np.array([1.0, 1e-30], np.float32)
        tree = oracle_mod.Tree(pos, mass, bucket=1, periodic=True, box=1.0)
        a, p, _ = tree.walk([1], 1.0, 1e-6, theta=0.01, ewald=True)
        e, pe = oracle_mod.ewald(pos, mass, np.array([1], np.uint32), 1.0, 1.0)
        # trilinear interpolation on the (box / 128) grid: ~h^2/8 of the
        # correction's curvature (4 pi / 3 from the background) per axis
        assert np.linalg.norm(a[0] - e[0]) <= 2e-4 * np.linalg.norm(e[0])
        assert abs(p[0] - pe[0]) <= 1.5e-4


def test_ewald_tree_converges_to_the_ewald_sum(oracle_mod):
    n = 12
    pos, mass = W.zeldovich(n, 6, rms_frac=0.3)
    tg = np.arange(0, n ** 3, 5).astype(np.uint32)
    e, pe = oracle_mod.ewald(pos, mass, tg, 1.0, 1.0)
    tree = oracle_mod.Tree(pos, mass, bucket=4, periodic=True, box=1.0, shift=tuple(W.root_shift(6)))
    errs = []
    for theta in (0.6, 0.3, 0.1):
        a, p, _ = tree.walk(tg, 1.0, 1e-4, theta=theta, ewald=True)
        errs.append(np.percentile(np.linalg.norm(a - e, axis=1) / np.linalg.norm(e, axis=1), 99))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-3, errs
    # potentials include each particle's own images and the background; the
    # trilinear table overestimates the convex correction by a nearly constant
    # ~h^2/8 x its curvature, and periodic potentials are compared up to a
    # constant
    dp = p - pe
    assert abs(dp.mean()) < 1e-4
    assert np.percentile(np.abs(dp - dp.mean()) / np.abs(pe).mean(), 99) < 1e-3
    # without the correction the nearest-image tree is far off
    a0, _, _ = tree.walk(tg, 1.0, 1e-4, theta=0.1)
    assert np.percentile(np.linalg.norm(a0 - e, axis=1) / np.linalg.norm(e, axis=1), 50) > 0.05
