"""The stored exact forces (tests/golden/exact_sums.npz, written by
tests/golden/make_exact_sums.py with the FP64 oracle) against the oracle
itself on a subset of the targets: the bench's accuracy figures rest on them."""
import os

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
EXACT = os.path.join(HERE, "golden", "exact_sums.npz")


@pytest.fixture(scope="module")
def ex():
    with np.load(EXACT) as f:
        return {k: f[k] for k in f.files}


def close(a, b, rtol=1e-10):
    np.testing.assert_allclose(a, b, rtol=rtol, atol=rtol * np.abs(b).max())


def test_hernquist_direct_sum(oracle_mod, ex):
    pos, mass = W.hernquist(1 << 20, W.CONFIG_SEEDS[2])
    tg = ex["hernquist_targets"]
    assert len(tg) == 4096 and len(np.unique(tg)) == 4096
    sub = np.arange(0, 4096, 171)
    a, p = oracle_mod.direct(pos, mass, tg[sub], 1.0, 0.005)
    close(a, ex["hernquist_acc"][sub])
    close(p, ex["hernquist_pot"][sub])


def test_zeldovich_ewald_sum(oracle_mod, ex):
    pos, mass = W.zeldovich(128, W.CONFIG_SEEDS[3])
    tg = ex["zeldovich_targets"]
    assert len(tg) == 2048
    sub = np.arange(0, 2048, 511)
    a, _ = oracle_mod.ewald(pos, mass, tg[sub], 1.0, 1.0)
    close(a, ex["zeldovich_acc"][sub])


def test_two_species_direct_sum(oracle_mod, ex):
    pos, mass, hs, _ = W.two_species(1 << 20, 1 << 18, W.CONFIG_SEEDS[2])
    tg = ex["two_species_targets"]
    sub = np.arange(0, 4096, 257)
    a, _ = oracle_mod.direct_soft(pos, mass, hs, tg[sub], 1.0)
    close(a, ex["two_species_acc"][sub])


def test_plummer_direct_sum(oracle_mod, ex):
    pos, mass = W.plummer(8192, W.CONFIG_SEEDS[1])
    np.testing.assert_array_equal(ex["plummer_targets"], np.arange(8192))
    a, p = oracle_mod.direct(pos, mass, np.arange(0, 8192, 97), 1.0, 0.01)
    close(a, ex["plummer_acc"][::97])
    # Newton's third law over the whole set: the stored forces are a direct sum
    m = mass.astype(np.float64)[:, None]
    assert np.abs((m * ex["plummer_acc"]).sum(0)).max() <= 1e-12 * np.abs(m * ex["plummer_acc"]).sum()
