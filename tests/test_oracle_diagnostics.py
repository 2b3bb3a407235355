"""Pins of the oracle's conservation diagnostics [Sec. 7]: closed forms for
constant fields, Newton's third law through the direct sum, and the potential
energy of the direct sum against the pairwise energy summed by brute force."""
import itertools

import numpy as np

import workloads as W


def test_constant_fields_closed_form(oracle_mod):
    n = 1000
    rng = np.random.default_rng(3)
    m = rng.uniform(0.5, 1.5, n)
    c, phi0, u = np.array([0.3, -1.2, 2.0]), -4.5, np.array([1.0, 2.0, -0.5])
    d = oracle_mod.diagnostics(m, np.tile(c, (n, 1)), np.full(n, phi0), np.tile(u, (n, 1)))
    M = m.sum()
    np.testing.assert_allclose(d["total_force"], M * c, rtol=1e-13)
    assert abs(d["force_scale"] - M * np.linalg.norm(c)) < 1e-12 * M * np.linalg.norm(c)
    assert abs(d["potential_energy"] - 0.5 * M * phi0) < 1e-12 * abs(0.5 * M * phi0)
    assert abs(d["kinetic_energy"] - 0.5 * M * (u @ u)) < 1e-12 * 0.5 * M * (u @ u)
    np.testing.assert_allclose(d["momentum"], M * u, rtol=1e-13)
    d0 = oracle_mod.diagnostics(m, np.tile(c, (n, 1)))
    assert d0["potential_energy"] == 0.0 and d0["kinetic_energy"] == 0.0 and not d0["momentum"].any()


def test_direct_sum_total_force_vanishes(oracle_mod):
    pos, mass = W.plummer(2000, 17)
    a, _ = oracle_mod.direct(pos, mass, np.arange(len(pos)), 1.0, 0.01)
    d = oracle_mod.diagnostics(mass, a)
    assert np.linalg.norm(d["total_force"]) < 1e-12 * d["force_scale"]


def test_direct_sum_potential_energy_is_the_pair_energy(oracle_mod):
    pos, mass = W.plummer(7, 5)
    h, G = 0.05, 1.3
    _, p = oracle_mod.direct(pos, mass, np.arange(7), G, h)
    pair = 0.0
    for i, j in itertools.combinations(range(7), 2):
        r = float(np.linalg.norm(pos[i] - pos[j]))
        pair += G * float(mass[i]) * float(mass[j]) * oracle_mod.kpot(r, h)
    d = oracle_mod.diagnostics(mass, np.zeros((7, 3)), p)
    assert abs(d["potential_energy"] - pair) < 1e-12 * abs(pair)
