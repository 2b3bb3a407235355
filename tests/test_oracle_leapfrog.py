"""Pins of the time-stepping oracle (oracle/leapfrog.py) against what the
paper and the mathematics fix: the bin a step criterion maps to (Sec. 7.2, a
table worked by hand), the nesting rule for longer steps, the one-bin case
against a textbook kick-drift-kick loop, a circular two-body orbit (closed
form), and time reversibility of the symmetric kicks."""
import math

import numpy as np
import pytest

from oracle import leapfrog as LF


def test_bin_for_dt_worked_table():
    # N = 3 (4 bins), tick 0.25: steps are 2.0 (bin 0), 1.0, 0.5, 0.25 (bin 3)
    cases = [(math.inf, 0), (5.0, 0), (2.0, 0), (1.9999, 1), (1.0, 1), (0.6, 2), (0.5, 2), (0.3, 3), (0.25, 3),
             (0.1, 3)]
    got = LF.bin_for_dt([d for d, _ in cases], 0.25, 4)
    assert list(got) == [b for _, b in cases]


def test_gravity_dt_closed_form():
    assert LF.gravity_dt(2.0, 0.025, 0.01) == pytest.approx(math.sqrt(2 * 0.025 * 0.01 / 2.0), rel=1e-15)
    assert LF.gravity_dt(0.0, 0.025, 0.01) == math.inf


def test_longer_steps_only_onto_due_bins():
    # N = 3: at tick t bin b is due when t is a multiple of 2^(3-b)
    #  tick 4: bins 1, 2, 3 due; tick 2: bins 2, 3; tick 1: bin 3; tick 0: all
    table = [  # (want, old, tick) -> new
        ((0, 2, 4), 1), ((0, 3, 2), 2), ((1, 3, 1), 3), ((0, 3, 0), 0), ((1, 2, 4), 1),
        ((3, 1, 5), 3), ((2, 0, 3), 2),  # shorter steps: always
        ((2, 2, 6), 2),
    ]
    for (want, old, tick), new in table:
        assert LF.next_bin(want, old, tick, 4)[0] == new, (want, old, tick)


def direct_forces(mass, h):
    import oracle

    def f(x, ids, amag_old):
        acc, _ = oracle.direct(x, mass, np.asarray(ids, dtype=np.uint32), 1.0, h, nthreads=1)
        return acc

    return f


def two_body():
    pos = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    vel = np.array([[0.0, 0.5, 0.0], [0.0, -0.5, 0.0]])  # omega = sqrt(G (m1 + m2) / d^3) = 1
    mass = np.array([0.5, 0.5], dtype=np.float32)
    return pos, vel, mass


def test_one_bin_is_textbook_leapfrog(oracle_mod):
    pos, vel, mass = two_body()
    f = direct_forces(mass, 1e-6)
    dt = 2 * math.pi / 64
    h = LF.Hierarchy(pos, vel, f, dt, 3, c_grav=1e-12, eps=1e-6)  # every particle on the finest bin
    assert (h.bins == 2).all()
    for _ in range(64):
        h.advance()
    # kick-drift-kick with a fixed step, written out
    x, v = pos.copy(), vel.copy()
    a = f(x, [0, 1], None)
    for _ in range(64):
        v = v + a * (dt * 0.5)
        x = x + v * dt
        a = f(x, [0, 1], None)
        v = v + a * (dt * 0.5)
    np.testing.assert_allclose(h.x, x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(h.synced_velocities(), v, rtol=0, atol=1e-13)


def test_circular_orbit_closes(oracle_mod):
    pos, vel, mass = two_body()
    f = direct_forces(mass, 1e-6)
    n_ticks = 1024
    h = LF.Hierarchy(pos, vel, f, 2 * math.pi / n_ticks, 4, c_grav=1e-12, eps=1e-6)
    for _ in range(n_ticks):
        h.advance()
    # one period later: leapfrog's phase error ~ (omega dt)^2 / 24 per radian
    assert np.abs(h.x - pos).max() < 1e-4
    v = h.synced_velocities()
    e0 = 0.5 * 0.5 * (0.25 + 0.25) - 0.25 / 1.0
    r = np.linalg.norm(h.x[0] - h.x[1])
    e1 = 0.5 * 0.5 * np.sum(v * v) - 0.25 / r
    assert abs(e1 - e0) < 1e-5 * abs(e0)


def test_time_reversible(oracle_mod):
    rng = np.random.default_rng(4)
    n = 48
    pos = rng.standard_normal((n, 3))
    vel = 0.3 * rng.standard_normal((n, 3))
    mass = np.full(n, 1.0 / n, np.float32)
    f = direct_forces(mass, 0.05)
    fwd = LF.Hierarchy(pos, vel, f, 0.01, 3, c_grav=1e-12, eps=0.05)
    for _ in range(40):
        fwd.advance()
    back = LF.Hierarchy(fwd.x, -fwd.synced_velocities(), f, 0.01, 3, c_grav=1e-12, eps=0.05)
    for _ in range(40):
        back.advance()
    np.testing.assert_allclose(back.x, pos, rtol=0, atol=1e-11)
    np.testing.assert_allclose(-back.synced_velocities(), vel, rtol=0, atol=1e-11)


def test_cycle_keeps_steps_nested(oracle_mod):
    import workloads as W

    pos, mass = W.plummer(400, 8)
    vel = np.zeros_like(pos)
    f = direct_forces(mass, 0.01)
    nb = 5
    h = LF.Hierarchy(pos, vel, f, 0.004, nb, c_grav=0.02, eps=0.01 / 2.8)
    assert len(set(h.bins.tolist())) >= 3  # the cycle exercises several bins
    forces = len(pos)
    for t in range(1, 1 << (nb - 1)):
        before = h.bins.copy()
        ids = h.advance()
        due = LF.due(before, t, nb)
        assert set(ids.tolist()) == set(np.nonzero(due)[0].tolist())
        assert (h.bins[~due] == before[~due]).all()  # a particle changes bin only at its step's end
        forces += len(ids)
        # a longer step only onto a bin due now, so the new step nests in the longer ones
        new, old = h.bins[ids], before[ids]
        assert ((new >= old) | (t % (1 << (nb - 1 - new)) == 0)).all()
    ids = h.advance()  # the end of the cycle: every particle is due
    assert len(ids) == len(pos)
    assert h.n_forces == forces + len(pos)


def eccentric_orbit_energy_error(LFmod):
    """Two equal masses on an e = 0.5 orbit (a = 1, G M = 1, period 2 pi),
    started at apocentre; the step criterion moves them between bins along
    the orbit.  Returns (relative energy error after one period, largest
    position offset from the start, bins used)."""
    import oracle

    e = 0.5
    vrel = math.sqrt((1 - e) / (1 + e))
    pos = np.array([[0.75, 0.0, 0.0], [-0.75, 0.0, 0.0]])
    vel = np.array([[0.0, vrel / 2, 0.0], [0.0, -vrel / 2, 0.0]])
    mass = np.array([0.5, 0.5], dtype=np.float32)
    f = direct_forces(mass, 1e-6)
    n_ticks = 1024
    h = LFmod.Hierarchy(pos, vel, f, 2 * math.pi / n_ticks, 4, c_grav=6.685e-5, eps=1.0)
    used = set(h.bins.tolist())
    for _ in range(n_ticks):
        h.advance()
        used |= set(h.bins.tolist())
    v = h.synced_velocities()
    r = np.linalg.norm(h.x[0] - h.x[1])
    e0 = 0.25 * np.sum(vel * vel) - 0.25 / 1.5
    e1 = 0.25 * np.sum(v * v) - 0.25 / r
    return abs(e1 - e0) / abs(e0), np.abs(h.x - pos).max(), used


def test_eccentric_orbit_across_bins(oracle_mod):
    de, dx, used = eccentric_orbit_energy_error(LF)
    assert len(used) >= 2  # the orbit changes bins
    assert de < 1e-5 and dx < 1e-3


def test_eccentric_orbit_pin_catches_a_wrong_closing_kick(oracle_mod, monkeypatch):
    # a planted mistake in the oracle: the closing half kick with the new step
    # instead of the one that ends -- second order is lost where bins change
    def advance_wrong(self):
        self.x += self.v * self.dt_tick
        self.tick += 1
        t = self.tick % (1 << (self.nbins - 1))
        ids = np.nonzero(LF.due(self.bins, t, self.nbins))[0]
        if len(ids) == 0:
            return ids
        a = self.forces(self.x, ids, self.amag[ids])
        amag = np.sqrt(np.sum(a * a, axis=1))
        want = LF.bin_for_dt(LF.gravity_dt(amag, self.c_grav, self.eps), self.dt_tick, self.nbins)
        new = LF.next_bin(want, self.bins[ids], t, self.nbins)
        self.v[ids] += a * self.step(new)[:, None] * 0.5
        self.bins[ids] = new
        self.v[ids] += a * self.step(new)[:, None] * 0.5
        self.amag[ids] = amag
        self.a[ids] = a
        return ids

    monkeypatch.setattr(LF.Hierarchy, "advance", advance_wrong)
    de, dx, _ = eccentric_orbit_energy_error(LF)
    assert not (de < 1e-5 and dx < 1e-3)
