"""FP64 oracle of gravitational time stepping with a power-of-two time-bin
hierarchy (paper Sec. 7.1-7.3).  Test infrastructure: only the tests, the
package's smoke check and the bench's CPU baseline may use it; the GPU path
shares no code with it.

What it computes, in the paper's order:

* Sec. 7.1, the gravity time-step criterion: a particle's step may not exceed
  sqrt(2 C_grav eps / |a|) (the paper prints the inequality with ">="; as an
  upper bound on the step it must read "<=");
* Sec. 7.2, local time stepping: a cycle of length T is cut into 2^N equal
  ticks; bin b (0 <= b <= N) has the step T / 2^b, so bin 0 is the longest
  and bin N the shortest, and bin b is due at every tick that is a multiple
  of 2^(N-b).  A particle takes the bin of the largest step not above its
  criterion.  It may always move to a shorter step; it moves to a longer one
  only onto a bin that is due at the current tick (shorter steps stay nested
  in longer ones) -- when the bin it asks for is not due, it takes the
  longest step between that bin and its current one that is due;
* Sec. 7.3, kick-drift-kick leapfrog: a particle's step opens with a half
  kick v += a dt/2 and closes with another with the force at the step's end;
  positions of all particles drift every tick with their current velocity
  (which, between a particle's kicks, is its mid-step velocity), and the tree
  is built anew at every tick (Sec. 3.1) for the forces on the particles due.
"""
from __future__ import annotations

import math

import numpy as np


def gravity_dt(amag, c_grav: float, eps: float):
    """Largest step the criterion allows: sqrt(2 C_grav eps / |a|) (inf for a = 0)."""
    amag = np.asarray(amag, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.sqrt(2.0 * c_grav * eps / amag)


def bin_for_dt(dt_max, dt_tick: float, nbins: int):
    """Bin of the largest step T / 2^b = 2^(N-b) dt_tick with step <= dt_max
    (N = nbins - 1); bin N when even the shortest step exceeds dt_max."""
    n = nbins - 1
    dt_max = np.atleast_1d(np.asarray(dt_max, dtype=np.float64))
    out = np.full(dt_max.shape, n, dtype=np.int64)
    for i, d in enumerate(dt_max):
        for b in range(0, n + 1):
            if math.ldexp(dt_tick, n - b) <= d:
                out[i] = b
                break
    return out


def due(bins, tick: int, nbins: int):
    """Whether bin b is due at ``tick``: tick a multiple of 2^(N-b)."""
    n = nbins - 1
    bins = np.asarray(bins)
    return (tick % (1 << (n - bins))) == 0


def next_bin(b_want, b_old, tick: int, nbins: int):
    """Sec. 7.2 hierarchy rule: a shorter step is always allowed; a longer one
    only onto a bin due at ``tick``: the longest due step in [b_want, b_old]."""
    b_want = np.atleast_1d(np.asarray(b_want, dtype=np.int64))
    b_old = np.atleast_1d(np.asarray(b_old, dtype=np.int64))
    out = b_want.copy()
    for i in range(len(out)):
        if b_want[i] < b_old[i]:
            b = b_want[i]
            while not due(b, tick, nbins):
                b += 1
            out[i] = b
    return out


class Hierarchy:
    """Positions (FP64), velocities (FP64) and time bins of n particles
    integrated tick by tick.  ``forces(x, ids, amag_old)`` returns the FP64
    accelerations (len(ids), 3) on particles ``ids`` from all particles at
    positions x; ``amag_old`` is None for the first evaluation (geometric
    criterion) and the particles' previous |a| afterwards (relative
    criterion)."""

    def __init__(self, pos, vel, forces, dt_tick: float, nbins: int, c_grav: float, eps: float,
                 box: float = 0.0):
        self.x = np.array(pos, dtype=np.float64)
        self.v = np.array(vel, dtype=np.float64)
        self.forces = forces
        self.dt_tick, self.nbins, self.c_grav, self.eps, self.box = dt_tick, nbins, c_grav, eps, box
        self.tick = 0
        n = len(self.x)
        ids = np.arange(n)
        a = forces(self.x, ids, None)
        self.a = a
        self.amag = np.sqrt(np.sum(a * a, axis=1))
        # tick 0 is due for every bin: any bin may be taken
        self.bins = bin_for_dt(gravity_dt(self.amag, c_grav, eps), dt_tick, nbins)
        self.v += a * self.step(self.bins)[:, None] * 0.5
        self.n_forces = n

    def step(self, bins):
        return np.ldexp(self.dt_tick, (self.nbins - 1) - np.asarray(bins))

    def advance(self):
        """One tick: drift everything, then close and reopen the steps of the
        particles due at the new tick."""
        self.x += self.v * self.dt_tick
        if self.box > 0.0:
            self.x -= np.floor(self.x / self.box) * self.box
            self.x[self.x >= self.box] -= self.box
        self.tick += 1
        t = self.tick % (1 << (self.nbins - 1))
        ids = np.nonzero(due(self.bins, t, self.nbins))[0]
        if len(ids) == 0:
            return ids
        a = self.forces(self.x, ids, self.amag[ids])
        self.n_forces += len(ids)
        old = self.bins[ids]
        self.v[ids] += a * self.step(old)[:, None] * 0.5  # closes the step
        amag = np.sqrt(np.sum(a * a, axis=1))
        want = bin_for_dt(gravity_dt(amag, self.c_grav, self.eps), self.dt_tick, self.nbins)
        new = next_bin(want, old, t, self.nbins)
        self.bins[ids] = new
        self.v[ids] += a * self.step(new)[:, None] * 0.5  # opens the next one
        self.amag[ids] = amag
        self.a[ids] = a
        return ids

    def synced_velocities(self):
        """Velocities at the current tick, v - a dt/2 with each particle's last
        force and current step; valid at a tick where every bin is due (every
        step has just been reopened)."""
        return self.v - self.a * self.step(self.bins)[:, None] * 0.5
