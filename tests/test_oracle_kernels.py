"""Pins for the oracle's pair laws (spline softening, TreePM split).

Each check ties the oracle to something other than its own formulas:
quadrature of the cubic-spline density, the paper's stated zero-lag
potential, numerical differentiation, and the 3-D Fourier transform that the
paper's k-space filter exp(-k^2 r_s^2) fixes.
"""
import math

import numpy as np
import pytest
from scipy import integrate

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def m4_density(r, h):
    """Cubic-spline (M4) density of unit mass with support h."""
    u = r / h
    norm = 8.0 / (math.pi * h ** 3)
    if u < 0.5:
        return norm * (1.0 - 6.0 * u * u + 6.0 * u ** 3)
    if u < 1.0:
        return norm * 2.0 * (1.0 - u) ** 3
    return 0.0


def enclosed(r, h):
    return integrate.quad(lambda s: 4.0 * math.pi * s * s * m4_density(s, h), 0.0, min(r, h),
                          points=[0.5 * h], epsabs=1e-15, epsrel=1e-13, limit=200)[0]


def potential_by_quadrature(r, h):
    """phi(r)/(G m) = -[M(<r)/r + int_r^h 4 pi s rho(s) ds]."""
    outer = 0.0
    if r < h:
        outer = integrate.quad(lambda s: 4.0 * math.pi * s * m4_density(s, h), r, h, points=[0.5 * h]
                               if r < 0.5 * h else None, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    return -(enclosed(r, h) / r + outer)


def test_zero_lag_potential_is_minus_one_over_eps(oracle_mod):
    # Sec. 3.2: the potential of a point mass at zero lag is -G m / eps and the
    # force is Newtonian from 2.8 eps on, so h = 2.8 eps.
    eps = 0.37
    h = 2.8 * eps
    assert oracle_mod.kpot(0.0, h) == pytest.approx(-1.0 / eps, rel=1e-14)


@pytest.mark.parametrize("h", [0.01, 1.0, 3.5])
def test_newtonian_beyond_support(oracle_mod, h):
    for r in (h, 1.0001 * h, 2.0 * h, 17.0 * h):
        assert oracle_mod.kforce(r, h) * r ** 3 == pytest.approx(1.0, rel=1e-14)
        assert oracle_mod.kpot(r, h) * r == pytest.approx(-1.0, rel=1e-14)


def test_enclosed_mass_is_one():
    assert enclosed(1.0, 1.0) == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("u", [1e-3, 0.05, 0.2, 0.37, 0.4999, 0.5, 0.5001, 0.63, 0.8, 0.95, 0.999])
def test_spline_matches_quadrature_of_density(oracle_mod, u):
    h = 0.7
    r = u * h
    kf_q = enclosed(r, h) / r ** 3
    assert oracle_mod.kforce(r, h) == pytest.approx(kf_q, rel=1e-11)
    assert oracle_mod.kpot(r, h) == pytest.approx(potential_by_quadrature(r, h), rel=1e-11)


@pytest.mark.parametrize("u0", [0.5, 1.0])
def test_spline_continuity(oracle_mod, u0):
    h = 1.3
    lo, hi = u0 * h * (1 - 1e-12), u0 * h * (1 + 1e-12)
    assert oracle_mod.kforce(lo, h) == pytest.approx(oracle_mod.kforce(hi, h), rel=1e-9)
    assert oracle_mod.kpot(lo, h) == pytest.approx(oracle_mod.kpot(hi, h), rel=1e-9)


def test_force_is_minus_gradient_of_potential(oracle_mod):
    h = 1.0
    for r in np.linspace(0.05, 1.5, 23):
        d = 1e-6
        dphi = (oracle_mod.kpot(r + d, h) - oracle_mod.kpot(r - d, h)) / (2 * d)
        # radial acceleration -dphi/dr equals -r kforce(r)
        assert -dphi == pytest.approx(-r * oracle_mod.kforce(r, h), rel=1e-7)


def test_short_range_force_factor_from_potential(oracle_mod):
    # g_s(r) must be the force of the short-range potential -erfc(r/2rs)/r,
    # relative to Newton: g_s = -r^2 d/dr [erfc(r/2rs)/r].
    rs = 0.3
    for r in np.linspace(0.01, 2.0, 31):
        d = 1e-6 * max(r, 0.1)
        f = lambda x: oracle_mod.gshort_pot(x, rs) / x
        num = -r * r * (f(r + d) - f(r - d)) / (2 * d)
        assert oracle_mod.gshort_force(r, rs) == pytest.approx(num, rel=1e-6, abs=1e-9)


def test_short_range_potential_matches_kspace_filter(oracle_mod):
    # Sec. 3.4: the long-range potential is Phi_k exp(-k^2 rs^2), so the
    # short-range kernel erfc(r/2rs)/r must transform to 4 pi / k^2 (1 - exp(-k^2 rs^2)).
    rs = 0.25
    for k in (0.7, 2.0, 5.0, 11.0):
        # 3-D transform of a radial f: (4 pi / k) int_0^inf r f(r) sin(k r) dr
        val = integrate.quad(lambda r: oracle_mod.gshort_pot(r, rs), 0.0, 40.0 * rs, weight="sin", wvar=k,
                             limit=400, epsabs=1e-14)[0]
        ft = 4.0 * math.pi / k * val
        assert ft == pytest.approx(4.0 * math.pi / k ** 2 * (1.0 - math.exp(-k * k * rs * rs)), rel=1e-8)


def test_short_range_limits(oracle_mod):
    rs = 0.1
    assert oracle_mod.gshort_force(0.0, rs) == 1.0
    assert oracle_mod.gshort_pot(0.0, rs) == 1.0
    # decays faster than any power beyond a few rs
    assert oracle_mod.gshort_force(10 * rs, rs) < 1e-9
