"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module draws particle sets and request streams and nothing else: it holds
none of the force method's arithmetic (no keys, trees, kernels or meshes).  The
paper's gravity examples start from external initial-condition generators and
stored reference runs that are not available here, so every workload is drawn
from closed-form distributions with a fixed seed (PCG64):

* ``plummer``       -- Plummer sphere, total mass M, scale radius a, G = 1.
* ``hernquist``     -- Hernquist halo truncated at ``rmax`` (default 100 a).
* ``zeldovich``     -- unit periodic box, n^3 lattice displaced by a first-order
                       (Zel'dovich) Gaussian field with P(k) ~ k^-2 (spherical
                       cut at the lattice Nyquist wavenumber).
* ``timebins``      -- power-of-two time bins from a seeded density proxy; the
                       hierarchy of active sets of the paper's local time
                       stepping (Section 7.2).
* ``request_sizes`` -- log-uniform request sizes for batched active sets.
* ``serving_catalogue`` / ``poisson_arrivals`` -- the served-system stream.

Every function returns numpy arrays: positions float64 (n, 3), masses float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "plummer",
    "hernquist",
    "zeldovich",
    "lattice",
    "random_targets",
    "timebins",
    "substep_active_bins",
    "request_sizes",
    "root_shift",
    "SystemSpec",
    "serving_catalogue",
    "poisson_arrivals",
    "CONFIG_SEEDS",
]

# One seed per workload: 1000 + workload number (Plummer 8192 = 1, Hernquist
# 2^20 = 2, periodic Zel'dovich box = 3, time-bin batching = 4, serving = 5).
CONFIG_SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere (cos(theta) uniform, phi uniform)."""
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def plummer(n: int, seed: int, a: float = 1.0, M: float = 1.0, with_vel: bool = False):
    """Plummer sphere of ``n`` equal-mass particles (G = 1).

    Radii invert the cumulative mass M(<r)/M = r^3/(r^2+a^2)^{3/2}:
    r = a / sqrt(u^{-2/3} - 1), u ~ U(0, 1).  Velocities (optional,
    diagnostics only) use the rejection sampler of Aarseth, Henon & Wielen
    (1974) for q = v / v_esc with g(q) = q^2 (1 - q^2)^{7/2}.
    """
    rng = _rng(seed)
    u = rng.uniform(0.0, 1.0, n)
    u = np.clip(u, 1e-300, 1.0 - 1e-16)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(rng, n)
    mass = np.full(n, M / n, dtype=np.float32)
    if not with_vel:
        return pos.astype(np.float64), mass
    q = np.empty(n)
    filled = 0
    while filled < n:
        m = 2 * (n - filled) + 16
        x = rng.uniform(0.0, 1.0, m)
        y = rng.uniform(0.0, 0.1, m)
        ok = x[y < x * x * (1.0 - x * x) ** 3.5]
        take = min(len(ok), n - filled)
        q[filled:filled + take] = ok[:take]
        filled += take
    vesc = math.sqrt(2.0 * M / a) * (1.0 + (r / a) ** 2) ** (-0.25)
    vel = (q * vesc)[:, None] * _isotropic(rng, n)
    return pos.astype(np.float64), mass, vel


def hernquist(n: int, seed: int, a: float = 1.0, M: float = 1.0, rmax: float = 100.0):
    """Hernquist halo of ``n`` equal-mass particles truncated at ``rmax``.

    The cumulative mass is M(<r)/M = (r/(r+a))^2, so with s ~ U[0, s_max),
    s_max = (rmax/(rmax+a))^2, r = a sqrt(s) / (1 - sqrt(s)).
    """
    rng = _rng(seed)
    smax = (rmax / (rmax + a)) ** 2
    s = rng.uniform(0.0, smax, n)
    rs = np.sqrt(s)
    r = a * rs / (1.0 - rs)
    pos = r[:, None] * _isotropic(rng, n)
    mass = np.full(n, M / n, dtype=np.float32)
    return pos.astype(np.float64), mass


def clusters_with_outliers(n: int, seed: int, n_a: int = 2030):
    """Two Plummer clusters (scale 1) 600 units apart per axis, with five
    isolated particles between them, in different directions (one at 4e4):
    a stress case for walk frames.  In key order one 32-particle chunk runs
    from the end of one cluster past four isolated particles into the other
    cluster, and another starts with the farthest particle."""
    pa, _ = plummer(n_a, seed)
    pb, _ = plummer(n - n_a - 5, seed + 1)
    far = np.array([[300.0, -300.0, -300.0], [-300.0, 300.0, -300.0], [300.0, 300.0, -300.0],
                    [-300.0, -300.0, 300.0], [3.0e4, -3.0e4, 300.0]])
    pos = np.concatenate([pa - 300.0, far, pb + 300.0])
    return pos, np.full(n, 1.0 / n, np.float32)


def lattice(ngrid: int, box: float = 1.0) -> np.ndarray:
    """Unperturbed cubic lattice of ngrid^3 points at (i, j, k) * box / ngrid."""
    i = np.arange(ngrid, dtype=np.float64) * (box / ngrid)
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)


def zeldovich(ngrid: int, seed: int, rms_frac: float = 0.3, box: float = 1.0, M: float = 1.0):
    """Lattice displaced by a first-order Gaussian displacement field.

    delta(k) is white noise times sqrt(P(k)) with P(k) ~ k^-2 for |k| below the
    lattice Nyquist wavenumber (spherical cut; modes on a Nyquist plane and the
    k = 0 mode are dropped).  The displacement is psi(k) = i k / k^2 delta(k),
    rescaled so that the rms of |psi| equals ``rms_frac`` lattice spacings.
    Positions are wrapped into [0, box).
    """
    rng = _rng(seed)
    white = rng.standard_normal((ngrid, ngrid, ngrid))
    wk = np.fft.rfftn(white)
    f = np.fft.fftfreq(ngrid, d=1.0 / ngrid)
    fz = np.fft.rfftfreq(ngrid, d=1.0 / ngrid)
    nx, ny, nz = np.meshgrid(f, f, fz, indexing="ij")
    n2 = nx * nx + ny * ny + nz * nz
    half = ngrid // 2
    keep = (n2 > 0) & (n2 <= half * half)
    keep &= (np.abs(nx) < half) & (np.abs(ny) < half) & (nz < half)
    amp = np.zeros_like(n2)
    amp[keep] = 1.0 / np.sqrt(n2[keep])  # sqrt(P) with P ~ k^-2
    dk = wk * amp
    inv = np.zeros_like(n2)
    inv[keep] = 1.0 / n2[keep]
    disp = []
    for comp in (nx, ny, nz):
        psik = 1j * comp * inv * dk
        disp.append(np.fft.irfftn(psik, s=(ngrid, ngrid, ngrid), axes=(0, 1, 2)).ravel())
    psi = np.stack(disp, axis=1)
    rms = math.sqrt(float(np.mean(np.sum(psi * psi, axis=1))))
    psi *= (rms_frac * box / ngrid) / rms
    pos = lattice(ngrid, box) + psi
    pos = np.mod(pos, box)
    pos[pos >= box] -= box  # np.mod can return box for tiny negatives
    n = ngrid ** 3
    mass = np.full(n, M / n, dtype=np.float32)
    return pos.astype(np.float64), mass


def random_targets(n: int, k: int, seed: int) -> np.ndarray:
    """``k`` distinct particle indices out of ``n`` (sorted ascending), uint32."""
    rng = _rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.uint32)


def root_shift(seed: int) -> np.ndarray:
    """Three uniform numbers in [0, 1): the random tree-root placement drawn per
    tree construction (Section 3.1, randomised domain centre / box shift)."""
    return _rng(seed ^ 0x5EED).uniform(0.0, 1.0, 3)


def two_species(n_dm: int, n_star: int, seed: int, h_dm: float = 0.005, h_star: float = 0.001,
                star_scale: float = 0.1, star_mass_frac: float = 0.1):
    """Two collisionless species with their own softening: a Hernquist halo
    (M = 1 - star_mass_frac, a = 1, spline support h_dm) around a compact
    Plummer sphere of stars (M = star_mass_frac, scale star_scale, support
    h_star), shuffled together.  Returns (pos, mass, hsoft, species)."""
    rng = _rng(seed)
    p_dm, m_dm = hernquist(n_dm, seed)
    p_st, m_st = plummer(n_star, seed + 1)
    pos = np.concatenate([p_dm, p_st * star_scale])
    mass = np.concatenate([m_dm * (1.0 - star_mass_frac), m_st * star_mass_frac]).astype(np.float32)
    hsoft = np.concatenate([np.full(n_dm, h_dm), np.full(n_star, h_star)]).astype(np.float32)
    species = np.concatenate([np.zeros(n_dm, np.int8), np.ones(n_star, np.int8)])
    order = rng.permutation(n_dm + n_star)
    return pos[order], mass[order], hsoft[order], species[order]


def timebins(pos: np.ndarray, seed: int, nbins: int = 8, a: float = 1.0, M: float = 1.0,
             scatter: float = 0.3) -> np.ndarray:
    """Power-of-two time bins (0 = longest step, nbins-1 = shortest).

    A density proxy (the analytic Hernquist density at each radius times seeded
    lognormal scatter) sets a step dt ~ rho^{-1/2}.  Bins are filled by quantile
    of dt so that the particles active on a substep of kind b form the
    fractions 1, 1/2, ..., 1/2^{nbins-1} of the set: the densest 1/2^{nbins-1}
    go to the finest bin, the next 1/2^{nbins-1} to the one above, then
    1/2^{nbins-2}, ..., and the sparsest half to bin 0.
    """
    rng = _rng(seed)
    r = np.sqrt(np.sum(pos * pos, axis=1))
    r = np.maximum(r, 1e-6 * a)
    rho = M * a / (2.0 * math.pi * r * (r + a) ** 3)
    rho = rho * np.exp(scatter * rng.standard_normal(len(r)))
    dt = rho ** -0.5
    order = np.argsort(dt, kind="stable")
    n = len(pos)
    bins = np.zeros(n, dtype=np.int32)
    # the fraction of particles in bins >= b is 2^-b (b >= 1); bin 0 takes the rest
    start = 0
    for b in range(nbins - 1, 0, -1):
        end = max(int(round(2.0 ** -b * n)), start)
        bins[order[start:end]] = b
        start = end
    bins[order[start:]] = 0
    return bins


def substep_active_bins(step: int, nbins: int = 8) -> int:
    """Lowest bin that is active on substep ``step`` of a 2^{nbins-1} cycle:
    bin b is active when step is a multiple of 2^{nbins-1-b}."""
    cycle = 1 << (nbins - 1)
    s = step % cycle
    if s == 0:
        return 0
    tz = (s & -s).bit_length() - 1
    return nbins - 1 - tz


def request_sizes(total: int, seed: int, lo: int = 64, hi: int = 65536) -> np.ndarray:
    """Log-uniform request sizes in [lo, hi] that add up to ``total``."""
    rng = _rng(seed)
    out = []
    left = total
    while left > 0:
        s = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        s = max(1, min(s, left))
        out.append(s)
        left -= s
    return np.asarray(out, dtype=np.int64)


@dataclass(frozen=True)
class SystemSpec:
    """One served system: a Plummer or Hernquist set drawn from (seed, sid)."""

    sid: int
    n: int
    profile: str  # "plummer" | "hernquist"
    seed: int
    h: float

    def particles(self):
        if self.profile == "plummer":
            return plummer(self.n, self.seed)
        return hernquist(self.n, self.seed)

    def particles_on_device(self, torch, device):
        """The same profile drawn on ``device`` with torch's generator seeded
        from ``seed`` (another sample than ``particles()``; for large served
        catalogues whose host generation would dominate): FP64 positions,
        FP32 masses, both device tensors."""
        g = torch.Generator(device=device)
        g.manual_seed(self.seed)
        u = torch.rand(self.n, dtype=torch.float64, device=device, generator=g)
        if self.profile == "plummer":
            u = u.clamp(1e-300, 1.0 - 1e-16)
            r = 1.0 / torch.sqrt(u ** (-2.0 / 3.0) - 1.0)
        else:
            rs = torch.sqrt(u * (100.0 / 101.0) ** 2)
            r = rs / (1.0 - rs)
        d = torch.randn(self.n, 3, dtype=torch.float64, device=device, generator=g)
        d = d / torch.linalg.vector_norm(d, dim=1, keepdim=True).clamp_min(1e-300)
        pos = (r[:, None] * d).contiguous()
        mass = torch.full((self.n,), 1.0 / self.n, dtype=torch.float32, device=device)
        return pos, mass


def serving_catalogue(count: int, seed: int, nmin: int = 1 << 12, nmax: int = 1 << 20):
    """``count`` system specs: N log-uniform in [nmin, nmax], profile 50/50,
    softening as the Plummer (h = 0.01) and Hernquist (h = 0.005) workloads."""
    rng = _rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), count)).astype(np.int64)
    prof = rng.integers(0, 2, count)
    seeds = rng.integers(1, 2**31 - 1, count)
    cat = []
    for i in range(count):
        p = "plummer" if prof[i] == 0 else "hernquist"
        cat.append(SystemSpec(i, int(ns[i]), p, int(seeds[i]), 0.01 if p == "plummer" else 0.005))
    return cat


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with mean ``rate`` per second."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))
