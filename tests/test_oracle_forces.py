"""Pins for the oracle's forces: direct sum against closed-form profiles and
Newton's third law, the tree walk against the direct sum (theta -> 0 limit,
N = 2, multipole error order), Ewald against symmetry and its own splitting
independence, and the PM / TreePM split against the linear-theory closed form
and the Ewald sum."""
import math

import numpy as np
import pytest

import workloads as W


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


# ------------------------------------------------------------------ direct sum
def test_direct_two_particles_closed_form(oracle_mod):
    pos = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]])
    mass = np.array([0.25, 0.5], np.float32)
    acc, pot = oracle_mod.direct(pos, mass, np.array([0, 1]), 2.0, 0.01)
    d = pos[1] - pos[0]
    r = np.linalg.norm(d)
    np.testing.assert_allclose(acc[0], 2.0 * 0.5 * d / r ** 3, rtol=1e-14)
    np.testing.assert_allclose(acc[1], -2.0 * 0.25 * d / r ** 3, rtol=1e-14)
    assert pot[0] == pytest.approx(-2.0 * 0.5 / r, rel=1e-14)


def test_direct_momentum_conservation(oracle_mod):
    pos, mass = W.plummer(2048, 21)
    acc, _ = oracle_mod.direct(pos, mass, np.arange(2048), 1.0, 0.01)
    tot = (mass[:, None].astype(np.float64) * acc).sum(0)
    scale = (mass[:, None] * np.abs(acc)).sum()
    assert np.abs(tot).max() < 1e-14 * scale


def gauss_law_ok(pos, mass, acc, G, edges, nsig=4.0):
    """Gauss's law: the radial field averaged over a sphere is -G M(<r) / r^2.
    Each shell's particles sample that average; M(<r_i) counts the
    realisation's own particles inside r_i (the shells lie beyond the
    softening, so the enclosed point masses act as Newtonian)."""
    r = np.linalg.norm(pos, axis=1)
    order = np.argsort(r)
    menc = np.empty(len(r))
    menc[order] = np.cumsum(mass[order].astype(np.float64)) - mass[order]
    ar = (acc * pos).sum(1) / r
    dev = ar + G * menc / (r * r)
    for lo, hi in zip(edges[:-1], edges[1:]):
        s = (r >= lo) & (r < hi)
        scale = np.abs(G * menc[s] / r[s] ** 2).mean()
        if abs(dev[s].mean()) > nsig * dev[s].std() / math.sqrt(s.sum()) + 1e-4 * scale:
            return False
    return True


def test_direct_plummer_gauss_law_and_G_sensitivity(oracle_mod):
    pos, mass = W.plummer(8192, 1001)
    acc, _ = oracle_mod.direct(pos, mass, np.arange(8192), 1.0, 0.01)
    edges = np.array([0.1, 0.2, 0.35, 0.5, 0.7, 1.0, 1.4, 2.0, 3.0])
    assert gauss_law_ok(pos, mass, acc, 1.0, edges)
    # a 1% change of G must break the check (adapted from the paper's
    # gravity example, where a 1% change of G leaves the tolerance)
    assert not gauss_law_ok(pos, mass, acc * 1.01, 1.0, edges)
    assert not gauss_law_ok(pos, mass, acc * 0.99, 1.0, edges)


def test_direct_hernquist_profile(oracle_mod):
    pos, mass = W.hernquist(8192, 1002)
    acc, _ = oracle_mod.direct(pos, mass, np.arange(8192), 1.0, 0.005)
    edges = np.array([0.15, 0.3, 0.6, 1.0, 2.0, 4.0, 8.0, 20.0])
    assert gauss_law_ok(pos, mass, acc, 1.0, edges)
    # and the realisation follows the truncated Hernquist mass profile
    r = np.sort(np.linalg.norm(pos, axis=1))
    frac = np.arange(1, len(r) + 1) / len(r)
    model = (r / (r + 1.0)) ** 2 / (100.0 / 101.0) ** 2
    assert np.abs(frac - model).max() < 2.0 / math.sqrt(len(r))


# ------------------------------------------------------------------ tree walk
@pytest.mark.parametrize("bucket", [1, 8])
def test_walk_theta_to_zero_is_direct_sum(oracle_mod, bucket):
    pos, mass = W.plummer(2000, 31)
    tg = np.arange(2000)
    ad, pd = oracle_mod.direct(pos, mass, tg, 1.0, 0.02)
    tree = oracle_mod.Tree(pos, mass, bucket=bucket, shift=W.root_shift(5))
    a, p, n = tree.walk(tg, 1.0, 0.02, crit="bh", theta=1e-12)
    assert np.all(n == 1999)
    assert rel_err(a, ad).max() < 1e-12
    np.testing.assert_allclose(p, pd, rtol=1e-12)
    # relative criterion with alpha = 0 opens everything too
    a2, p2, n2 = tree.walk(tg, 1.0, 0.02, crit="rel", alpha=0.0, a_old=np.ones(2000, np.float32))
    assert np.all(n2 == 1999) and rel_err(a2, ad).max() < 1e-12


def test_walk_two_particles(oracle_mod):
    pos = np.array([[0.1, 0.2, 0.3], [2.0, -1.0, 0.5]])
    mass = np.array([0.5, 0.5], np.float32)
    tree = oracle_mod.Tree(pos, mass)
    a, p, n = tree.walk([0, 1], 1.0, 0.01, theta=0.7)
    ad, pd = oracle_mod.direct(pos, mass, np.array([0, 1]), 1.0, 0.01)
    np.testing.assert_allclose(a, ad, rtol=1e-14)
    assert list(n) == [1, 1]


def test_walk_monopole_error_is_quadrupole_order(oracle_mod):
    # a compact cluster seen from afar: the monopole about the centre of mass
    # (dipole zero) errs at O((L/d)^2)
    rng = np.random.default_rng(3)
    cl = rng.uniform(-0.5, 0.5, (200, 3)) * np.array([1.0, 0.6, 0.3])
    errs = []
    for d in (8.0, 16.0, 32.0):
        pos = np.vstack([cl, [[d, 0.3, -0.2]]])
        mass = np.full(len(pos), 1.0 / len(pos), np.float32)
        tree = oracle_mod.Tree(pos, mass, bucket=1, shift=(0.5, 0.5, 0.5))
        a, _, n = tree.walk([200], 1.0, 1e-3, theta=1.0, box_guard=True)
        ad, _ = oracle_mod.direct(pos, mass, np.array([200]), 1.0, 1e-3)
        errs.append(rel_err(a, ad)[0])
        assert n[0] < 20
    assert errs[0] > 0
    # quadrupole scaling: halving L/d cuts the error by about 4
    assert 2.5 < errs[0] / errs[1] < 6.0 and 2.5 < errs[1] / errs[2] < 6.0


def test_walk_accuracy_improves_with_theta(oracle_mod):
    pos, mass = W.plummer(4096, 41)
    tg = np.arange(0, 4096, 4)
    ad, _ = oracle_mod.direct(pos, mass, tg, 1.0, 0.01)
    tree = oracle_mod.Tree(pos, mass, bucket=4, shift=W.root_shift(7))
    p99 = []
    nint = []
    for th in (0.9, 0.6, 0.3):
        a, _, n = tree.walk(tg, 1.0, 0.01, theta=th)
        p99.append(np.percentile(rel_err(a, ad), 99))
        nint.append(n.mean())
    assert p99[0] > p99[1] > p99[2] and p99[2] < 5e-3
    assert nint[0] < nint[1] < nint[2]


def test_relative_criterion_bounds_error(oracle_mod):
    pos, mass = W.hernquist(8192, 17)
    tg = np.arange(0, 8192, 8)
    ad, _ = oracle_mod.direct(pos, mass, tg, 1.0, 0.005)
    tree = oracle_mod.Tree(pos, mass, bucket=8, shift=W.root_shift(8))
    a1, _, _ = tree.walk(tg, 1.0, 0.005, theta=0.5)
    aold = np.linalg.norm(a1, axis=1).astype(np.float32)
    prev = None
    for alpha in (0.01, 0.0025, 0.0005):
        a, _, n = tree.walk(tg, 1.0, 0.005, crit="rel", alpha=alpha, a_old=aold)
        p99 = np.percentile(rel_err(a, ad), 99)
        assert p99 < 8 * alpha
        if prev is not None:
            assert p99 < prev
        prev = p99


def test_walk_box_guard_never_accepts_own_node(oracle_mod):
    # with a huge opening angle only the box guard keeps a particle from
    # accepting a node that contains it; the self term never appears
    pos, mass = W.plummer(512, 51)
    tree = oracle_mod.Tree(pos, mass, bucket=2)
    a, p, n = tree.walk(np.arange(512), 1.0, 0.01, theta=100.0)
    assert np.all(np.isfinite(a)) and np.all(n >= 1)


@pytest.mark.parametrize("off,nint_guard", [(0.55, 4), (0.59, 4), (0.61, 3), (0.65, 3)])
def test_walk_box_guard_is_1_2_L(oracle_mod, off, nint_guard):
    # Sec. 3.1: a node is opened when the particle lies inside a cube of side
    # 1.2 L about the node's geometric centre, whatever the opening angle.  The
    # anchors fix the root (x0 = 0, L0 = 128); the pair at (65..66)^3 forms the
    # level-5 node [64, 68)^3 (centre 66, side 4); the probe sits at
    # x = 66 + off * 4 in its own leaf.  With theta = 100 only the guard can
    # open the pair's node: 2 anchors + 2 pair particles when opened, 2 + 1
    # monopole when not; without the guard the whole root is one monopole.
    pos = np.array([[0, 0, 0], [100, 100, 100], [65, 65, 65], [66, 66, 66], [66 + off * 4, 66, 66]], float)
    mass = np.full(5, 0.2, np.float32)
    tree = oracle_mod.Tree(pos, mass, bucket=1, shift=(0.0, 0.0, 0.0))
    assert list(tree.x0) == [0.0, 0.0, 0.0] and tree.L0 == 128.0
    _, _, n = tree.walk([4], 1.0, 1e-3, theta=100.0, box_guard=True)
    assert n[0] == nint_guard
    _, _, n = tree.walk([4], 1.0, 1e-3, theta=100.0, box_guard=False)
    assert n[0] == 1


@pytest.mark.parametrize("theta,nint", [(0.25, 4), (0.27, 3), (0.29, 3)])
def test_walk_bh_distance_is_to_the_centre_of_mass(oracle_mod, theta, nint):
    # Sec. 3.1 (reading A5): the geometric criterion compares L with theta
    # times the distance to the node's centre of mass, not to its geometric
    # centre.  The level-5 node [64, 68)^3 (side 4) holds a heavy particle
    # near its -x face and a light one near its +x face; from the probe at
    # x = 80, L / d is 0.258 to the centre of mass and 0.285 to the centre, so
    # theta = 0.27 accepts the node (3 interactions: 2 anchors + 1 monopole)
    # only under the centre-of-mass reading; the box guard is off.
    pos = np.array([[0, 0, 0], [100, 100, 100], [64.5, 66.5, 66.5], [67.5, 66.5, 66.5], [80.0, 66.5, 66.5]], float)
    mass = np.array([1e-6, 1e-6, 1.0, 1e-3, 1e-6], np.float32)
    tree = oracle_mod.Tree(pos, mass, bucket=1, shift=(0.0, 0.0, 0.0))
    assert list(tree.x0) == [0.0, 0.0, 0.0] and tree.L0 == 128.0
    _, _, n = tree.walk([4], 1.0, 1e-3, theta=theta, box_guard=False)
    assert n[0] == nint


@pytest.mark.parametrize("f,nint", [(0.99, 4), (1.01, 3)])
def test_relative_criterion_threshold(oracle_mod, f, nint):
    # Sec. 3.1: the relative criterion opens a node when G M L^2 exceeds
    # alpha |a_old| d^4 (d to the centre of mass, reading A6).  For the same
    # level-5 node as above (M = 1.001, L = 4) seen from x = 80 with G = 2 and
    # |a_old| = 1 the decision flips at alpha* = G M L^2 / d^4: just below it
    # the node is opened (4 interactions), just above it accepted (3).  A d^2,
    # a missing G or a missing M would move alpha* by far more than 1%.
    pos = np.array([[0, 0, 0], [100, 100, 100], [64.5, 66.5, 66.5], [67.5, 66.5, 66.5], [80.0, 66.5, 66.5]], float)
    mass = np.array([1e-6, 1e-6, 1.0, 1e-3, 1e-6], np.float32)
    tree = oracle_mod.Tree(pos, mass, bucket=1, shift=(0.0, 0.0, 0.0))
    M = float(mass[2]) + float(mass[3])
    com = (pos[2] * float(mass[2]) + pos[3] * float(mass[3])) / M
    d = np.linalg.norm(pos[4] - com)
    G = 2.0
    alpha_star = G * M * 4.0 ** 2 / d ** 4
    _, _, n = tree.walk([4], G, 1e-3, crit="rel", alpha=f * alpha_star, a_old=np.array([1.0], np.float32))
    assert n[0] == nint


@pytest.mark.parametrize("rcut,nint", [(11.9, 0), (12.1, 1), (15.0, 1)])
def test_treepm_cutoff_uses_the_distance_to_the_cube(oracle_mod, rcut, nint):
    # Sec. 3.4 (reading A9): a node is skipped when the particle's smallest
    # distance to the node's cube exceeds r_cut.  The level-5 node [64, 68)^3
    # is 12 from the probe at x = 80 (its centre of mass 15.5, its centre 14.0);
    # at theta = 0.4 the nodes above it open and it is accepted, so it adds one
    # interaction for any r_cut above 12 and none below.
    pos = np.array([[0, 0, 0], [100, 100, 100], [64.5, 66.5, 66.5], [67.5, 66.5, 66.5], [80.0, 66.5, 66.5]], float)
    mass = np.array([1e-6, 1e-6, 1.0, 1e-3, 1e-6], np.float32)
    tree = oracle_mod.Tree(pos, mass, bucket=1, shift=(0.0, 0.0, 0.0))
    _, _, n = tree.walk([4], 1.0, 1e-3, theta=0.4, treepm=True, rs=rcut / 4.5, rcut=rcut)
    assert n[0] == nint


# ------------------------------------------------------------------ Ewald
def test_ewald_splitting_independent(oracle_mod):
    pos, mass = W.zeldovich(8, 4, rms_frac=0.3)
    tg = np.arange(0, 512, 7)
    # truncation at erfc(5.5) ~ 1e-14 on both sides: only the splitting differs
    a1, p1 = oracle_mod.ewald(pos, mass, tg, 1.0, 1.0, *oracle_mod.ewald_params(1.0, 5.5, rreal_frac=0.3))
    a2, p2 = oracle_mod.ewald(pos, mass, tg, 1.0, 1.0, *oracle_mod.ewald_params(1.0, 5.5, rreal_frac=0.45))
    assert rel_err(a1, a2).max() < 1e-9
    np.testing.assert_allclose(p1, p2, rtol=1e-9)


def test_ewald_lattice_is_force_free(oracle_mod):
    n = 8
    pos = W.lattice(n)
    mass = np.full(n ** 3, 1.0 / n ** 3, np.float32)
    a, _ = oracle_mod.ewald(pos, mass, np.arange(0, n ** 3, 13), 1.0, 1.0)
    scale = (1.0 / n ** 3) / (1.0 / n) ** 2
    assert np.abs(a).max() < 1e-10 * scale


@pytest.mark.parametrize("probe", [[0.5, 0.5, 0.5], [0.5, 0.0, 0.0], [0.0, 0.5, 0.5]])
def test_ewald_symmetric_points_force_free(oracle_mod, probe):
    pos = np.array([[0.0, 0.0, 0.0], probe])
    mass = np.array([1.0, 1.0], np.float32)
    a, _ = oracle_mod.ewald(pos, mass, np.array([1]), 1.0, 1.0)
    assert np.abs(a).max() < 1e-10


def test_ewald_close_pair_is_newtonian(oracle_mod):
    pos = np.array([[0.3, 0.3, 0.3], [0.3 + 0.004, 0.3 + 0.003, 0.3]])
    mass = np.array([1.0, 1.0], np.float32)
    a, _ = oracle_mod.ewald(pos, mass, np.array([0]), 1.0, 1.0)
    d = pos[1] - pos[0]
    newton = d / np.linalg.norm(d) ** 3
    # correction from images and background is O(r / L^3) ~ 1e-7 relative
    assert rel_err(a, newton[None])[0] < 1e-6


def plane_wave(n, amp_frac, mode=2, offset=0.0):
    pos = W.lattice(n) + offset
    amp = amp_frac / n
    psi = amp * np.sin(2 * math.pi * mode * pos[:, 0])
    pos = pos.copy()
    pos[:, 0] = (pos[:, 0] + psi) % 1.0
    return pos, psi


def test_ewald_zeldovich_plane_wave(oracle_mod):
    # linear theory: a = 4 pi G rho_bar psi for a displaced lattice (rho_bar = 1)
    n = 16
    pos, psi = plane_wave(n, 1e-3)
    mass = np.full(n ** 3, 1.0 / n ** 3, np.float32)
    tg = np.arange(0, n ** 3, 5)
    a, _ = oracle_mod.ewald(pos, mass, tg, 1.0, 1.0)
    lin = 4 * math.pi * psi[tg]
    amp = np.abs(lin).max()
    assert np.abs(a[:, 0] - lin).max() < 0.03 * amp
    assert np.abs(a[:, 1:]).max() < 1e-6 * amp


# ------------------------------------------------------------------ PM / TreePM
def test_pm_long_range_plane_wave(oracle_mod):
    # the long-range part of the linear force is filtered by exp(-k^2 rs^2)
    # lattice points half a mesh cell off the mesh nodes: a particle sitting
    # exactly on a node with a tiny displacement meets the kink of the CIC
    # weights, which adds even harmonics of relative size ~ k dx / 2
    n, ng = 32, 64
    pos, psi = plane_wave(n, 1e-3, mode=3, offset=0.5 / ng)
    mass = np.full(n ** 3, 1.0 / n ** 3, np.float32)
    rs = 1.25 / ng
    phi = oracle_mod.pm_potential(pos, mass, 1.0, ng, rs)
    tg = np.arange(0, n ** 3, 3)
    a, _ = oracle_mod.pm_interpolate(phi, pos[tg], 1.0)
    k = 2 * math.pi * 3
    lin = 4 * math.pi * psi[tg] * math.exp(-k * k * rs * rs)
    amp = np.abs(lin).max()
    assert np.abs(a[:, 0] - lin).max() < 5e-3 * amp
    assert np.abs(a[:, 1:]).max() < 1e-6 * amp


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mesh_forces_single_mode_closed_forms(oracle_mod, axis):
    # Phi = A cos(k x_a + p) on the mesh nodes: the spectral derivative gives
    # -dPhi/dx_a = A k sin(k x_a + p) exactly, the 4-point difference gives it
    # times its transfer function (4/3 sin(k dx) - 1/6 sin(2 k dx)) / (k dx);
    # the other components vanish
    ng, m, A, p = 32, 3, 0.7, 0.4
    x = np.arange(ng) / ng
    k = 2 * math.pi * m
    shape = [1, 1, 1]
    shape[axis] = ng
    phi = np.broadcast_to((A * np.cos(k * x + p)).reshape(shape), (ng, ng, ng)).copy()
    want = np.broadcast_to((A * k * np.sin(k * x + p)).reshape(shape), (ng, ng, ng))
    f_ik = oracle_mod.mesh_forces(phi, 1.0, "ik")
    np.testing.assert_allclose(f_ik[axis], want, atol=1e-12 * A * k)
    kdx = k / ng
    tf = ((4.0 / 3.0) * math.sin(kdx) - (1.0 / 6.0) * math.sin(2 * kdx)) / kdx
    f_fd = oracle_mod.mesh_forces(phi, 1.0, "fd4")
    np.testing.assert_allclose(f_fd[axis], tf * want, atol=1e-12 * A * k)
    for other in range(3):
        if other != axis:
            assert np.abs(f_ik[other]).max() < 1e-12 * A * k
            assert np.abs(f_fd[other]).max() < 1e-12 * A * k
    # the Nyquist mode (alternating signs) has no derivative on a real mesh
    nyq = np.broadcast_to(((-1.0) ** np.arange(ng)).reshape(shape), (ng, ng, ng)).copy()
    assert np.abs(oracle_mod.mesh_forces(nyq, 1.0, "ik")[axis]).max() < 1e-12


def test_pm_long_range_plane_wave_spectral(oracle_mod):
    # the linear plane wave of test_pm_long_range_plane_wave with the spectral
    # gradient: the same filtered closed form
    n, ng = 32, 64
    pos, psi = plane_wave(n, 1e-3, mode=3, offset=0.5 / ng)
    mass = np.full(n ** 3, 1.0 / n ** 3, np.float32)
    rs = 1.25 / ng
    phi = oracle_mod.pm_potential(pos, mass, 1.0, ng, rs)
    tg = np.arange(0, n ** 3, 3)
    a, _ = oracle_mod.pm_interpolate(phi, pos[tg], 1.0, grad="ik")
    k = 2 * math.pi * 3
    lin = 4 * math.pi * psi[tg] * math.exp(-k * k * rs * rs)
    amp = np.abs(lin).max()
    assert np.abs(a[:, 0] - lin).max() < 5e-3 * amp
    assert np.abs(a[:, 1:]).max() < 1e-6 * amp


@pytest.mark.parametrize("grad", ["fd4", "ik"])
def test_pm_pair_force_matches_long_range_closed_form(oracle_mod, grad):
    # one unit mass: the mesh force at r = 2..4 r_s must follow the long-range
    # closed form g_l(r) / r^2, g_l = erf(x) - 2x/sqrt(pi) e^{-x^2}, x = r/2r_s,
    # less the uniform background's pull (4 pi / 3) r (periodic box, mean
    # density removed); CIC anisotropy leaves a few per cent of scatter
    ng = 32
    rs = 1.25 / ng
    rng = np.random.default_rng(2)
    for r in (2 * rs, 3 * rs, 4 * rs):
        ratios = []
        for _ in range(8):
            src = rng.uniform(0, 1, (1, 3))
            d = rng.standard_normal((40, 3))
            d /= np.linalg.norm(d, axis=1)[:, None]
            probes = (src + r * d) % 1.0
            pos = np.vstack([src, probes])
            mass = np.zeros(len(pos), np.float32)
            mass[0] = 1.0
            phi = oracle_mod.pm_potential(pos, mass, 1.0, ng, rs)
            a, _ = oracle_mod.pm_interpolate(phi, probes, 1.0, grad=grad)
            x = r / (2 * rs)
            gl = math.erf(x) - 2 * x / math.sqrt(math.pi) * math.exp(-x * x)
            expect = gl / r ** 2 - 4 * math.pi / 3 * r
            ratios.append(-(a * d).sum(1) / expect)
        ratios = np.concatenate(ratios)
        assert abs(ratios.mean() - 1.0) < 0.02 and ratios.std() < 0.03 and np.abs(ratios - 1).max() < 0.1


def test_treepm_converges_to_ewald(oracle_mod):
    # short-range tree (theta -> 0) plus PM against the Ewald sum: the error
    # comes from the PM at the split scale and the cutoff, so it must shrink as
    # the split is resolved by more mesh cells and the cutoff widens
    n = 8
    pos, mass = W.zeldovich(n, 9, rms_frac=0.3)
    tg = np.arange(0, n ** 3, 3)
    ae, pe = oracle_mod.ewald(pos, mass, tg, 1.0, 1.0)
    med = []
    for ng, asmth, rcut in ((32, 1.25, 4.5), (64, 2.5, 7.0), (128, 5.0, 7.0)):
        a, p, nint = oracle_mod.treepm(pos, mass, tg, 1.0, ng, asmth, rcut, 1.0, 1e-4, theta=1e-6, bucket=4)
        med.append(np.median(rel_err(a, ae)))
        last = (a, p)
    assert med[0] > med[1] > med[2] and med[2] < 1e-3 and med[0] < 3e-2
    a, p = last
    assert np.percentile(rel_err(a, ae), 99) < 5e-3
    # periodic potential: compare up to a constant
    assert np.abs((p - p.mean()) - (pe - pe.mean())).max() < 1e-2 * np.abs(pe - pe.mean()).max()


def test_treepm_pair_small_separation_is_newtonian(oracle_mod):
    ng = 32
    rs = 1.25 / ng
    r = 0.2 * rs
    pos = np.array([[0.3, 0.4, 0.5], [0.3 + 0.6 * r, 0.4 + 0.8 * r, 0.5]])
    mass = np.array([1.0, 1.0], np.float32)
    ae, _ = oracle_mod.ewald(pos, mass, np.array([0]), 1.0, 1.0)
    a, _, _ = oracle_mod.treepm(pos, mass, np.array([0]), 1.0, ng, 1.25, 4.5, 1.0, 1e-6, theta=1e-6, bucket=1)
    assert rel_err(a, ae)[0] < 1e-4
