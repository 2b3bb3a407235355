"""Time stepping on the GPU (tpm_drift, tpm_active_set, tpm_kick and the
Integrator that sequences them with the force path) against the FP64 oracle
of oracle/leapfrog.py.

* With the same accelerations fed to both sides, every FP64 position and
  velocity, every bin and the due sets agree bit for bit: both sides round
  the same operations in the same order.
* A whole cycle of the hierarchy with forces from the tree walk (FP32 on the
  GPU, FP64 in the oracle): a force differs by |da|/|a| ~ 1e-6 (p99 <= 2e-5,
  the walk parity tolerance), so after the cycle a velocity differs by about
  that times |a| T and a position by that times |a| T^2 (T the cycle
  length).  A bin can differ where the criterion falls within that margin of
  a bin boundary; such particles (and only those) may differ by more.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpm():
    import paper_1909_04667_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(tpm):
    c = tpm.Context(0)
    yield c
    c.close()


def state(n, seed, periodic):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 1, (n, 3)) if periodic else rng.standard_normal((n, 3))
    vel = 0.5 * rng.standard_normal((n, 3))
    # accelerations over four decades, so the criterion spreads over all bins
    mag = 10.0 ** rng.uniform(-2, 2, n)
    d = rng.standard_normal((n, 3))
    acc = (d / np.linalg.norm(d, axis=1)[:, None] * mag[:, None]).astype(np.float32)
    return pos, vel, acc


@pytest.mark.parametrize("periodic", [False, True])
def test_kernels_bit_exact_with_oracle(tpm, ctx, periodic, oracle_mod):
    import torch

    from oracle import leapfrog as LF

    n, nb = 6001, 5
    sp = tpm.StepParams(dt_tick=1e-3, nbins=nb, c_grav=0.02, eps=0.004)
    pos, vel, table = state(n, 11 + periodic, periodic)
    scale = lambda t: np.float32(1.0 + 0.5 * math.sin(0.7 * t))  # forces change from tick to tick

    def forces(x, ids, amag_old):
        return (table[ids] * scale(ref.tick)).astype(np.float64)

    ref = None
    ref = LF.Hierarchy.__new__(LF.Hierarchy)  # bound before __init__ calls forces()
    ref.tick = 0
    LF.Hierarchy.__init__(ref, pos, vel, forces, sp.dt_tick, nb, sp.c_grav, sp.eps, box=1.0 if periodic else 0.0)

    dev = torch.device("cuda", 0)
    x = torch.from_numpy(pos).to(dev)
    v = torch.from_numpy(vel).to(dev)
    bins = torch.zeros(n, dtype=torch.int8, device=dev)
    amag = torch.zeros(n, dtype=torch.float32, device=dev)
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    a_old = torch.empty(n, dtype=torch.float32, device=dev)
    tab = torch.from_numpy(table).to(dev)
    tpm.kick(ctx, ids, n, tab * float(scale(0)), v, bins, amag, 0, sp, first=True)
    for t in range(1, 2 * (1 << (nb - 1)) + 1):
        tpm.drift(ctx, x, v, sp.dt_tick, periodic, 1.0)
        prev_amag = amag.clone()
        k = tpm.active_set(ctx, bins, t, nb, ids, amag=amag, a_old=a_old)
        due = ref.advance()
        assert k == len(due)
        got = ids[:k].cpu().numpy()
        np.testing.assert_array_equal(got, due)
        np.testing.assert_array_equal(a_old[:k].cpu().numpy(), prev_amag.cpu().numpy()[got])
        if k:
            acc = tab[ids[:k].long()] * float(scale(t))
            tpm.kick(ctx, ids, k, acc.contiguous(), v, bins, amag, t, sp)
        np.testing.assert_array_equal(x.cpu().numpy(), ref.x)
        np.testing.assert_array_equal(v.cpu().numpy(), ref.v)
        np.testing.assert_array_equal(bins.cpu().numpy(), ref.bins)
        np.testing.assert_array_equal(amag.cpu().numpy(), ref.amag.astype(np.float32))
    assert len(set(ref.bins.tolist())) == nb  # every bin was used


def test_integrator_cycle_matches_oracle(tpm, ctx, oracle_mod):
    from oracle import leapfrog as LF

    from paper_1909_04667_gb300.integrate import Integrator

    n, nb, h = 4096, 4, 0.01
    pos, mass = W.plummer(n, 1001)
    rng = np.random.default_rng(5)
    vel = 0.3 * rng.standard_normal((n, 3))
    shift = tuple(W.root_shift(9))
    sp = tpm.StepParams(dt_tick=0.004, nbins=nb, c_grav=0.025, eps=h / 2.8)
    bp = tpm.BuildParams(G=1.0, h=h, shift=shift, leaf_bucket=8)
    fp_first = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5)
    fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.0025)
    gpu = Integrator(ctx, pos, vel, mass, bp, sp, fp_first, fp)

    def forces(x, ids, amag_old):
        tree = oracle_mod.Tree(x, mass, bucket=8, shift=shift)
        if amag_old is None:
            acc, _, _ = tree.walk(ids, 1.0, h, theta=0.5)
        else:
            acc, _, _ = tree.walk(ids, 1.0, h, crit="rel", alpha=0.0025, a_old=amag_old)
        return acc

    ref = LF.Hierarchy(pos, vel, forces, sp.dt_tick, nb, sp.c_grav, sp.eps)
    assert np.mean(gpu.bins.cpu().numpy() != ref.bins) <= 0.005  # first bins: the same but for margin cases
    forces_gpu = gpu.run_cycle()
    for _ in range(1 << (nb - 1)):
        ref.advance()
    assert len(set(ref.bins.tolist())) >= 3
    bins = gpu.bins.cpu().numpy()
    same = bins == ref.bins
    assert np.mean(~same) <= 0.005
    T = sp.dt_tick * (1 << (nb - 1))
    a = np.maximum(ref.amag, 1e-12)
    ev = np.linalg.norm(gpu.vel.cpu().numpy() - ref.v, axis=1) / (a * T)
    ex = np.linalg.norm(gpu.pos.cpu().numpy() - ref.x, axis=1) / (a * T * T)
    msg = "v p99 %.3g max %.3g, x p99 %.3g max %.3g, bins differ %d" % (
        np.percentile(ev[same], 99), ev[same].max(), np.percentile(ex[same], 99), ex[same].max(), np.sum(~same))
    assert np.percentile(ev[same], 99) <= 5e-5 and np.percentile(ex[same], 99) <= 5e-5, msg
    assert forces_gpu == ref.n_forces - n


def test_time_stepping_rejects_bad_arguments(tpm, ctx):
    import torch

    dev = torch.device("cuda", 0)
    x = torch.zeros((10, 3), dtype=torch.float64, device=dev)
    with pytest.raises(tpm.TreePMError, match="device memory"):
        tpm.drift(ctx, x, np.zeros((10, 3)), 0.1)
    bins = torch.zeros(10, dtype=torch.int8, device=dev)
    ids = torch.zeros(10, dtype=torch.int32, device=dev)
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):
        tpm.active_set(ctx, bins, 0, 40, ids)
    amag = torch.zeros(10, dtype=torch.float32, device=dev)
    acc = torch.zeros((10, 3), dtype=torch.float32, device=dev)
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):
        tpm.kick(ctx, ids, 10, acc, x, bins, amag, 0, tpm.StepParams(dt_tick=-1.0))
