"""The periodic tree with the Ewald correction on the GPU (treepm = 0 on a
periodic system) against the FP64 oracle walk with the same correction.

Same decisions as the oracle walk; the pair terms and the trilinear table
interpolation run in FP32 (table values rounded to FP32 from the FP64 Ewald
sums).  A linear box's total forces are small sums of thousands of large,
nearly cancelling terms; each interaction's pair term and correction are
added first and then into compensated sums, so forces agree at the FP32 tier
(p99 1e-5, max 5e-5) where the interaction counts agree.  Potentials are
compared up to a constant (periodic potentials)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpm():
    import paper_1909_04667_gb300 as m

    return m


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.device("cuda", 0))


@pytest.mark.parametrize("crit", ["bh", "rel"])
def test_ewald_tree_matches_oracle(oracle_mod, tpm, crit):
    ng = 24
    pos, mass = W.zeldovich(ng, 1003)
    n = len(pos)
    h = (1.0 / ng) / 40
    shift = tuple(W.root_shift(13))
    tg = np.arange(0, n, 3).astype(np.uint32)
    ctx = tpm.Context(0)
    s = ctx.build_tree(dev(pos), dev(mass), tpm.BuildParams(G=1.0, h=h, periodic=True, box=1.0, shift=shift,
                                                            leaf_bucket=8))
    tree = oracle_mod.Tree(pos, mass, bucket=8, periodic=True, box=1.0, shift=shift)
    if crit == "bh":
        fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5)
        acc, pot, nint = s.compute_forces(active_ids=dev(tg), fp=fp)
        a_o, p_o, n_o = tree.walk(tg, 1.0, h, theta=0.5, ewald=True)
    else:
        a_bh, _, _ = tree.walk(tg, 1.0, h, theta=0.5, ewald=True)
        a_old = np.linalg.norm(a_bh, axis=1).astype(np.float32)
        fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.005)
        acc, pot, nint = s.compute_forces(active_ids=dev(tg), a_old=dev(a_old), fp=fp)
        a_o, p_o, n_o = tree.walk(tg, 1.0, h, crit="rel", alpha=0.005, a_old=a_old, ewald=True)
    s.sync_status()
    s.release()
    ctx.close()
    a, nint, p = acc.cpu().numpy().astype(np.float64), nint.cpu().numpy(), pot.cpu().numpy().astype(np.float64)
    same = nint == n_o
    assert np.mean(~same) <= 0.005
    e = rel(a, a_o)
    print("Ewald tree (%s) vs oracle: p99 %.3g max %.3g, counts differ %d" % (
        crit, np.percentile(e[same], 99), e[same].max(), (~same).sum()))
    assert np.percentile(e[same], 99) <= 1e-5 and e[same].max() <= 5e-5, (np.percentile(e[same], 99), e.max())
    dp = p - p_o
    assert np.percentile(np.abs(dp - dp.mean())[same], 99) <= 1e-4 * np.abs(p_o).mean()


def test_ewald_noalloc_needs_the_table(tpm):
    import torch

    pos, mass = W.zeldovich(8, 4)
    ctx = tpm.Context(0)
    s = ctx.build_tree(dev(pos), dev(mass), tpm.BuildParams(G=1.0, h=1e-3, periodic=True, box=1.0))
    ids = dev(np.arange(len(pos), dtype=np.int32))
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5)
    out = torch.empty((len(pos), 3), device=torch.device("cuda", 0))
    with pytest.raises(tpm.TreePMError, match="Ewald"):
        s.compute_forces_noalloc(ids, out, fp=fp)
    ref, _, _ = s.compute_forces(active_ids=ids, fp=fp)  # builds the table
    s.compute_forces_noalloc(ids, out, fp=fp)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=2e-5, atol=1e-7 * float(ref.abs().max()))
    s.release()
    ctx.close()
