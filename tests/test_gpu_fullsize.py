"""Full-size checks in the launch configuration bench.py times: the GPU
computes every particle; the oracle recomputes a seeded sample one by one.

Hernquist N = 2^20: geometric first force (theta = 0.5), then the relative
criterion (alpha = 0.0025) against the previous |a|, at the headline's leaf
bucket (bench.HERNQUIST).  The
periodic 128^3 Zel'dovich box: PM 256^3, a_s = 1.25, a_cut = 4.5.
"""
import numpy as np
import pytest

import bench
import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.fixture(scope="module")
def tpm():
    import paper_1909_04667_gb300 as m

    return m


def test_hernquist_full_size(oracle_mod, tpm):
    import torch

    dev = torch.device("cuda", 0)
    cfg = bench.HERNQUIST
    pos, mass = bench.hernquist_inputs()
    n = len(pos)
    shift = bench.root_shift(0, 2)
    ctx = tpm.Context(0)
    s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                       tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=shift, leaf_bucket=cfg["bucket"]))
    a_bh, _, n_bh = s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"]))
    a_old = torch.linalg.vector_norm(a_bh, dim=1).contiguous()
    a_rel, _, n_rel = s.compute_forces(a_old=a_old, fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"]))
    a_bh, n_bh = a_bh.cpu().numpy().astype(np.float64), n_bh.cpu().numpy()
    a_rel, n_rel = a_rel.cpu().numpy().astype(np.float64), n_rel.cpu().numpy()
    s.release()
    ctx.close()
    tg = W.random_targets(n, 1024, 99)
    tree = oracle_mod.Tree(pos, mass, bucket=cfg["bucket"], shift=shift)
    o_bh, _, on_bh = tree.walk(tg, cfg["G"], cfg["h"], theta=cfg["theta"])
    # the geometric pass: same decisions, FP32 vs FP64 arithmetic
    e = rel(a_bh[tg], o_bh)
    same = n_bh[tg] == on_bh
    assert same.mean() >= 0.995 and np.percentile(e[same], 99) < 2e-5
    # the relative pass, |a_old| from each side's own first pass
    aold_o = np.linalg.norm(o_bh, axis=1).astype(np.float32)
    o_rel, _, on_rel = tree.walk(tg, cfg["G"], cfg["h"], crit="rel", alpha=cfg["alpha"], a_old=aold_o)
    e = rel(a_rel[tg], o_rel)
    same = n_rel[tg] == on_rel
    assert same.mean() >= 0.99 and np.percentile(e[same], 99) < 2e-5
    # accuracy against the exact softened direct sum: the GPU matches the
    # method's own floor (the oracle walk's error)
    ad, _ = oracle_mod.direct(pos, mass, tg, cfg["G"], cfg["h"])
    gpu_p99 = np.percentile(rel(a_rel[tg], ad), 99)
    floor_p99 = np.percentile(rel(o_rel, ad), 99)
    assert gpu_p99 <= 5e-3 and gpu_p99 <= 1.05 * floor_p99 + 1e-5


@pytest.mark.parametrize("grad", ["fd4", "ik"])
def test_zeldovich_full_size(oracle_mod, tpm, grad):
    import torch

    dev = torch.device("cuda", 0)
    cfg = bench.ZELDOVICH
    pos, mass = bench.zeldovich_inputs()
    n = len(pos)
    h = bench.zeldovich_h()
    shift = bench.root_shift(0, 3)
    common = dict(treepm=True, pm_n=cfg["pm_n"], asmth=cfg["asmth"], rcut=cfg["rcut"],
                  pm_grad=tpm.GRAD_IK if grad == "ik" else tpm.GRAD_FD4)
    fp_bh = tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"], **common)
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"], **common)
    ctx = tpm.Context(0)
    s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                       tpm.BuildParams(G=cfg["G"], h=h, periodic=True, box=1.0, shift=shift,
                                       leaf_bucket=cfg["bucket"]))
    s.pm_long_range(fp_bh)
    a_bh, _, _ = s.compute_forces(fp=fp_bh)
    a_old = torch.linalg.vector_norm(a_bh, dim=1).contiguous()
    a_rel, _, n_rel = s.compute_forces(a_old=a_old, fp=fp_rel)
    a_rel, n_rel = a_rel.cpu().numpy().astype(np.float64), n_rel.cpu().numpy()
    xtree = s.tree_export()["xtree"]
    s.release()
    ctx.close()
    tg = W.random_targets(n, 256, 98)
    rs = cfg["asmth"] / cfg["pm_n"]
    tree = oracle_mod.Tree(pos, mass, bucket=cfg["bucket"], periodic=True, box=1.0, shift=shift)
    phi = oracle_mod.pm_potential(xtree, mass, 1.0, cfg["pm_n"], rs)
    a_l, _ = oracle_mod.pm_interpolate(phi, xtree[tg], 1.0, grad=grad)
    o_bh, _, _ = tree.walk(tg, cfg["G"], h, theta=cfg["theta"], treepm=True, rs=rs, rcut=cfg["rcut"] * rs)
    aold_o = np.linalg.norm(o_bh + a_l, axis=1).astype(np.float32)
    o_s, _, on_rel = tree.walk(tg, cfg["G"], h, crit="rel", alpha=cfg["alpha"], a_old=aold_o, treepm=True, rs=rs,
                               rcut=cfg["rcut"] * rs)
    o_rel = o_s + a_l
    e = rel(a_rel[tg], o_rel)
    same = n_rel[tg] == on_rel
    assert same.mean() >= 0.98 and np.percentile(e[same], 99) < 1e-4
    # error against the exact periodic (Ewald) force: GPU at the method's floor
    ae, _ = oracle_mod.ewald(pos, mass, tg, cfg["G"], 1.0)
    gpu = rel(a_rel[tg], ae)
    floor = rel(o_rel, ae)
    print("periodic TreePM (%s) vs Ewald: GPU p50 %.3g p99 %.3g; oracle p50 %.3g p99 %.3g" % (
        grad, np.median(gpu), np.percentile(gpu, 99), np.median(floor), np.percentile(floor, 99)))
    assert np.percentile(gpu, 99) <= 1.05 * np.percentile(floor, 99) + 1e-4


@pytest.mark.parametrize("pm_n,asmth,bound", [(128, 1.25, None), (64, 2.5, 5e-3)])
def test_hernquist_isolated_treepm_full_size(oracle_mod, tpm, pm_n, asmth, bound):
    # TreePM with open boundaries (zero-padded mesh) on the Hernquist 2^20 set:
    # the relative pass must sit at the oracle TreePM's own floor against the
    # FP64 direct sum.  That floor is set by the mesh at the split scale (CIC
    # and the 4-point difference leave ~1% pair-force errors at r ~ 2-4 r_s):
    # p99 ~1.4e-2 with r_s = 1.25 cells, within the method's 5e-3 once the
    # split is resolved (r_s = 2.5 cells)
    import torch

    dev = torch.device("cuda", 0)
    cfg = bench.HERNQUIST
    pos, mass = bench.hernquist_inputs()
    n = len(pos)
    shift = bench.root_shift(0, 2)
    common = dict(treepm=True, pm_n=pm_n, asmth=asmth, rcut=4.5)
    ctx = tpm.Context(0)
    s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                       tpm.BuildParams(G=cfg["G"], h=cfg["h"], shift=shift, leaf_bucket=cfg["bucket"]))
    s.pm_long_range(tpm.ForceParams(**common))
    a_bh, _, _ = s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"], **common))
    a_old = torch.linalg.vector_norm(a_bh, dim=1).contiguous()
    a_rel, _, _ = s.compute_forces(a_old=a_old, fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"],
                                                                   **common))
    a_rel = a_rel.cpu().numpy().astype(np.float64)
    s.release()
    ctx.close()
    tg = W.random_targets(n, 1024, 98)
    ad, _ = oracle_mod.direct(pos, mass, tg, cfg["G"], cfg["h"])
    o_bh, _, _ = oracle_mod.treepm_isolated(pos, mass, tg, pm_n, asmth, 4.5, cfg["G"], cfg["h"], theta=cfg["theta"],
                                            shift=shift)
    o_rel, _, _ = oracle_mod.treepm_isolated(pos, mass, tg, pm_n, asmth, 4.5, cfg["G"], cfg["h"], crit="rel",
                                             alpha=cfg["alpha"], a_old=np.linalg.norm(o_bh, axis=1), shift=shift)
    gpu_p99 = np.percentile(rel(a_rel[tg], ad), 99)
    floor_p99 = np.percentile(rel(o_rel, ad), 99)
    assert gpu_p99 <= 1.05 * floor_p99 + 1e-5, (gpu_p99, floor_p99)
    if bound:
        assert gpu_p99 <= bound, gpu_p99


def test_zeldovich_ewald_tree_full_size(oracle_mod, tpm):
    # the 128^3 box as a pure tree with the Ewald correction (no mesh): the
    # geometric first pass, then the relative criterion; parity with the
    # oracle walk on sampled particles and the error against the exact
    # Ewald sum at the oracle's floor
    import torch

    dev = torch.device("cuda", 0)
    cfg = bench.ZELDOVICH
    pos, mass = bench.zeldovich_inputs()
    n = len(pos)
    h = bench.zeldovich_h()
    shift = bench.root_shift(0, 3)
    ctx = tpm.Context(0)
    s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                       tpm.BuildParams(G=cfg["G"], h=h, periodic=True, box=1.0, shift=shift, leaf_bucket=cfg["bucket"]))
    a_bh, _, _ = s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=cfg["theta"]))
    a_old = torch.linalg.vector_norm(a_bh, dim=1).contiguous()
    # the sampled particles take the oracle's |a_old| on both sides: each has
    # thousands of relative decisions in this box of cancelling forces, so an
    # inherited |a_old| difference would flip some of them
    tg = W.random_targets(n, 512, 97)
    tree = oracle_mod.Tree(pos, mass, bucket=cfg["bucket"], periodic=True, box=1.0, shift=shift)
    o_bh, _, _ = tree.walk(tg, cfg["G"], h, theta=cfg["theta"], ewald=True)
    aold_o = np.linalg.norm(o_bh, axis=1).astype(np.float32)
    a_old[torch.from_numpy(tg.astype(np.int64)).to(dev)] = torch.from_numpy(aold_o).to(dev)
    a_rel, _, n_rel = s.compute_forces(a_old=a_old, fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=cfg["alpha"]))
    a_rel, n_rel = a_rel.cpu().numpy().astype(np.float64), n_rel.cpu().numpy()
    s.release()
    ctx.close()
    o_rel, _, on_rel = tree.walk(tg, cfg["G"], h, crit="rel", alpha=cfg["alpha"], a_old=aold_o, ewald=True)
    same = n_rel[tg] == on_rel
    assert same.mean() >= 0.995
    # ~10^4 terms that nearly cancel (a linear box): the running sum reaches
    # ~4 pi G rho L/2 ~ 6 while a force is ~0.03; with compensated sums the
    # rounding stays at the FP32 tier of the rms force
    scale = np.sqrt(np.mean(np.sum(o_rel * o_rel, axis=1)))
    e = np.linalg.norm(a_rel[tg] - o_rel, axis=1) / scale
    e_rel = rel(a_rel[tg], o_rel)
    print("periodic Ewald tree vs oracle walk: same counts %.4f, p99 %.3g of the rms force, p99 %.3g relative" % (
        same.mean(), np.percentile(e[same], 99), np.percentile(e_rel[same], 99)))
    assert np.percentile(e[same], 99) < 2e-5 and e[same].max() < 1e-4, (np.percentile(e[same], 99), e.max())
    ae, _ = oracle_mod.ewald(pos, mass, tg, cfg["G"], 1.0)
    gpu, floor = rel(a_rel[tg], ae), rel(o_rel, ae)
    print("periodic Ewald tree vs Ewald: GPU p50 %.3g p99 %.3g; oracle p50 %.3g p99 %.3g" % (
        np.median(gpu), np.percentile(gpu, 99), np.median(floor), np.percentile(floor, 99)))
    assert np.percentile(gpu, 99) <= 1.05 * np.percentile(floor, 99) + 1e-4
