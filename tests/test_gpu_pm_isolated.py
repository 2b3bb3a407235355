"""TreePM with open boundaries on the GPU (zero-padded mesh, isolated Green's
function) against the FP64 oracle of oracle/__init__.py.

Tolerances as for the periodic mesh: the FP32 mesh potential within 1e-5 of
its maximum (FP32 transforms of a smooth field), forces p99 1e-4 and max 1e-3
where the interaction counts agree (the FP32 walk plus the FP32 mesh); at full
size the total force must meet the method's accuracy against the FP64 direct
sum (p99 <= 5e-3 of |a|)."""
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


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.device("cuda", 0))


@pytest.mark.parametrize("crit", ["bh", "rel"])
def test_isolated_treepm_matches_oracle(oracle_mod, tpm, ctx, crit):
    ng, h = 32, 0.01
    pos, mass = W.plummer(20000, 1001)
    n = len(pos)
    shift = tuple(W.root_shift(21))
    bp = tpm.BuildParams(G=1.0, h=h, shift=shift, leaf_bucket=8)
    tg = np.arange(0, n, 5).astype(np.uint32)
    rng = np.random.default_rng(1)
    a_old = (10.0 ** rng.uniform(-1, 0.5, len(tg))).astype(np.float32)
    if crit == "bh":
        fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5, treepm=True, pm_n=ng, asmth=1.25, rcut=4.5)
    else:
        fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.0025, treepm=True, pm_n=ng, asmth=1.25, rcut=4.5)
    s = ctx.build_tree(dev(pos), dev(mass), bp)
    s.pm_long_range(fp)
    phi_gpu = s.pm_export(2 * ng).astype(np.float64)
    acc, pot, nint = s.compute_forces(active_ids=dev(tg), a_old=dev(a_old) if crit == "rel" else None, fp=fp)
    s.release()
    corner, side = oracle_mod.pm_region_isolated(pos)
    rs = 1.25 * side / ng
    phi_o = oracle_mod.pm_potential_isolated(pos, mass, corner, side, ng, rs)
    phys = (slice(0, ng + 1),) * 3
    assert np.abs(phi_gpu[phys] - phi_o[phys]).max() < 1e-5 * np.abs(phi_o[phys]).max()
    kw = dict(theta=0.5) if crit == "bh" else dict(crit="rel", alpha=0.0025, a_old=a_old)
    a_ref, p_ref, n_ref = oracle_mod.treepm_isolated(pos, mass, tg, ng, 1.25, 4.5, 1.0, h, shift=shift, **kw)
    a, nint = acc.cpu().numpy().astype(np.float64), nint.cpu().numpy()
    same = nint == n_ref
    assert np.mean(~same) <= 0.005
    e = rel(a, a_ref)
    assert np.percentile(e[same], 99) <= 1e-4 and e[same].max() <= 1e-3, (np.percentile(e[same], 99), e.max())
    p = pot.cpu().numpy().astype(np.float64)
    assert np.percentile(np.abs(p - p_ref)[same] / np.abs(p_ref[same]), 99) <= 1e-4


def test_isolated_treepm_rejects_oversized_mesh(tpm, ctx):
    pos, mass = W.plummer(1000, 2)
    s = ctx.build_tree(dev(pos), dev(mass), tpm.BuildParams())
    with pytest.raises(tpm.TreePMError, match="pm_n"):
        s.pm_long_range(tpm.ForceParams(treepm=True, pm_n=1024))
    with pytest.raises(tpm.TreePMError, match="long-range mesh"):
        s.compute_forces(fp=tpm.ForceParams(treepm=True, pm_n=64))
    s.release()
