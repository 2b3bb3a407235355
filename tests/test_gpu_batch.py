"""Batched evaluation (tpm_compute_forces_batch) against per-request calls.

Each request of a batch must get what tpm_compute_forces gives for that
request alone: the same per-particle decisions (interaction counts equal up to
FP32 margin flips, at most 0.5%) and forces within the FP32 tolerance of the
parity tests -- only the grouping of particles into warps, hence the order of
FP32 summation, differs.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

P99_TOL = 2e-5
MAX_TOL = 2e-4


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def oracle_check(acc, nint, a_o, n_o, p99=P99_TOL, mx=MAX_TOL):
    """The batched walk against the oracle's per-particle walk: interaction
    counts equal except for FP32 margin flips (0.5%, or one particle in a
    small request), forces within the FP32 tolerance where counts agree and
    within the method's 5e-3 where a decision flipped."""
    same = nint == n_o
    assert np.mean(~same) <= 0.005 or (~same).sum() <= 1, "%d counts differ" % (~same).sum()
    e = rel(acc.astype(np.float64), a_o)
    if same.any():
        assert np.percentile(e[same], 99) <= p99 and e[same].max() <= mx, (np.percentile(e[same], 99), e[same].max())
    if (~same).any():
        assert e[~same].max() <= 5e-3


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    ctx = tpm.Context(0)
    p1, m1 = W.plummer(20000, 5)
    p2, m2 = W.hernquist(60000, 6)
    s1 = ctx.build_tree(torch.from_numpy(p1).to(dev), torch.from_numpy(m1).to(dev),
                        tpm.BuildParams(G=1.0, h=0.01, shift=tuple(W.root_shift(5)), leaf_bucket=8))
    s2 = ctx.build_tree(torch.from_numpy(p2).to(dev), torch.from_numpy(m2).to(dev),
                        tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(6)), leaf_bucket=8))
    # |a_old| from a geometric pass
    aold = {}
    for s in (s1, s2):
        a, _, _ = s.compute_forces(fp=tpm.ForceParams(theta=0.5))
        aold[s.handle] = torch.linalg.vector_norm(a, dim=1).contiguous()
    rng = np.random.default_rng(3)
    reqs = []
    for r in range(9):  # uneven sizes, both systems, both criteria, unsorted ids
        s = (s1, s2)[r % 2]
        size = int(rng.integers(1, 5000)) if r != 4 else 1
        ids = rng.choice(s.n, size, replace=False).astype(np.int32)
        fp = tpm.ForceParams(theta=0.6) if r % 3 else tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.002)
        reqs.append((s, ids, fp))
    yield tpm, torch, dev, ctx, reqs, aold
    ctx.close()


def batch_inputs(torch, dev, reqs, aold):
    ids = np.concatenate([r[1] for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r[1]) for r in reqs])])
    a_old = torch.cat([aold[s.handle][torch.from_numpy(i.astype(np.int64)).to(dev)] for s, i, _ in reqs])
    return torch.from_numpy(ids).to(dev), off, a_old


def reference(tpm, torch, dev, reqs, aold):
    out = []
    for s, ids, fp in reqs:
        ti = torch.from_numpy(ids).to(dev)
        a, p, n = s.compute_forces(active_ids=ti, a_old=aold[s.handle][ti.long()].contiguous(), fp=fp)
        out.append((a.cpu().numpy(), p.cpu().numpy(), n.cpu().numpy()))
    return out


def check(ref, acc, pot, nint, off):
    for r, (a, p, n) in enumerate(ref):
        sl = slice(off[r], off[r + 1])
        same = nint[sl] == n
        assert np.mean(~same) <= 0.005 or (~same).sum() <= 1
        e = rel(acc[sl].astype(np.float64), a.astype(np.float64))
        assert np.percentile(e[same], 99) <= P99_TOL and e[same].max() <= MAX_TOL
        np.testing.assert_allclose(pot[sl][same], p[same], rtol=P99_TOL)


@pytest.mark.parametrize("group", [64, 32, 16, 8])
def test_batch_matches_per_request_calls(env, group):
    tpm, torch, dev, ctx, reqs, aold = env
    ids, off, a_old = batch_inputs(torch, dev, reqs, aold)
    plan = ctx.create_plan(int(off[-1]) + 100, 16)
    plan.group_size = group
    acc = torch.empty((len(ids), 3), device=dev)
    pot = torch.empty(len(ids), device=dev)
    nint = torch.empty(len(ids), dtype=torch.int32, device=dev)
    plan.compute_forces_batch([r[0] for r in reqs], off, [r[2] for r in reqs], ids, acc, a_old=a_old, pot=pot,
                              n_int=nint)
    plan.sync_status()
    check(reference(tpm, torch, dev, reqs, aold), acc.cpu().numpy(), pot.cpu().numpy(), nint.cpu().numpy(), off)
    plan.close()


def test_batch_with_empty_and_large_requests(env):
    """Empty requests between others, and one request spanning many key
    blocks (all 60000 particles of a tree): every id finds its own request,
    and each request gets what a plain call gives it (bit for bit at the
    plan's default group size and depth)."""
    tpm, torch, dev, ctx, reqs, aold = env
    s1, s2 = reqs[0][0], reqs[1][0]
    rng = np.random.default_rng(12)
    empty = np.zeros(0, np.int32)
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.002)
    mixed = [(s1, empty, fp_rel), (s2, rng.permutation(s2.n).astype(np.int32), fp_rel), (s1, empty, fp_rel),
             (s1, empty, fp_rel), (s1, rng.choice(s1.n, 700, replace=False).astype(np.int32), fp_rel),
             (s2, empty, fp_rel)]
    ids, off, a_old = batch_inputs(torch, dev, mixed, aold)
    plan = ctx.create_plan(int(off[-1]), 8)
    acc = torch.empty((len(ids), 3), device=dev)
    pot = torch.empty(len(ids), device=dev)
    nint = torch.empty(len(ids), dtype=torch.int32, device=dev)
    plan.compute_forces_batch([r[0] for r in mixed], off, [r[2] for r in mixed], ids, acc, a_old=a_old, pot=pot,
                              n_int=nint)
    plan.sync_status()
    acc, nint = acc.cpu().numpy(), nint.cpu().numpy()
    for r, (a, p, n) in enumerate(reference(tpm, torch, dev, mixed, aold)):
        sl = slice(off[r], off[r + 1])
        np.testing.assert_array_equal(acc[sl], a)
        np.testing.assert_array_equal(nint[sl], n)
    plan.close()


def test_batch_presorted_and_graph_replay(env):
    tpm, torch, dev, ctx, reqs, aold = env
    # ids in each tree's key order: the presorted flag skips the sort
    sorted_reqs = []
    for s, ids, fp in reqs:
        perm = s.tree_export()["perm"]
        rank = np.empty(s.n, np.int64)
        rank[perm] = np.arange(s.n)
        sorted_reqs.append((s, ids[np.argsort(rank[ids])], fp))
    ids, off, a_old = batch_inputs(torch, dev, sorted_reqs, aold)
    plan = ctx.create_plan(int(off[-1]), len(reqs))
    acc = torch.zeros((len(ids), 3), device=dev)
    nint = torch.zeros(len(ids), dtype=torch.int32, device=dev)
    args = ([r[0] for r in sorted_reqs], off, [r[2] for r in sorted_reqs], ids, acc)
    plan.compute_forces_batch(*args, a_old=a_old, n_int=nint, presorted=True)
    torch.cuda.synchronize()
    eager = (acc.cpu().numpy().copy(), nint.cpu().numpy().copy())
    ref = reference(tpm, torch, dev, sorted_reqs, aold)
    for r, (a, p, n) in enumerate(ref):
        sl = slice(off[r], off[r + 1])
        assert np.mean(eager[1][sl] != n) <= 0.005 or (eager[1][sl] != n).sum() <= 1
    # capture the batched call in a CUDA graph and replay it
    g = torch.cuda.CUDAGraph()
    acc.zero_()
    nint.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.compute_forces_batch(*args, a_old=a_old, n_int=nint, presorted=True)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        acc.zero_()
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(acc.cpu().numpy(), eager[0])
        np.testing.assert_array_equal(nint.cpu().numpy(), eager[1])
    plan.sync_status()
    plan.close()


def test_autotune_and_errors(env):
    tpm, torch, dev, ctx, reqs, aold = env
    ids, off, a_old = batch_inputs(torch, dev, reqs, aold)
    plan = ctx.create_plan(int(off[-1]), len(reqs))
    acc = torch.empty((len(ids), 3), device=dev)
    g, ms = plan.autotune([r[0] for r in reqs], off, [r[2] for r in reqs], ids, acc, a_old=a_old, reps=2)
    assert g in (8, 16, 32, 64) and plan.group_size == g and ms > 0
    assert plan.stack_depth in (128, 192, 256)
    # every stack depth makes the same decisions (interaction counts); the
    # order of the sums may differ where a shallower stack takes candidates one
    # at a time earlier
    ref = None
    for depth in (192, 128, 256):
        plan.stack_depth = depth
        a = torch.empty((len(ids), 3), device=dev)
        k = torch.empty(len(ids), dtype=torch.int32, device=dev)
        plan.compute_forces_batch([r[0] for r in reqs], off, [r[2] for r in reqs], ids, a, a_old=a_old, n_int=k)
        plan.sync_status()
        a, k = a.cpu().numpy().astype(np.float64), k.cpu().numpy()
        if ref is None:
            ref = (a, k)
            continue
        np.testing.assert_array_equal(k, ref[1])
        err = np.linalg.norm(a - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
        assert np.percentile(err, 99) < 1e-5 and err.max() < 1e-4
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):
        plan.stack_depth = 100
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):  # more requests than the plan holds
        plan.compute_forces_batch([reqs[0][0]] * (len(reqs) + 1), np.zeros(len(reqs) + 2, np.int64),
                                  tpm.ForceParams(), ids, acc)
    bad = ids.clone()
    bad[0] = 10 ** 9
    plan.compute_forces_batch([r[0] for r in reqs], off, [r[2] for r in reqs], bad, acc, a_old=a_old)
    with pytest.raises(tpm.TreePMError, match="out of range"):
        plan.sync_status()
    plan.close()


@pytest.fixture(scope="module")
def oracle_env(oracle_mod):
    """Three systems (a Plummer sphere, a Hernquist halo, two clusters with
    isolated particles between them) with their oracle trees, |a_old| from a
    geometric GPU pass, and uneven requests on all three."""
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    ctx = tpm.Context(0)
    specs = [(W.plummer(12000, 15), 0.01, 15), (W.hernquist(30000, 16), 0.005, 16),
             (W.clusters_with_outliers(4096, 78), 0.01, 78)]
    systems, trees, aold = [], [], {}
    for (pos, mass), h, seed in specs:
        shift = tuple(W.root_shift(seed))
        s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                           tpm.BuildParams(G=1.0, h=h, shift=shift, leaf_bucket=8))
        a, _, _ = s.compute_forces(fp=tpm.ForceParams(theta=0.5))
        aold[s.handle] = torch.linalg.vector_norm(a, dim=1).contiguous()
        systems.append((s, h))
        trees.append(oracle_mod.Tree(pos, mass, bucket=8, shift=shift))
    rng = np.random.default_rng(17)
    reqs = []
    for r in range(8):
        k = r % 3
        s, h = systems[k]
        size = s.n if (k == 2 and r < 3) else int(rng.integers(1, 3000))
        ids = rng.choice(s.n, size, replace=False).astype(np.int32)
        fp = tpm.ForceParams(theta=0.6) if r % 2 else tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.002)
        reqs.append((k, ids, fp))
    # the oracle walk of every request
    ref = []
    for k, ids, fp in reqs:
        s, h = systems[k]
        ao = aold[s.handle][torch.from_numpy(ids.astype(np.int64)).to(dev)].cpu().numpy()
        if fp.crit == tpm.CRIT_RELATIVE:
            a_o, _, n_o = trees[k].walk(ids, 1.0, h, crit="relative", alpha=fp.alpha, a_old=ao)
        else:
            a_o, _, n_o = trees[k].walk(ids, 1.0, h, theta=fp.theta)
        ref.append((a_o, n_o))
    yield tpm, torch, dev, ctx, systems, reqs, aold, ref
    ctx.close()


@pytest.mark.parametrize("group", [8, 16, 32, 64])
@pytest.mark.parametrize("depth", [128, 192, 256])
def test_batch_matches_oracle_walk(oracle_env, group, depth):
    """Every group size and stack depth of the persistent batched walk against
    the oracle's per-particle walk directly (not through the plain call)."""
    tpm, torch, dev, ctx, systems, reqs, aold, ref = oracle_env
    ids = np.concatenate([r[1] for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r[1]) for r in reqs])])
    a_old = torch.cat([aold[systems[k][0].handle][torch.from_numpy(i.astype(np.int64)).to(dev)]
                       for k, i, _ in reqs])
    plan = ctx.create_plan(int(off[-1]), len(reqs))
    plan.group_size = group
    plan.stack_depth = depth
    acc = torch.empty((len(ids), 3), device=dev)
    nint = torch.empty(len(ids), dtype=torch.int32, device=dev)
    plan.compute_forces_batch([systems[k][0] for k, _, _ in reqs], off, [r[2] for r in reqs],
                              torch.from_numpy(ids).to(dev), acc, a_old=a_old, n_int=nint)
    plan.sync_status()
    acc, nint = acc.cpu().numpy(), nint.cpu().numpy()
    for r, (a_o, n_o) in enumerate(ref):
        sl = slice(off[r], off[r + 1])
        try:
            oracle_check(acc[sl], nint[sl], a_o, n_o)
        except AssertionError as e:
            raise AssertionError("request %d (system %d, %d ids, crit %d): %s" % (r, reqs[r][0], len(reqs[r][1]),
                                                                                   reqs[r][2].crit, e))
    plan.close()
