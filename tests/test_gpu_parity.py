"""GPU-vs-oracle parity through the C ABI (libtreepm via its thin binding).

Tolerances:
* tree structure (keys, permutation, node table) and FP64 node masses and
  centres of mass: bit-exact -- both sides sum in the same fixed order with
  correctly rounded FP64 operations;
* forces: the GPU walk makes the same per-particle decisions as the oracle
  walk but evaluates pairs in FP32 with FP32 accumulation.  Each pair term
  carries a relative rounding error of a few 2^-24 ~ 1e-7 and a force sums
  10^2..10^4 terms that partly cancel, so |da|/|a| stays near 1e-6; we
  require p99 <= 2e-5 and max <= 2e-4 where the interaction sets agree.  An
  opening decision whose margin is below FP32 resolution can flip (a node
  accepted instead of opened): at most 0.5% of particles may differ in their
  interaction count, and those stay within the method's own error (5e-3).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

P99_TOL = 2e-5
MAX_TOL = 2e-4
ROOT_DIR = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))


@pytest.fixture(scope="module")
def tpm():
    import paper_1909_04667_gb300 as m

    return m


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    assert torch.cuda.is_available()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def ctx(tpm):
    c = tpm.Context(0)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def to_dev(x, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def compare_forces(acc, ref, nint, nref, p99=P99_TOL, mx=MAX_TOL, flip_frac=0.005):
    e = rel(acc, ref)
    same = nint == nref
    assert np.mean(~same) <= flip_frac, "interaction counts differ for %d particles" % np.sum(~same)
    assert np.percentile(e[same], 99) <= p99, "p99 %.3g" % np.percentile(e[same], 99)
    assert e[same].max() <= mx, "max %.3g" % e[same].max()
    if (~same).any():
        assert e[~same].max() <= 5e-3
    return e


def clustered(n, seed, dup=0):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (5, 3))
    pos = c[rng.integers(0, 5, n)] + 0.03 * rng.standard_normal((n, 3)) ** 3
    if dup:
        pos[:dup] = pos[0]
    return pos, np.full(n, 1.0 / n, np.float32)


def triplets(n_trip, seed):
    """Tight triplets: each needs a chain of cells down to the depth cap, so the
    tree has several times more nodes than particles and the build's first
    guess of the node space overflows."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (n_trip, 3))
    pos = np.repeat(c, 3, axis=0) + 1e-9 * rng.standard_normal((3 * n_trip, 3))
    return pos, np.full(3 * n_trip, 1.0 / (3 * n_trip), np.float32)


TREE_CASES = [
    ("plummer8192_B1", lambda: W.plummer(8192, 1001), 1, False),
    ("plummer8192_B8", lambda: W.plummer(8192, 1001), 8, False),
    ("hernquist20000_B8", lambda: W.hernquist(20000, 5), 8, False),
    ("clustered_dups_B4", lambda: clustered(3001, 7, dup=40), 4, False),
    ("ragged33_B1", lambda: W.plummer(33, 9), 1, False),
    ("single", lambda: W.plummer(1, 9), 1, False),
    ("pair", lambda: W.plummer(2, 9), 1, False),
    ("zeldovich32_B4", lambda: W.zeldovich(32, 3), 4, True),
    ("triplets_node_overflow_B2", lambda: triplets(1500, 11), 2, False),
]


@pytest.mark.parametrize("name,make,bucket,periodic", TREE_CASES, ids=[c[0] for c in TREE_CASES])
def test_tree_bit_exact(oracle_mod, tpm, ctx, torch_dev, name, make, bucket, periodic):
    pos, mass = make()
    shift = tuple(W.root_shift(31))
    bp = tpm.BuildParams(G=1.0, h=0.01, periodic=periodic, box=1.0, shift=shift, leaf_bucket=bucket)
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev), bp)
    ex = s.tree_export()
    s.release()
    ref = oracle_mod.Tree(pos, mass, bucket=bucket, periodic=periodic, box=1.0, shift=shift)
    rx = ref.export()
    assert ex["n_nodes"] == ref.nnodes
    np.testing.assert_array_equal(ex["x0"], ref.x0)
    assert ex["L0"] == ref.L0
    for k in ("key", "perm", "level", "prefix", "first", "count", "skip", "mass", "com", "xtree"):
        np.testing.assert_array_equal(ex[k], rx[k], err_msg=k)


def test_tree_host_inputs_same_as_device(tpm, ctx, torch_dev):
    pos, mass = W.hernquist(5000, 12)
    bp = tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(2)), leaf_bucket=8)
    a = ctx.build_tree(pos, mass, bp).tree_export()
    b = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev), bp).tree_export()
    for k in ("key", "perm", "prefix", "skip", "mass", "com"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("bucket", [1, 8, 16])
def test_walk_bh_plummer(oracle_mod, tpm, ctx, torch_dev, bucket):
    n = 8192
    pos, mass = W.plummer(n, 1001)
    shift = tuple(W.root_shift(1))
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=1.0, h=0.01, shift=shift, leaf_bucket=bucket))
    acc, pot, nint = s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.7))
    s.sync_status()
    acc, pot, nint = acc.cpu().numpy(), pot.cpu().numpy(), nint.cpu().numpy()
    s.release()
    tree = oracle_mod.Tree(pos, mass, bucket=bucket, shift=shift)
    a_o, p_o, n_o = tree.walk(np.arange(n), 1.0, 0.01, theta=0.7)
    compare_forces(acc.astype(np.float64), a_o, nint, n_o)
    np.testing.assert_allclose(pot, p_o, rtol=2e-5)


def test_depth_cap_with_far_outlier(oracle_mod, tpm, ctx, torch_dev):
    """One particle 10^7 scale lengths out makes the root cube 2^24 wide, so a
    level-21 cell (the depth cap) is 8 wide and holds a large share of the
    Plummer core: leaves of ~500 particles, far beyond the bucket of 8, and a
    walk that is nearly a direct sum.  The tree equals the oracle's bit for
    bit, every interaction count agrees, and every particle's force is within
    the FP32 tolerance -- including the 31 that share the outlier's
    32-particle chunk, whose walk is cut into runs with frames of their own
    (the chunk's frame would be the whole 2^24-wide root)."""
    n = 4096
    pos, mass = W.plummer(n, 77)
    pos[-1] = [1.0e7, 0.0, 0.0]
    shift = tuple(W.root_shift(77))
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=1.0, h=0.01, shift=shift, leaf_bucket=8))
    ex = s.tree_export()
    ref = oracle_mod.Tree(pos, mass, bucket=8, shift=shift)
    rx = ref.export()
    assert ex["n_nodes"] == ref.nnodes and ex["L0"] == ref.L0
    for k in ("key", "perm", "level", "prefix", "first", "count", "skip", "mass", "com"):
        np.testing.assert_array_equal(ex[k], rx[k], err_msg=k)
    assert ex["count"][ex["level"] == 21].max() > 400
    acc, pot, nint = s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5))
    s.sync_status()
    s.release()
    a_o, p_o, n_o = ref.walk(np.arange(n), 1.0, 0.01, theta=0.5)
    nint = nint.cpu().numpy()
    np.testing.assert_array_equal(nint, n_o)
    compare_forces(acc.cpu().numpy().astype(np.float64), a_o, nint, n_o)
    np.testing.assert_allclose(pot.cpu().numpy(), p_o, rtol=P99_TOL)


@pytest.mark.parametrize("walk", ["group", "lanes"])
def test_several_far_outliers_every_particle(oracle_mod, tpm, torch_dev, walk, tmp_path):
    """Two clusters and five isolated particles: one chunk runs from one
    cluster past four isolated particles into the other, another starts with
    the farthest particle.  Both criteria: every particle's force and count as
    the oracle walk's (the lane walk hands cut chunks to the group walk's runs
    too)."""
    import subprocess
    import sys

    out = tmp_path / "o.npz"
    code = OUTLIER_SCRIPT
    env = dict(__import__("os").environ, TPM_WALK=walk)
    r = subprocess.run([sys.executable, "-c", code, str(out)], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    res = np.load(out)
    pos, mass = W.clusters_with_outliers(4096, 78)
    shift = tuple(W.root_shift(78))
    ref = oracle_mod.Tree(pos, mass, bucket=8, shift=shift)
    a_o, p_o, n_o = ref.walk(np.arange(4096), 1.0, 0.01, theta=0.5)
    compare_forces(res["acc_bh"].astype(np.float64), a_o, res["n_bh"], n_o)
    a_old = np.linalg.norm(a_o, axis=1).astype(np.float32)
    a_r, p_r, n_r = ref.walk(np.arange(4096), 1.0, 0.01, crit="relative", alpha=0.001, a_old=a_old)
    compare_forces(res["acc_rel"].astype(np.float64), a_r, res["n_rel"], n_r)


OUTLIER_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, %r)
import workloads as W
import paper_1909_04667_gb300 as tpm
dev = torch.device("cuda", 0)
ctx = tpm.Context(0)
pos, mass = W.clusters_with_outliers(4096, 78)
s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                   tpm.BuildParams(G=1.0, h=0.01, shift=tuple(W.root_shift(78)), leaf_bucket=8))
a, p, n = s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5))
s.sync_status()
out = dict(acc_bh=a.cpu().numpy(), n_bh=n.cpu().numpy())
import oracle
ref = oracle.Tree(pos, mass, bucket=8, shift=tuple(W.root_shift(78)))
a_o, _, _ = ref.walk(np.arange(4096), 1.0, 0.01, theta=0.5)
a_old = torch.from_numpy(np.linalg.norm(a_o, axis=1).astype(np.float32)).to(dev)
a, p, n = s.compute_forces(a_old=a_old, fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.001))
s.sync_status()
out.update(acc_rel=a.cpu().numpy(), n_rel=n.cpu().numpy())
np.savez(sys.argv[1], **out)
""" % ROOT_DIR


def test_plain_fp32_arm_loses_precision_far_from_the_origin(oracle_mod, tpm, ctx, torch_dev):
    """The plain FP32 comparison arm (every pair vector a difference of
    absolute FP32 coordinates) against the mixed scheme, both against the
    oracle walk: at the origin both are at the FP32 rounding floor; 10^3
    scale lengths away the plain form's coordinates carry ~6e-5 of rounding,
    while the mixed scheme's offsets from each group's frame do not grow."""
    pos0, mass = W.plummer(8192, 1001)
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.7)
    fpp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.7, plain_fp32=True)
    p99 = {}
    for off in (0.0, 1.0e3):
        pos = pos0 + off
        shift = tuple(W.root_shift(4))
        s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                           tpm.BuildParams(G=1.0, h=0.01, shift=shift, leaf_bucket=8))
        a_m, _, n_m = s.compute_forces(fp=fp)
        a_p, _, _ = s.compute_forces(fp=fpp)
        s.sync_status()
        a_m, a_p, n_m = a_m.cpu().numpy().astype(np.float64), a_p.cpu().numpy().astype(np.float64), n_m.cpu().numpy()
        s.release()
        ref = oracle_mod.Tree(pos, mass, bucket=8, shift=shift)
        a_o, _, n_o = ref.walk(np.arange(len(pos)), 1.0, 0.01, theta=0.7)
        compare_forces(a_m, a_o, n_m, n_o)
        p99[off] = (np.percentile(rel(a_m, a_o), 99), np.percentile(rel(a_p, a_o), 99))
    assert p99[0.0][1] < 1e-4
    assert p99[1.0e3][1] > 1e-4 and p99[1.0e3][1] > 20 * p99[1.0e3][0], p99


@pytest.mark.parametrize("bucket", [8, 16])
def test_walk_relative_hernquist(oracle_mod, tpm, ctx, torch_dev, bucket):
    n = 1 << 16
    pos, mass = W.hernquist(n, 1002)
    shift = tuple(W.root_shift(2))
    tree = oracle_mod.Tree(pos, mass, bucket=bucket, shift=shift)
    a_bh, _, _ = tree.walk(np.arange(n), 1.0, 0.005, theta=0.5)
    a_old = np.linalg.norm(a_bh, axis=1).astype(np.float32)
    a_o, p_o, n_o = tree.walk(np.arange(n), 1.0, 0.005, crit="rel", alpha=0.0025, a_old=a_old)
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=1.0, h=0.005, shift=shift, leaf_bucket=bucket))
    acc, pot, nint = s.compute_forces(a_old=to_dev(a_old, torch_dev),
                                      fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.0025))
    s.release()
    compare_forces(acc.cpu().numpy().astype(np.float64), a_o, nint.cpu().numpy(), n_o)


def test_active_subset_in_caller_order(oracle_mod, tpm, ctx, torch_dev):
    n = 10000
    pos, mass = W.plummer(n, 44)
    shift = tuple(W.root_shift(4))
    rng = np.random.default_rng(1)
    ids = rng.choice(n, 1237, replace=False).astype(np.uint32)  # unsorted, ragged count
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=2.0, h=0.02, shift=shift, leaf_bucket=4))
    acc, pot, nint = s.compute_forces(active_ids=to_dev(ids, torch_dev), fp=tpm.ForceParams(theta=0.6))
    tree = oracle_mod.Tree(pos, mass, bucket=4, shift=shift)
    a_o, p_o, n_o = tree.walk(ids, 2.0, 0.02, theta=0.6)
    compare_forces(acc.cpu().numpy().astype(np.float64), a_o, nint.cpu().numpy(), n_o)
    # the same through host buffers (numpy in, numpy out)
    acc_h = np.zeros((len(ids), 3), np.float32)
    pot_h = np.zeros(len(ids), np.float32)
    nint_h = np.zeros(len(ids), np.uint32)
    s.compute_forces(active_ids=ids, fp=tpm.ForceParams(theta=0.6), acc=acc_h, pot=pot_h, n_int=nint_h)
    np.testing.assert_array_equal(acc_h, acc.cpu().numpy())
    np.testing.assert_array_equal(nint_h, nint.cpu().numpy().astype(np.uint32))
    s.release()


def test_page_locked_host_buffers(tpm, ctx, torch_dev):
    """The tree build reads page-locked host inputs in place (no staging
    copy), the force call stages page-locked and pageable host arguments
    alike; the tree and the forces equal those of device buffers bit for bit,
    for the build inputs, the active ids, a_old and every output."""
    import torch

    n = 20000
    pos, mass = W.hernquist(n, 21)
    bp = tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(21)), leaf_bucket=8)
    ids = np.random.default_rng(5).choice(n, 4321, replace=False).astype(np.uint32)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    s_dev = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev), bp)
    s_pin = ctx.build_tree(pin(pos), pin(mass), bp)
    s_pag = ctx.build_tree(pos, mass, bp)
    ex = [s.tree_export() for s in (s_dev, s_pin, s_pag)]
    for k in ("key", "perm", "level", "prefix", "first", "count", "skip", "mass", "com", "xtree"):
        np.testing.assert_array_equal(ex[1][k], ex[0][k], err_msg=k)
        np.testing.assert_array_equal(ex[2][k], ex[0][k], err_msg=k)
    a0, _, _ = s_dev.compute_forces(active_ids=to_dev(ids, torch_dev), fp=tpm.ForceParams(theta=0.5))
    a_old = np.linalg.norm(a0.cpu().numpy(), axis=1).astype(np.float32)
    fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.0025)
    acc_d, pot_d, nint_d = s_dev.compute_forces(active_ids=to_dev(ids, torch_dev), a_old=to_dev(a_old, torch_dev),
                                                fp=fp)
    ref = (acc_d.cpu().numpy(), pot_d.cpu().numpy(), nint_d.cpu().numpy().astype(np.uint32))
    acc_p = torch.zeros((len(ids), 3), dtype=torch.float32).pin_memory()
    pot_p = torch.zeros(len(ids), dtype=torch.float32).pin_memory()
    nint_p = torch.zeros(len(ids), dtype=torch.int32).pin_memory()
    s_pin.compute_forces(active_ids=pin(ids.view(np.int32)), a_old=pin(a_old), fp=fp, acc=acc_p, pot=pot_p,
                         n_int=nint_p)
    np.testing.assert_array_equal(acc_p.numpy(), ref[0])
    np.testing.assert_array_equal(pot_p.numpy(), ref[1])
    np.testing.assert_array_equal(nint_p.numpy().astype(np.uint32), ref[2])
    acc_h = np.zeros((len(ids), 3), np.float32)
    pot_h = np.zeros(len(ids), np.float32)
    nint_h = np.zeros(len(ids), np.uint32)
    s_pag.compute_forces(active_ids=ids, a_old=a_old, fp=fp, acc=acc_h, pot=pot_h, n_int=nint_h)
    np.testing.assert_array_equal(acc_h, ref[0])
    np.testing.assert_array_equal(pot_h, ref[1])
    np.testing.assert_array_equal(nint_h, ref[2])
    for s in (s_dev, s_pin, s_pag):
        s.release()


def test_walk_deterministic(tpm, ctx, torch_dev):
    pos, mass = W.hernquist(30000, 3)
    bp = tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(3)), leaf_bucket=8)
    outs = []
    for _ in range(2):
        s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev), bp)
        a, p, k = s.compute_forces(fp=tpm.ForceParams(theta=0.5))
        outs.append((a.cpu().numpy(), p.cpu().numpy(), k.cpu().numpy()))
        s.release()
    for x, y in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(x, y)
    # periodic TreePM: the short-range walk over one mesh gives the same bits
    # twice (the mesh itself is summed with float atomics, so it is formed once)
    pos, mass = W.zeldovich(32, 8)
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=1.0, h=(1 / 32) / 40, periodic=True, box=1.0, shift=tuple(W.root_shift(8)),
                                       leaf_bucket=8))
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5, treepm=True, pm_n=32, asmth=1.25, rcut=4.5)
    s.pm_long_range(fp)
    outs = [tuple(x.cpu().numpy() for x in s.compute_forces(fp=fp)) for _ in range(2)]
    s.release()
    for x, y in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(x, y)


def test_theta_zero_is_direct_sum(oracle_mod, tpm, ctx, torch_dev):
    n = 3000
    pos, mass = W.plummer(n, 8)
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=1.0, h=0.01, shift=(0.3, 0.6, 0.1), leaf_bucket=8))
    acc, pot, nint = s.compute_forces(fp=tpm.ForceParams(theta=1e-9))
    s.release()
    assert np.all(nint.cpu().numpy() == n - 1)
    ad, pd = oracle_mod.direct(pos, mass, np.arange(n), 1.0, 0.01)
    e = rel(acc.cpu().numpy().astype(np.float64), ad)
    assert np.percentile(e, 99) < P99_TOL and e.max() < MAX_TOL


def test_edge_cases(tpm, ctx, torch_dev):
    # one particle: no interaction at all
    s = ctx.build_tree(np.array([[0.5, 0.5, 0.5]]), np.array([1.0], np.float32), tpm.BuildParams())
    a, p, k = s.compute_forces(fp=tpm.ForceParams())
    assert np.all(a.cpu().numpy() == 0) and k.cpu().numpy()[0] == 0
    # an empty active set is a no-op
    s.compute_forces(active_ids=np.zeros(0, np.uint32), fp=tpm.ForceParams())
    s.release()
    # coincident particles share one level-21 leaf and feel no force from each other
    pos = np.zeros((6, 3))
    pos[3:] = [[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]
    s = ctx.build_tree(pos, np.full(6, 1 / 6, np.float32), tpm.BuildParams(leaf_bucket=1))
    a, p, k = s.compute_forces(fp=tpm.ForceParams(theta=1e-9))
    assert np.all(np.isfinite(a.cpu().numpy())) and list(k.cpu().numpy()[:3]) == [5, 5, 5]
    s.release()


def test_errors(tpm, ctx):
    E = tpm.TreePMError
    pos, mass = W.plummer(100, 1)
    s = ctx.build_tree(pos, mass, tpm.BuildParams())
    with pytest.raises(E, match="TPM_EINVAL"):  # relative criterion without a_old
        s.compute_forces(fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE))
    with pytest.raises(E, match="TPM_EINVAL"):  # out-of-range id (host)
        s.compute_forces(active_ids=np.array([5, 100], np.uint32), fp=tpm.ForceParams())
    with pytest.raises(E, match="TPM_ENAN"):
        s.compute_forces(active_ids=np.array([1], np.uint32), a_old=np.array([np.nan], np.float32),
                         fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE))
    with pytest.raises(E, match="TPM_EINVAL"):  # treepm on an open system
        s.compute_forces(fp=tpm.ForceParams(treepm=True))
    bad = pos.copy()
    bad[3, 1] = np.inf
    with pytest.raises(E, match="TPM_ENAN"):
        ctx.build_tree(bad, mass, tpm.BuildParams())
    with pytest.raises(E, match="TPM_EINVAL"):  # periodic positions outside [0, box)
        ctx.build_tree(pos, mass, tpm.BuildParams(periodic=True, box=1.0))
    s.release()
    with pytest.raises(E, match="TPM_ENOSYS_HANDLE"):
        s.handle = 12345
        s.release()


def test_host_argument_checks_report_first_index(tpm, ctx):
    """Host a_old and active ids are checked block by block; the error names
    the first failing element, also past the first block and in the tail."""
    E = tpm.TreePMError
    n = 20000
    pos, mass = W.plummer(n, 6)
    s = ctx.build_tree(pos, mass, tpm.BuildParams())
    ids = np.arange(n, dtype=np.uint32)
    fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE)
    aold = np.full(n, np.finfo(np.float32).max, np.float32)  # large but finite
    aold[::7] = np.float32(1e-42)  # subnormal, finite
    s.compute_forces(active_ids=ids, a_old=aold, fp=fp)  # accepted
    for bad_at in ([9001, 12288], [19999], [0, 5]):
        a = aold.copy()
        a[bad_at[0]] = np.nan
        for k in bad_at[1:]:
            a[k] = -np.inf
        with pytest.raises(E, match=r"a_old\[%d\] is not finite" % bad_at[0]):
            s.compute_forces(active_ids=ids, a_old=a, fp=fp)
    for bad_at in ([17000, 17001], [4096], [19999]):
        i = ids.copy()
        i[bad_at] = n + np.arange(len(bad_at), dtype=np.uint32)
        with pytest.raises(E, match=r"active_ids\[%d\] = %d out of range" % (bad_at[0], n)):
            s.compute_forces(active_ids=i, fp=tpm.ForceParams())
    s.release()


def test_budget_admission_has_no_side_effects(tpm):
    small = tpm.Context(0, budget_bytes=8 << 20)
    pos, mass = W.hernquist(200000, 2)
    used0, _ = small.memory()
    with pytest.raises(tpm.TreePMError, match="TPM_EBUDGET"):
        small.build_tree(pos, mass, tpm.BuildParams())
    assert small.memory()[0] == used0
    ok = small.build_tree(*W.plummer(1000, 2), tpm.BuildParams())
    ok.release()
    small.close()


@pytest.mark.parametrize("grad", ["fd4", "ik"])
def test_periodic_treepm_matches_oracle(oracle_mod, tpm, ctx, torch_dev, grad):
    """The 4-point difference and the spectral gradient of the mesh force."""
    ng_part, ng = 32, 64
    pos, mass = W.zeldovich(ng_part, 1003)
    n = len(pos)
    shift = tuple(W.root_shift(3))
    h = (1.0 / ng_part) / 40
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5, treepm=True, pm_n=ng, asmth=1.25, rcut=4.5,
                         pm_grad=tpm.GRAD_IK if grad == "ik" else tpm.GRAD_FD4)
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=1.0, h=h, periodic=True, box=1.0, shift=shift, leaf_bucket=8))
    s.pm_long_range(fp)
    phi_gpu = s.pm_export(ng).astype(np.float64)
    tg = np.arange(0, n, 7).astype(np.uint32)
    acc, pot, nint = s.compute_forces(active_ids=to_dev(tg, torch_dev), fp=fp)
    xtree = s.tree_export()["xtree"]
    s.release()
    # mesh potential (computed in the shifted frame the tree uses)
    rs = 1.25 / ng
    phi_o = oracle_mod.pm_potential(xtree, mass, 1.0, ng, rs)
    assert np.abs(phi_gpu - phi_o).max() < 1e-5 * np.abs(phi_o).max()
    # short-range walk + long-range mesh, element by element
    tree = oracle_mod.Tree(pos, mass, bucket=8, periodic=True, box=1.0, shift=shift)
    a_s, p_s, n_o = tree.walk(tg, 1.0, h, theta=0.5, treepm=True, rs=rs, rcut=4.5 * rs)
    a_l, p_l = oracle_mod.pm_interpolate(phi_o, xtree[tg], 1.0, grad=grad)
    compare_forces(acc.cpu().numpy().astype(np.float64), a_s + a_l, nint.cpu().numpy(), n_o, p99=1e-4, mx=1e-3)
    pot = pot.cpu().numpy().astype(np.float64)
    po = p_s + p_l
    assert np.abs((pot - pot.mean()) - (po - po.mean())).max() < 1e-4 * np.abs(po).max()


def test_spectral_gradient_needs_its_mesh(tpm, ctx, torch_dev):
    """A force call whose gradient differs from the solved mesh's is refused,
    and an open system takes only the 4-point difference."""
    pos, mass = W.zeldovich(16, 1003)
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev),
                       tpm.BuildParams(G=1.0, h=1e-3, periodic=True, box=1.0, leaf_bucket=8))
    fp = tpm.ForceParams(theta=0.5, treepm=True, pm_n=32, asmth=1.25, rcut=4.5)
    s.pm_long_range(fp)
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):
        s.compute_forces(fp=tpm.ForceParams(theta=0.5, treepm=True, pm_n=32, asmth=1.25, rcut=4.5,
                                            pm_grad=tpm.GRAD_IK))
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):
        s.pm_long_range(tpm.ForceParams(theta=0.5, treepm=True, pm_n=32, asmth=1.25, rcut=4.5, pm_grad=7))
    s.release()
    p2, m2 = W.plummer(2000, 3)
    s2 = ctx.build_tree(p2, m2, tpm.BuildParams())
    with pytest.raises(tpm.TreePMError, match="periodic"):
        s2.pm_long_range(tpm.ForceParams(theta=0.5, treepm=True, pm_n=32, asmth=1.25, rcut=4.5,
                                         pm_grad=tpm.GRAD_IK))
    s2.release()


LANE_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1909_04667_gb300 as tpm, workloads as W
dev = torch.device('cuda', 0)
ctx = tpm.Context(0)
out = {}
pos, mass = W.hernquist(50000, 8)
s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                   tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(8)), leaf_bucket=8))
a, p, n = s.compute_forces(fp=tpm.ForceParams(theta=0.5))
s.sync_status()
out['acc'], out['nint'] = a.cpu().numpy(), n.cpu().numpy()
pos, mass = W.zeldovich(32, 5)
fp = tpm.ForceParams(theta=0.5, treepm=True, pm_n=64, asmth=1.25, rcut=4.5)
s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                   tpm.BuildParams(G=1.0, h=1e-3, periodic=True, box=1.0, shift=tuple(W.root_shift(9)), leaf_bucket=8))
s.pm_long_range(fp)
ids = torch.from_numpy(np.arange(0, len(pos), 3).astype(np.int32)).to(dev)
a, p, n = s.compute_forces(active_ids=ids, fp=fp)
s.sync_status()
out['pacc'], out['pnint'] = a.cpu().numpy(), n.cpu().numpy()
s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                   tpm.BuildParams(G=1.0, h=1e-3, periodic=True, box=1.0, shift=tuple(W.root_shift(9)), leaf_bucket=8))
a, p, n = s.compute_forces(active_ids=ids, fp=tpm.ForceParams(theta=0.5))
s.sync_status()
out['eacc'], out['enint'] = a.cpu().numpy(), n.cpu().numpy()
np.savez(sys.argv[2], **out)
"""


def test_group_walk_matches_lane_walk(tmp_path):
    # two kernels, the same per-particle decisions: the default group walk and
    # the lane walk (TPM_WALK=lanes) must give the same interaction counts and
    # forces within FP32 summation-order differences
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "walk.py"
    script.write_text(LANE_SCRIPT)
    outs = []
    for mode in ("group", "lanes"):
        env = dict(os.environ)
        env["TPM_WALK"] = mode
        out = tmp_path / (mode + ".npz")
        subprocess.run([sys.executable, str(script), root, str(out)], check=True, env=env, timeout=600)
        outs.append(np.load(out))
    g, l = outs
    # open boundaries, periodic TreePM subset, periodic Ewald tree subset (the
    # linear box's small total forces: the periodic tolerance of its parity test)
    for acc, nint, p99, mx in (("acc", "nint", P99_TOL, MAX_TOL), ("pacc", "pnint", P99_TOL, MAX_TOL),
                               ("eacc", "enint", 1e-4, 1e-3)):
        assert np.mean(g[nint] != l[nint]) < 1e-3
        same = g[nint] == l[nint]
        e = rel(g[acc].astype(np.float64), l[acc].astype(np.float64))
        assert np.percentile(e[same], 99) < p99 and e[same].max() < mx, (acc, np.percentile(e[same], 99))


def test_sync_status_reports_device_errors(tpm, ctx, torch_dev):
    pos, mass = W.plummer(500, 4)
    s = ctx.build_tree(to_dev(pos, torch_dev), to_dev(mass, torch_dev), tpm.BuildParams())
    s.compute_forces(fp=tpm.ForceParams())
    s.sync_status()  # clean
    bad = to_dev(np.array([3, 7, 9999], np.uint32), torch_dev)  # device ids are checked on the device
    s.compute_forces(active_ids=bad, fp=tpm.ForceParams())
    with pytest.raises(tpm.TreePMError, match="out of range"):
        s.sync_status()
    s.sync_status()  # the word was cleared
    s.release()
