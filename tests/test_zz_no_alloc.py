"""tpm_compute_forces_noalloc: the force evaluation for callers that cannot let
the library allocate device memory (their device memory already belongs to
their own allocator, or an allocation inside the time-step loop is not
allowed).  It must give what tpm_compute_forces gives, call after call, with
its scratch in the library's fixed device array.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

P99_TOL = 2e-5  # the FP32 walk tolerance of the parity tests
MAX_TOL = 2e-4


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def close(a, b):
    e = rel(a.astype(np.float64), b.astype(np.float64))
    return np.percentile(e, 99) <= P99_TOL and e.max() <= MAX_TOL


def test_noalloc_matches_compute_forces_two_calls():
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    ctx = tpm.Context(0)
    pos, mass = W.hernquist(40000, 21)
    s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                       tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(21)), leaf_bucket=8))
    rng = np.random.default_rng(5)
    fp_bh = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5)
    fp_rel = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.0025)
    for call, fp in enumerate((fp_bh, fp_rel)):
        # a different ragged, unsorted active set on each call
        ids = torch.from_numpy(rng.choice(len(pos), 7001 + 1234 * call, replace=False).astype(np.int32)).to(dev)
        a_old = torch.rand(len(ids), device=dev) + 0.5 if fp is fp_rel else None
        ref_acc, ref_pot, ref_n = s.compute_forces(active_ids=ids, a_old=a_old, fp=fp)
        acc = torch.full((len(ids), 3), float("nan"), device=dev)
        pot = torch.full((len(ids),), float("nan"), device=dev)
        n_int = torch.zeros(len(ids), dtype=torch.int32, device=dev)
        s.compute_forces_noalloc(ids, acc, a_old=a_old, fp=fp, pot=pot, n_int=n_int)
        torch.cuda.synchronize()
        assert close(acc.cpu().numpy(), ref_acc.cpu().numpy())
        np.testing.assert_allclose(pot.cpu().numpy(), ref_pot.cpu().numpy(), rtol=P99_TOL)
        np.testing.assert_array_equal(n_int.cpu().numpy(), ref_n.cpu().numpy())
    s.release()
    ctx.close()


def test_noalloc_at_the_maximum_size():
    """Exactly TPM_NOALLOC_MAX_ACTIVE ids: the sort's temporary storage fits
    the fixed array (the sort runs on double buffers), results as the plain
    call's."""
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    ctx = tpm.Context(0)
    n = tpm.NOALLOC_MAX_ACTIVE + 4097
    pos, mass = W.hernquist(n, 22)
    s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                       tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(22)), leaf_bucket=8))
    rng = np.random.default_rng(6)
    ids = torch.from_numpy(rng.permutation(n)[:tpm.NOALLOC_MAX_ACTIVE].astype(np.int32)).to(dev)
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.5)
    ref_acc, ref_pot, ref_n = s.compute_forces(active_ids=ids, fp=fp)
    acc = torch.full((len(ids), 3), float("nan"), device=dev)
    pot = torch.full((len(ids),), float("nan"), device=dev)
    n_int = torch.zeros(len(ids), dtype=torch.int32, device=dev)
    s.compute_forces_noalloc(ids, acc, fp=fp, pot=pot, n_int=n_int)
    s.sync_status()
    assert close(acc.cpu().numpy(), ref_acc.cpu().numpy())
    np.testing.assert_allclose(pot.cpu().numpy(), ref_pot.cpu().numpy(), rtol=P99_TOL)
    np.testing.assert_array_equal(n_int.cpu().numpy(), ref_n.cpu().numpy())
    s.release()
    ctx.close()


def test_noalloc_reports_an_out_of_range_id():
    """An id >= n in device memory (built on the host, so nothing faults) is
    read as particle 0 and reported by the next sync_status, as for the plain
    call; the status word is cleared, and the next good call succeeds."""
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    ctx = tpm.Context(0)
    pos, mass = W.plummer(2000, 8)
    s = ctx.build_tree(pos, mass, tpm.BuildParams())
    ids_h = np.arange(0, 2000, 7, dtype=np.int32)
    ids_h[5] = 2000  # one past the last particle
    ids = torch.from_numpy(ids_h).to(dev)
    acc = torch.empty((len(ids), 3), device=dev)
    s.compute_forces_noalloc(ids, acc)
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL.*out of range"):
        s.sync_status()
    ids_h[5] = 1999
    ids = torch.from_numpy(ids_h).to(dev)
    s.compute_forces_noalloc(ids, acc)
    s.sync_status()
    ref, _, _ = s.compute_forces(active_ids=ids)
    assert close(acc.cpu().numpy(), ref.cpu().numpy())
    s.release()
    ctx.close()


def test_noalloc_rejects_what_it_cannot_hold():
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    ctx = tpm.Context(0)
    pos, mass = W.plummer(1000, 3)
    s = ctx.build_tree(pos, mass, tpm.BuildParams())
    too_many = torch.zeros(tpm.NOALLOC_MAX_ACTIVE + 1, dtype=torch.int32, device=dev)
    acc = torch.empty((len(too_many), 3), device=dev)
    with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):
        s.compute_forces_noalloc(too_many, acc)
    host_ids = np.arange(10, dtype=np.uint32)
    with pytest.raises(tpm.TreePMError, match="device memory"):
        s.compute_forces_noalloc(host_ids, torch.empty((10, 3), device=dev))
    with pytest.raises(ValueError, match="acc must have shape"):
        s.compute_forces_noalloc(torch.zeros(10, dtype=torch.int32, device=dev), torch.empty((9, 3), device=dev))
    s.release()
    ctx.close()
