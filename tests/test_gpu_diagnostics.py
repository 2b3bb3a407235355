"""FP64 conservation diagnostics on the GPU [Sec. 7] against the oracle's
plain sums of the same arrays, the tree's total-force residual against the
oracle tree walk's (the same interactions), and bit-reproducibility."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_diagnostics_match_oracle(oracle_mod):
    import torch

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    n = 20000
    pos, mass = W.plummer(n, 23)
    rng = np.random.default_rng(4)
    vel = rng.normal(size=(n, 3))
    shift = tuple(W.root_shift(23))
    with tpm.Context(0) as ctx:
        s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                           tpm.BuildParams(G=1.0, h=0.01, shift=shift, leaf_bucket=8))
        acc, pot, _ = s.compute_forces(fp=tpm.ForceParams(theta=0.5))
        v_d = torch.from_numpy(vel).to(dev)
        d = s.diagnostics(acc, pot, v_d)
        d2 = s.diagnostics(acc, pot, v_d)
        with pytest.raises(tpm.TreePMError, match="TPM_EINVAL"):  # host arrays
            s.diagnostics(acc.cpu(), pot)
        s.release()
    ref = oracle_mod.diagnostics(mass, acc.cpu().numpy(), pot.cpu().numpy(), vel)
    scale = ref["force_scale"]
    assert abs(d["force_scale"] - scale) < 1e-12 * scale
    assert np.abs(d["total_force"] - ref["total_force"]).max() < 1e-12 * scale
    for k in ("potential_energy", "kinetic_energy"):
        assert abs(d[k] - ref[k]) < 1e-12 * abs(ref[k])
    np.testing.assert_allclose(d["momentum"], ref["momentum"], rtol=0, atol=1e-12 * np.abs(vel).sum() / n)
    for k in d:  # fixed order: the same bits on every call
        np.testing.assert_array_equal(d[k], d2[k])
    # the tree's residual equals the oracle tree walk's within the FP32 force rounding
    tree = oracle_mod.Tree(pos, mass, bucket=8, shift=shift)
    a_o, _, _ = tree.walk(np.arange(n), 1.0, 0.01, theta=0.5)
    r_o = oracle_mod.diagnostics(mass, a_o)["total_force"]
    assert np.linalg.norm(r_o) > 1e-6 * scale  # a tree is not exactly symmetric
    assert np.linalg.norm(d["total_force"] - r_o) < 1e-5 * scale


def test_hernquist_potential_energy_closed_form():
    """The potential energy of a Hernquist sample truncated at 100 a (the
    workload normalises the mass inside 100 a to 1: M(r) = c (r / (r + a))^2,
    c = (101/100)^2) against W = -G int M dM / r = -2 c^2 G M^2 / a
    int_0^100 r^2 / (r + 1)^5 dr, within the sampling noise of 2^18 particles
    and the method's error."""
    import torch
    from scipy import integrate

    import paper_1909_04667_gb300 as tpm

    dev = torch.device("cuda", 0)
    pos, mass = W.hernquist(1 << 18, 31)
    c = (101.0 / 100.0) ** 2
    w_exact = -2.0 * c * c * integrate.quad(lambda r: r * r / (r + 1.0) ** 5, 0.0, 100.0)[0]
    with tpm.Context(0) as ctx:
        s = ctx.build_tree(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                           tpm.BuildParams(G=1.0, h=0.005, shift=tuple(W.root_shift(31)), leaf_bucket=8))
        acc, pot, _ = s.compute_forces(fp=tpm.ForceParams(theta=0.5))
        d = s.diagnostics(acc, pot)
        s.release()
    assert abs(d["potential_energy"] - w_exact) < 1e-2 * abs(w_exact)
