"""The GPU walk's opening decisions at their exact boundaries (Sec. 3.1, 3.4),
on the hand-built trees the oracle pins use (tests/test_oracle_forces.py): the
1.2 L box guard, the distance to the centre of mass in the geometric
criterion, the relative criterion's threshold G M L^2 / d^4 and the TreePM
cutoff measured to the node's cube.  Each case sits 1-3% from its boundary,
far above FP32 resolution, so the GPU and the FP64 oracle must count the same
interactions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ANCHORS = [[0, 0, 0], [100, 100, 100]]  # fix the root: x0 = 0, L0 = 128


@pytest.fixture(scope="module")
def tpm():
    import paper_1909_04667_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(tpm):
    c = tpm.Context(0)
    yield c
    c.close()


def counts(tpm, ctx, oracle_mod, pos, mass, G, fp, owalk):
    """Interaction count of the probe (index 4) on the GPU and in the oracle."""
    bp = tpm.BuildParams(G=G, h=1e-3, shift=(0.0, 0.0, 0.0), leaf_bucket=1)
    s = ctx.build_tree(pos, mass, bp)
    try:
        ti = s.tree_info()
        if fp.treepm:
            s.pm_long_range(fp)
        kw = {}
        if fp.crit == tpm.CRIT_RELATIVE:
            kw["a_old"] = np.array([1.0], np.float32)
        acc = np.zeros((1, 3), np.float32)
        nint = np.zeros(1, np.uint32)
        s.compute_forces(active_ids=np.array([4], np.uint32), fp=fp, acc=acc, n_int=nint, **kw)
        s.sync_status()
    finally:
        s.release()
    tree = oracle_mod.Tree(pos, mass, bucket=1, shift=(0.0, 0.0, 0.0))
    _, _, n_o = owalk(tree)
    return int(nint[0]), int(n_o[0]), ti


@pytest.mark.parametrize("off,expect", [(0.55, 4), (0.59, 4), (0.61, 3), (0.65, 3)])
def test_box_guard_boundary(tpm, ctx, oracle_mod, off, expect):
    pos = np.array(ANCHORS + [[65, 65, 65], [66, 66, 66], [66 + off * 4, 66, 66]], float)
    mass = np.full(5, 0.2, np.float32)
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=100.0, box_guard=True)
    g, o, _ = counts(tpm, ctx, oracle_mod, pos, mass, 1.0, fp,
                     lambda t: t.walk([4], 1.0, 1e-3, theta=100.0, box_guard=True))
    assert g == o == expect


PAIR = ANCHORS + [[64.5, 66.5, 66.5], [67.5, 66.5, 66.5], [80.0, 66.5, 66.5]]
PAIR_MASS = np.array([1e-6, 1e-6, 1.0, 1e-3, 1e-6], np.float32)


@pytest.mark.parametrize("theta,expect", [(0.25, 4), (0.27, 3), (0.29, 3)])
def test_geometric_criterion_uses_centre_of_mass(tpm, ctx, oracle_mod, theta, expect):
    pos = np.array(PAIR, float)
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=theta, box_guard=False)
    g, o, _ = counts(tpm, ctx, oracle_mod, pos, PAIR_MASS, 1.0, fp,
                     lambda t: t.walk([4], 1.0, 1e-3, theta=theta, box_guard=False))
    assert g == o == expect


@pytest.mark.parametrize("f,expect", [(0.99, 4), (1.01, 3)])
def test_relative_criterion_threshold(tpm, ctx, oracle_mod, f, expect):
    pos = np.array(PAIR, float)
    M = float(PAIR_MASS[2]) + float(PAIR_MASS[3])
    com = (pos[2] * float(PAIR_MASS[2]) + pos[3] * float(PAIR_MASS[3])) / M
    G = 2.0
    alpha = f * G * M * 4.0 ** 2 / np.linalg.norm(pos[4] - com) ** 4
    fp = tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=alpha)
    g, o, _ = counts(tpm, ctx, oracle_mod, pos, PAIR_MASS, G, fp,
                     lambda t: t.walk([4], G, 1e-3, crit="rel", alpha=alpha, a_old=np.array([1.0], np.float32)))
    assert g == o == expect


@pytest.mark.parametrize("rcut,expect", [(11.9, 0), (12.1, 1), (15.0, 1)])
def test_treepm_cutoff_to_the_cube(tpm, ctx, oracle_mod, rcut, expect):
    # open boundaries: the mesh spans the root cube (128), r_s = 1.25 * 128 / 32 = 5
    pos = np.array(PAIR, float)
    rs = 1.25 * 128.0 / 32
    fp = tpm.ForceParams(crit=tpm.CRIT_BH, theta=0.4, treepm=True, pm_n=32, asmth=1.25, rcut=rcut / rs)
    g, o, ti = counts(tpm, ctx, oracle_mod, pos, PAIR_MASS, 1.0, fp,
                      lambda t: t.walk([4], 1.0, 1e-3, theta=0.4, treepm=True, rs=rs, rcut=rcut))
    assert ti["L0"] == 128.0
    assert g == o == expect
