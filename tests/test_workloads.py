"""The seeded generators: shapes, determinism and the time-bin hierarchy."""
import numpy as np

import workloads as W


def test_generators_are_deterministic_and_shaped():
    for f, args in ((W.plummer, (1000, 3)), (W.hernquist, (1000, 3))):
        a, m = f(*args)
        b, _ = f(*args)
        assert a.shape == (1000, 3) and a.dtype == np.float64 and m.dtype == np.float32
        np.testing.assert_array_equal(a, b)
    z, m = W.zeldovich(16, 3)
    assert z.shape == (4096, 3) and np.all(z >= 0) and np.all(z < 1)
    d = (z - W.lattice(16) + 0.5) % 1.0 - 0.5
    assert abs(np.sqrt((d ** 2).sum(1).mean()) - 0.3 / 16) < 1e-12


def test_timebins_give_power_of_two_active_fractions():
    pos, _ = W.hernquist(1 << 14, 2)
    bins = W.timebins(pos, 4)
    n = len(bins)
    for step in range(128):
        b = W.substep_active_bins(step)
        frac = np.mean(bins >= b)
        assert abs(frac - 2.0 ** -b) < 2.0 / n
    # the densest (innermost) particles get the shortest steps on average
    r = np.linalg.norm(pos, axis=1)
    assert np.median(r[bins == 7]) < np.median(r[bins == 0])


def test_request_sizes_cover_the_set():
    s = W.request_sizes(100000, 7)
    assert s.sum() == 100000 and s.min() >= 1 and s.max() <= 65536


def test_clusters_with_outliers_layout():
    pos, mass = W.clusters_with_outliers(4096, 78)
    assert pos.shape == (4096, 3) and mass.dtype == np.float32 and abs(mass.sum() - 1.0) < 1e-5
    far = pos[2030:2035]
    assert np.all(np.abs(far) >= 300.0) and np.abs(far).max() == 3.0e4
    np.testing.assert_allclose(pos[:2030].mean(0), -300.0, atol=1.0)
    np.testing.assert_allclose(pos[2035:].mean(0), 300.0, atol=1.0)
