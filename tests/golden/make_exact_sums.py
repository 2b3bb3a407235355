"""Writes tests/golden/exact_sums.npz: the exact forces that the accuracy
figures of the bench and of the full-size tests are measured against.

Every value comes from the FP64 oracle (oracle/) on the seeded inputs of
workloads/; nothing here touches the CUDA library.

* ``hernquist``: the Hernquist halo, N = 2^20 (seed 1002), softening support
  0.005: the softened FP64 direct sum on 4096 seeded random targets.
* ``zeldovich``: the 128^3 Zel'dovich box (seed 1003): the FP64 Ewald sum with
  a neutralising background on 2048 seeded random targets (the potential is
  defined up to a constant and not stored).
* ``two_species``: the Hernquist halo (support 0.005) plus 2^18 stellar
  particles (support 0.001): the symmetrised (larger support) softened direct
  sum on 4096 targets.
* ``plummer``: the Plummer sphere, N = 8192 (seed 1001), support 0.01: the
  direct sum on every particle.

Run:  python tests/golden/make_exact_sums.py   (a few minutes on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "exact_sums.npz")
TARGET_SEEDS = {"hernquist": 4096, "zeldovich": 2048, "two_species": 4097}


def targets(name: str, n: int, k: int) -> np.ndarray:
    return W.random_targets(n, k, TARGET_SEEDS[name])


def main():
    oracle.build()
    out = {}
    t0 = time.time()
    pos, mass = W.hernquist(1 << 20, W.CONFIG_SEEDS[2])
    tg = targets("hernquist", len(pos), 4096)
    a, p = oracle.direct(pos, mass, tg, 1.0, 0.005)
    out.update(hernquist_targets=tg, hernquist_acc=a, hernquist_pot=p)
    print("hernquist %.1f s" % (time.time() - t0))
    pos, mass = W.zeldovich(128, W.CONFIG_SEEDS[3])
    tg = targets("zeldovich", len(pos), 2048)
    a, _ = oracle.ewald(pos, mass, tg, 1.0, 1.0)
    out.update(zeldovich_targets=tg, zeldovich_acc=a)
    print("zeldovich %.1f s" % (time.time() - t0))
    pos, mass, hs, _ = W.two_species(1 << 20, 1 << 18, W.CONFIG_SEEDS[2])
    tg = targets("two_species", len(pos), 4096)
    a, p = oracle.direct_soft(pos, mass, hs, tg, 1.0)
    out.update(two_species_targets=tg, two_species_acc=a, two_species_pot=p)
    print("two_species %.1f s" % (time.time() - t0))
    pos, mass = W.plummer(8192, W.CONFIG_SEEDS[1])
    tg = np.arange(8192, dtype=np.uint32)
    a, p = oracle.direct(pos, mass, tg, 1.0, 0.01)
    out.update(plummer_targets=tg, plummer_acc=a, plummer_pot=p)
    np.savez_compressed(OUT, **out)
    print("wrote %s (%.1f s)" % (OUT, time.time() - t0))


if __name__ == "__main__":
    main()
