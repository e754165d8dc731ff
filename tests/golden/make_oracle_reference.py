"""Write the high-statistics oracle doses the GPU parity tests compare to.

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``paper_1809_03927_gb300.workloads``).  For each case the oracle runs
``n_hist`` histories as ``n_batches`` interleaved batches (batch b = the
histories h with h mod n_batches == b, so every batch samples every spot); the file
stores, inside the bounding box of voxels at or above 5 % of the maximum,
the mean dose and its standard error (batch method), as float32:

  oracle_<case>.npz: lo (k, j, i of the box corner), mean, sem, dmax,
                     n_hist, seed, n_batches

Usage: python tests/golden/make_oracle_reference.py [case ...]
Cases:
  pencil_1e7   single 150 MeV pencil beam, sigma 4 mm, in water 64x64x160 at
               2 mm, 1e7 histories;
  slab_2e8     slab phantom 128^3 at 2 mm, 400 spots on 10 layers 70-200 MeV
               (the benchmark workload), 2e8 histories, so that the standard
               error of the voxels above 10 % of the maximum stays below about
               0.4 % of it;
  4dct_p0_1e8  phase 0 of the 10-phase 256x256x160 4DCT at 1x1x2.5 mm, the
               whole 3000-spot plan (20 layers, 70-180 MeV) along +y, 1e8
               histories (dmax taken inside the body, density >= 0.1).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1809_03927_gb300 import workloads as W  # noqa: E402

def _4dct_phase0():
    ph, _, geo = W.phantom_4dct()
    return ph, W.tumour_plan(geo, ph.origin)


CASES = {
    "pencil_1e7": dict(make=lambda: (W.water_phantom(), W.pencil_plan(150.0, 4.0)),
                       n_hist=10_000_000, seed=101, n_batches=100),
    "slab_2e8": dict(make=lambda: (W.slab_phantom(128), W.slab_plan(seed=2)),
                     n_hist=200_000_000, seed=102, n_batches=100),
    "4dct_p0_1e8": dict(make=_4dct_phase0, n_hist=100_000_000, seed=103, n_batches=100, phase=0),
}


def run(name):
    c = CASES[name]
    phantom, plan = c["make"]()
    n, seed, nb = c["n_hist"], c["seed"], c["n_batches"]
    phase = c.get("phase")
    rho = oracle.density(phantom, phase)
    w_bar = float(np.sum(plan.protons.astype(np.float64))) / n
    v = phantom.d[0] * phantom.d[1] * phantom.d[2] / 1000.0
    s1 = np.zeros(rho.shape)
    s2 = np.zeros(rho.shape)
    t0 = time.time()
    for b in range(nb):
        r = oracle.transport(phantom, plan, n, seed, phase=phase, stream=phase or 0, batch=(b, nb))
        d = oracle.normalise(r["edep"], rho, w_bar, v) * (n / r["histories"])
        s1 += d
        s2 += d * d
        if b % 10 == 9:
            print(f"{name}: batch {b + 1}/{nb}, {time.time() - t0:.0f} s", flush=True)
    mean = s1 / nb
    var = np.maximum(s2 / nb - mean * mean, 0.0) * nb / (nb - 1)
    sem = np.sqrt(var / nb)
    dmax = mean[rho >= 0.1].max()
    idx = np.argwhere((mean >= 0.05 * dmax) & (rho >= 0.1))
    lo, hi = idx.min(axis=0), idx.max(axis=0) + 1
    box = tuple(slice(a, b) for a, b in zip(lo, hi))
    out = os.path.join(HERE, f"oracle_{name}.npz")
    np.savez_compressed(out, lo=lo.astype(np.int32), mean=mean[box].astype(np.float32),
                        sem=sem[box].astype(np.float32), dmax=np.float64(dmax), n_hist=n, seed=seed,
                        n_batches=nb)
    print(f"{name}: {time.time() - t0:.0f} s, box {hi - lo}, {out}")


if __name__ == "__main__":
    oracle.build()
    for name in (sys.argv[1:] or list(CASES)):
        run(name)
