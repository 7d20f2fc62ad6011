"""Writes the expected results of the full-run parity windows of the 128^3
shell (config 1) and the 256^3 biventricular heart (config 2) by running the
FP64 oracle (``oracle/``) -- the only code this script runs; inputs come from
``workloads`` (seeded, closed form) and the spectral interval from the
oracle's operator (``tests/spectra.py``).

Each window starts from ``workloads.front_state`` (a front ten voxels above
the apex) and runs the bidomain step with the elliptic solve by the Chebyshev
semi-iteration on a fixed interval, to rel_tol 1e-6; tests/test_gpu_windows.py
runs the same steps on the library with its damped Jacobi and with the
Chebyshev semi-iteration on the same interval, to the same tolerance.
  config 1: 60 steps; the interval from the oracle's spectrum of D^-1 A
            (smallest nonzero x 0.8, largest x 1.05);
  config 2: 1 step; the largest eigenvalue by Lanczos (x 1.05) and the
            lower end a literal 1e-3 (factorising the 3.4M-voxel operator is
            out of reach).  The oracle's FP64 solve of the first step takes
            2961 sweeps (half an hour on 8 cores); the second, from the first
            one's v_e, did not finish within an hour, so the window is one
            complete step.
Stored (npz): the interval, sweeps per step, and at the end of the window
activation times, v and v_e -- for config 1 on every tissue voxel, for
config 2 on the voxels that activated or lie on the front (0.01 < v < 0.99)
plus 20000 seeded random tissue voxels.

Usage: python tests/golden/make_windows.py [config1|config2]  (about 1 h for config 1, 45 min for
config 2, on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import spectra  # noqa: E402
import workloads as W  # noqa: E402

WINDOWS = {"config1": 60, "config2": 1}
CONFIG2_LMIN = 1e-3


def make(name: str) -> str:
    c = W.config1() if name == "config1" else W.config2()
    p = c.params
    sL, sT = p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT
    g = oracle.Grid.elliptic_from_case(c)
    t0 = time.time()
    if name == "config1":
        lmin, lmax = spectra.chebyshev_params(g, sL, sT)
    else:
        lmin, lmax = CONFIG2_LMIN, 1.05 * spectra.largest(g, sL, sT)
    print(f"{name}: interval [{lmin:.6g}, {lmax:.6g}] in {time.time() - t0:.0f} s", flush=True)
    p.solver, p.cheb_lmin, p.cheb_lmax = 1, lmin, lmax
    o = oracle.Sim(c)
    o.set_state(*W.front_state(c), 0)
    sweeps = []
    for i in range(WINDOWS[name]):
        t0 = time.time()
        st = o.step()
        assert st == 0, f"oracle step {i} returned {st}"
        sweeps.append(o.last_iters)
        print(f"  step {i + 1}: {o.last_iters} sweeps, {time.time() - t0:.0f} s", flush=True)
    s = o.state()
    tissue = np.nonzero(c.mask.reshape(-1))[0]
    if name == "config1":
        sel = tissue
    else:
        front = tissue[(s["tact"][tissue] > 0) | ((s["v"][tissue] > 0.01) & (s["v"][tissue] < 0.99))]
        rng = np.random.default_rng(0)
        sel = np.union1d(front, rng.choice(tissue, 20000, replace=False))
    out = os.path.join(HERE, f"window_{name}.npz")
    np.savez_compressed(out, steps=WINDOWS[name], lmin=lmin, lmax=lmax, sweeps=np.array(sweeps),
                        idx=sel.astype(np.int32), tact=s["tact"][sel], v=s["v"][sel].astype(np.float32),
                        ve=s["ve"][sel].astype(np.float32), n_tissue=len(tissue))
    return out


if __name__ == "__main__":
    for name in sys.argv[1:] or ["config1", "config2"]:
        print(make(name), flush=True)
