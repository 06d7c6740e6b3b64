"""Writes c1_plain_basic_32.npz: the oracle's solution of the 32^3 plain basic-scheme workload.

Workload: 32^3 periodic grid, centred sharp cubic inclusion of edge 16 voxels (by voxel index),
isotropic matrix E = 1, nu = 0.3 and inclusion E = 10, nu = 0.3; reference medium 1/2 (min + max)
of each Lame constant; mean strain E_xx = 0.01; plain Fourier wave vectors (TD); stop at eta < 1e-8.
Stored: iteration count, final residual, mean stress, the strain norm and the strain at 256 seeded
sample voxels.  Calls only the oracle (about two minutes of CPU).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import gfp_oracle as O  # noqa: E402
from paper_2009_03762_gb300 import microstructure as M  # noqa: E402

if __name__ == "__main__":
    lam, mu = M.sharp_cube(32, 16, 1.0, 10.0, 0.3)
    r = O.solve(lam, mu, "F", [0.01, 0, 0, 0, 0, 0], tol=1e-8, maxit=20000)
    rng = np.random.default_rng(2024)
    idx = rng.choice(lam.size, size=256, replace=False)
    eps = r.eps.reshape(6, -1)
    np.savez(os.path.join(HERE, "c1_plain_basic_32.npz"), iters=r.iters, residual=r.residual,
             sigma_mean=r.sigma_mean, eps_norm=np.linalg.norm(eps), sample_idx=idx, eps_samples=eps[:, idx],
             history=np.array(r.history))
    print("iters", r.iters, "residual", r.residual)
