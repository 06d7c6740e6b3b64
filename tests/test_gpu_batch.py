"""Batched homogenization (gfp_solve_batch): cells of different sizes x 6 Voigt loads in one
graph-replayed batch, mixed precision; against per-cell solves and the FP64 oracle."""
import numpy as np
import pytest

from oracle import gfp_oracle as O
from paper_2009_03762_gb300 import microstructure as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gfp():
    from paper_2009_03762_gb300 import gfp as G
    G.lib()
    return G


def test_batch_matches_single_solves_and_oracle(gfp):
    specs = [dict(n=16, vf=0.2, contrast=30.0, seed=3), dict(n=24, vf=0.15, contrast=0.05, seed=4),
             dict(n=32, vf=0.25, contrast=200.0, seed=5)]
    grids, fields = [], []
    for sp in specs:
        lam, mu = M.random_spheres(sp["n"], vf=sp["vf"], rmin=2.0, rmax=4.0, contrast=sp["contrast"], seed=sp["seed"])
        g = gfp.Grid(sp["n"], sp["n"], sp["n"])
        g.set_phases(lam, mu)
        grids.append(g)
        fields.append((lam, mu))
    sch = gfp.scheme("AFB_R", "PCD", "MIXED")
    C, its, rc = gfp.solve_batch(grids, sch, tol=1e-8, maxit=20000)
    assert rc == 0 and np.all(its > 0)
    for i, g in enumerate(grids):
        Cs, _, rcs = g.effective_stiffness(sch, 1e-8, 20000)
        assert rcs == 0
        assert np.abs(C[i] - Cs).max() / np.abs(Cs).max() <= 1e-6
        np.testing.assert_allclose(C[i], C[i].T, rtol=1e-5, atol=1e-7 * np.abs(C[i]).max())
    lam, mu = fields[0]
    Cref, _, _ = O.effective_stiffness(lam, mu, "AFB_R", tol=1e-10, maxit=20000, disc="PCD")
    assert np.abs(C[0] - Cref).max() / np.abs(Cref).max() <= 1e-6
