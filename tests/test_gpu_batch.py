"""Batched homogenization (gfp_batch_create / gfp_batch_solve / gfp_solve_batch): cells of different
sizes x 6 Voigt loads as one CUDA graph in which every (cell, load) slot loops on the device, mixed
precision; against per-cell solves and the FP64 oracle."""
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


def _cells(gfp, specs, rmin=2.0, rmax=4.0):
    grids, fields = [], []
    for sp in specs:
        lam, mu = M.random_spheres(sp["n"], vf=sp["vf"], rmin=rmin, rmax=rmax, contrast=sp["contrast"],
                                   seed=sp["seed"])
        g = gfp.Grid(sp["n"], sp["n"], sp["n"])
        g.set_phases(lam, mu)
        grids.append(g)
        fields.append((lam, mu))
    return grids, fields


def _against_single(gfp, C, grids, sch, tol=1e-8):
    for i, g in enumerate(grids):
        Cs, _, rcs = g.effective_stiffness(sch, tol, 20000)
        assert rcs == 0
        assert np.abs(C[i] - Cs).max() / np.abs(Cs).max() <= 1e-6


def test_batch_matches_single_solves_and_oracle(gfp):
    specs = [dict(n=16, vf=0.2, contrast=30.0, seed=3), dict(n=24, vf=0.15, contrast=0.05, seed=4),
             dict(n=32, vf=0.25, contrast=200.0, seed=5)]
    grids, fields = _cells(gfp, specs)
    sch = gfp.scheme("AFB_R", "PCD", "MIXED")
    C, its, rc = gfp.solve_batch(grids, sch, tol=1e-8, maxit=20000)
    assert rc == 0 and np.all(its > 0)
    _against_single(gfp, C, grids, sch)
    for i in range(len(grids)):
        np.testing.assert_allclose(C[i], C[i].T, rtol=1e-5, atol=1e-7 * np.abs(C[i]).max())
    lam, mu = fields[0]
    Cref, _, _ = O.effective_stiffness(lam, mu, "AFB_R", tol=1e-10, maxit=20000, disc="PCD")
    assert np.abs(C[0] - Cref).max() / np.abs(Cref).max() <= 1e-6


def test_batch_handle_reuse_and_new_phases(gfp):
    """A handle solved twice gives the same results bit for bit (every slot starts again from E_J);
    new phases on one grid make the next solve rebuild the graph, and it matches a single solve."""
    specs = [dict(n=16, vf=0.2, contrast=10.0, seed=7), dict(n=24, vf=0.25, contrast=0.1, seed=8)]
    grids, _ = _cells(gfp, specs)
    sch = gfp.scheme("ACD", "PCD", "MIXED")
    b = gfp.Batch(grids, sch)
    try:
        C1, it1, rc1 = b.solve(1e-8, 20000)
        C2, it2, rc2 = b.solve(1e-8, 20000)
        assert rc1 == 0 and rc2 == 0
        assert np.array_equal(C1, C2) and np.array_equal(it1, it2)
        lam, mu = M.random_spheres(24, vf=0.2, rmin=2.0, rmax=4.0, contrast=40.0, seed=9)
        grids[1].set_phases(lam, mu)
        C3, it3, rc3 = b.solve(1e-8, 20000)
        assert rc3 == 0
        assert np.array_equal(C3[0], C1[0])
        _against_single(gfp, C3, grids, sch)
    finally:
        b.close()


def test_batch_window_budget_ends_every_loop(gfp):
    """With a budget of two windows (maxit 40) the slots' device loops end after two windows and the
    call reports GFP_ERR_NOT_CONVERGED with the iterations done."""
    specs = [dict(n=16, vf=0.25, contrast=1000.0, seed=11)]
    grids, _ = _cells(gfp, specs)
    sch = gfp.scheme("AFB_R", "PCD", "MIXED")
    C, its, rc = gfp.solve_batch(grids, sch, tol=1e-12, maxit=40)
    assert rc == -4
    assert np.all(its > 0) and np.all(its <= 64)
    assert np.isfinite(C).all()


def test_batch_config_sizes_against_single_solves(gfp):
    """Cells of the batched configuration's sizes 64^3, 96^3 and 128^3 (radii U[6, 16] scaled by n/128)."""
    specs = [dict(n=64, vf=0.2, contrast=20.0, seed=21), dict(n=96, vf=0.3, contrast=0.05, seed=22),
             dict(n=128, vf=0.15, contrast=5.0, seed=23)]
    grids = []
    for sp in specs:
        f = sp["n"] / 128.0
        lam, mu = M.random_spheres(sp["n"], vf=sp["vf"], rmin=6.0 * f, rmax=16.0 * f, contrast=sp["contrast"],
                                   seed=sp["seed"])
        g = gfp.Grid(sp["n"], sp["n"], sp["n"])
        g.set_phases(lam, mu)
        grids.append(g)
    sch = gfp.scheme("AFB_R", "PCD", "MIXED")
    C, its, rc = gfp.solve_batch(grids, sch, tol=1e-8, maxit=20000)
    assert rc == 0 and np.all(its > 0)
    _against_single(gfp, C, grids, sch)
