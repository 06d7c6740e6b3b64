"""Mixed precision (FP32 FFT / Gamma / stress inner iterations, FP64 residual, mean strain and
refinement) against the FP64 oracle and the FP64 GPU solve.

Bar: the mixed solve reaches the FP64 residual tolerance; its effective stiffness matches the FP64
oracle to a relative error <= 1e-6.
"""
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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.mark.parametrize("op", ["AFB_R", "ACD", "CD", "AHC"])
def test_mixed_reaches_fp64_tolerance_and_matches_oracle(gfp, op):
    lam, mu = M.random_spheres(24, vf=0.25, rmin=3.0, rmax=5.0, contrast=100.0, seed=1)
    E = [0.0, 0.0, 0.0, 0.0, 0.0, 0.5]
    g = gfp.Grid(24, 24, 24)
    g.set_phases(lam, mu)
    r = g.solve(gfp.scheme(op, "PCD", "MIXED"), E, 1e-8, 20000)
    assert r.converged and r.residual < 1e-8 and r.outer >= 2
    eps = g.strain()
    ref = O.solve(lam, mu, op, E, tol=1e-8, maxit=20000, disc="PCD")
    assert _rel(r.sigma_mean, ref.sigma_mean) <= 1e-6
    assert _rel(eps, ref.eps) <= 1e-6
    # the mean strain is held exactly in FP64
    np.testing.assert_allclose(eps.reshape(6, -1).mean(axis=1), E, atol=1e-12)


def test_mixed_effective_stiffness_matches_oracle(gfp):
    lam, mu = M.random_spheres(16, vf=0.2, rmin=2.0, rmax=4.0, contrast=100.0, seed=3)
    g = gfp.Grid(16, 16, 16)
    g.set_phases(lam, mu)
    C, its, rc = g.effective_stiffness(gfp.scheme("AFB_R", "PCD", "MIXED"), 1e-8, 20000)
    Cref, _, _ = O.effective_stiffness(lam, mu, "AFB_R", tol=1e-10, maxit=20000, disc="PCD")
    assert rc == 0
    assert np.abs(C - Cref).max() / np.abs(Cref).max() <= 1e-6


def test_mixed_unsupported_combinations(gfp):
    lam, mu = M.random_field(8, 8, 8, seed=2)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    for op in ("F", "HC"):
        with pytest.raises(gfp.GfpError) as e:
            g.solve(gfp.scheme(op, prec="MIXED"), [0.01, 0, 0, 0, 0, 0], 1e-8, 100, raise_on_error=True)
        assert e.value.code == -8


@pytest.mark.parametrize("zcols", [8, -8, 4, 2])
def test_mixed_z_tile_widths_on_256_columns(gfp, zcols):
    """z-pass tiles of 8 columns (two lines per thread; -8: TMA-fed with warp-shuffle transforms), 4 and
    2 on n3 = 256 with a ragged k1 range (n1/2 + 1 = 9 columns): the mixed solve matches the FP64 GPU
    solve."""
    lam, mu = M.random_field(16, 8, 256, seed=5)
    E = [0.0, 0.0, 0.0, 0.3, 0.0, 0.0]
    g = gfp.Grid(16, 8, 256)
    g.set_phases(lam, mu)
    g.set_tiles(gfp.MIXED, [2, 8, zcols])
    r = g.solve(gfp.scheme("AFB_R", "PCD", "MIXED"), E, 1e-9, 20000)
    assert r.converged and r.residual < 1e-9
    eps = g.strain()
    r64 = g.solve(gfp.scheme("AFB_R", "PCD", "FP64"), E, 1e-9, 20000)
    assert r64.converged
    assert _rel(eps, g.strain()) <= 1e-6
    assert _rel(r.sigma_mean, r64.sigma_mean) <= 1e-6


def test_mixed_shuffle_z_pass_matches_oracle(gfp):
    """The TMA-fed 8-column z-pass with warp-shuffle line transforms (square plan 64 = 8 x 8; the
    256 = 16 x 16 plan is checked against the FP64 GPU solve above) against the FP64 oracle, with a
    ragged k1 range (13 columns: a full and a partial tile)."""
    shape = (24, 16, 64)
    n1, n2, n3 = shape
    lam, mu = M.random_spheres(shape, vf=0.25, rmin=2.0, rmax=4.0, contrast=20.0, seed=n3)
    E = [0.002, 0.0, -0.001, 0.0, 0.004, 0.0]
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    g.set_tiles(gfp.MIXED, [2, 4, -8])
    r = g.solve(gfp.scheme("AFB_R", "PCD", "MIXED"), E, 1e-8, 20000)
    assert r.converged and r.residual < 1e-8
    ref = O.solve(lam, mu, "AFB_R", E, tol=1e-8, maxit=20000, disc="PCD")
    assert _rel(r.sigma_mean, ref.sigma_mean) <= 1e-6
    assert _rel(g.strain(), ref.eps) <= 1e-6
