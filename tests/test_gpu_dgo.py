"""Discrete Green operator (Algorithm D-3D, polarization form, s^2 weights) on the GPU against the
FP64 oracle, element by element."""
import numpy as np
import pytest

from oracle import gfp_oracle as O
from paper_2009_03762_gb300 import microstructure as M

pytestmark = pytest.mark.gpu
REL = 1e-10


@pytest.fixture(scope="module")
def gfp():
    from paper_2009_03762_gb300 import gfp as G
    G.lib()
    return G


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _solve(gfp, lam, mu, E, tol, maxit, m=0):
    n3, n2, n1 = lam.shape
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    r = g.solve(gfp.scheme("DGO", "PCD", dgo_m=m), E, tol, maxit)
    return r, g.strain()


def test_dgo_homogeneous_one_iteration(gfp):
    lam = np.full((8, 8, 8), 2.0)
    mu = np.full((8, 8, 8), 0.9)
    E = [0.01, 0.0, -0.003, 0.002, 0.0, 0.001]
    n = 8
    g = gfp.Grid(n, n, n)
    g.set_phases(lam, mu, ref=(1.0, 0.5))
    r = g.solve(gfp.scheme("DGO", "PCD"), E, 1e-12, 10)
    assert r.iters == 1 and r.converged
    np.testing.assert_allclose(g.strain(), np.array(E)[:, None, None, None] * np.ones((6, n, n, n)), atol=1e-15)


@pytest.mark.parametrize("shape,m", [((8, 8, 8), 0), ((6, 8, 12), 0), ((12, 12, 12), 2), ((16, 6, 9), 0)])
def test_dgo_parity_random_field(gfp, shape, m):
    n3, n2, n1 = shape
    lam, mu = M.random_field(n1, n2, n3, seed=21)
    E = [0.01, -0.002, 0.003, 0.0, 0.002, -0.001]
    r, eps = _solve(gfp, lam, mu, E, 1e-10, 2000, m)
    ref = O.solve(lam, mu, "DGO", E, tol=1e-10, maxit=2000, dgo_m=(m or None))
    assert r.iters == ref.iters, (r.iters, ref.iters)
    assert _rel(eps, ref.eps) <= REL
    assert _rel(r.sigma_mean, ref.sigma_mean) <= REL


def test_dgo_smooth_cube_contrast(gfp):
    lam, mu = M.smooth_cube(16, 8, 10.0, width=2.0, sampling="PCD")
    E = [0.0, 0.0, 0.0, 0.0, 0.0, 0.5]
    r, eps = _solve(gfp, lam, mu, E, 1e-10, 3000)
    ref = O.solve(lam, mu, "DGO", E, tol=1e-10, maxit=3000)
    assert r.converged and r.iters == ref.iters
    assert _rel(eps, ref.eps) <= REL


def test_dgo_fixed_iterations_register_fft_size(gfp):
    """32^3 (register-FFT kernels): exactly 4 iterations element by element (m = 2 keeps the oracle quick)."""
    lam, mu = M.sharp_cube(32, 16, 1.0, 10.0)
    E = [0.01, 0, 0, 0, 0, 0]
    r, eps = _solve(gfp, lam, mu, E, 0.0, 4, m=2)
    ref = O.solve(lam, mu, "DGO", E, max_iters_exact=4, dgo_m=2)
    assert r.iters == 4
    assert _rel(eps, ref.eps) <= REL


VARIANTS = [(p, f, r) for p in (1, 2) for f in ("polarization", "stress") for r in ("printed", "symmetric")]


@pytest.mark.parametrize("power,form,rng", VARIANTS)
def test_dgo_variants_fixed_iterations(gfp, power, form, rng):
    """Every weight / update-form / alias-range variant of the discrete Green operator, 40 iterations on a
    non-cubic random field element by element (the printed s weights grow there in the stress form; the
    iterates still agree), with the residual history."""
    n1, n2, n3 = 8, 6, 4
    lam, mu = M.random_field(n1, n2, n3, seed=5)
    E = [0.01, 0.0, 0.0, 0.0, 0.003, 0.0]
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    sch = gfp.scheme("DGO", "PCD", dgo_power=power, dgo_form=form, dgo_range=rng)
    r = g.solve(sch, E, 0.0, 40, history=True)
    ref = O.solve(lam, mu, "DGO", E, max_iters_exact=40, dgo_form=form, dgo_power=power, dgo_range=rng)
    assert r.iters == 40 == ref.iters
    assert _rel(g.strain(), ref.eps) <= REL
    np.testing.assert_allclose(r.history, ref.history, rtol=1e-8)


@pytest.mark.parametrize("power,rng", [(1, "printed"), (1, "symmetric"), (2, "symmetric")])
def test_dgo_variants_converged_iteration_count(gfp, power, rng):
    """Polarization-form variants that converge on a 6^3 random field: the same iteration count to 1e-10."""
    lam, mu = M.random_field(6, 6, 6, seed=3)
    E = [0.01, 0.0, 0.0, 0.0, 0.003, 0.0]
    g = gfp.Grid(6, 6, 6)
    g.set_phases(lam, mu)
    r = g.solve(gfp.scheme("DGO", "PCD", dgo_power=power, dgo_range=rng), E, 1e-10, 1000)
    ref = O.solve(lam, mu, "DGO", E, tol=1e-10, maxit=1000, dgo_power=power, dgo_range=rng)
    assert r.converged and ref.converged and r.iters == ref.iters
    assert _rel(g.strain(), ref.eps) <= REL
    assert _rel(r.sigma_mean, ref.sigma_mean) <= REL
