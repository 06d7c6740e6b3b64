"""Eigenstrain generalization (end of Sec. 6: T = C[E - E_*], T^(0) = C_i[E_bar - E_*i]) on the GPU,
through the C ABI, against the FP64 oracle and the laminate closed form."""
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
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def _eigenstrain(shape, seed, scale=0.01):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-scale, scale, size=(6,) + shape)


@pytest.mark.parametrize("op", ["F", "AFB_R", "ACD"])
@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 9, 12), (32, 32, 32)])
def test_fixed_iterations_match_oracle(gfp, op, shape):
    """Four iterations from E_bar with a voxelwise random eigenstrain, element by element (FP64)."""
    n3, n2, n1 = shape
    lam, mu = M.random_field(n1, n2, n3, seed=17)
    es = _eigenstrain(shape, 3)
    E = [0.002, -0.001, 0.003, 0.0, 0.001, 0.002]
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    g.set_eigenstrain(es)
    r = g.solve(gfp.scheme(op, "PCD", "FP64"), E, 0.0, 4)
    ref = O.solve(lam, mu, op, E, max_iters_exact=4, disc="PCD", estar=es)
    assert _rel(g.strain(), ref.eps) <= REL
    assert _rel(r.sigma_mean, ref.sigma_mean) <= REL
    g.close()


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_converged_solution_matches_oracle(gfp, prec):
    lam, mu = M.random_spheres(24, vf=0.2, rmin=3.0, rmax=5.0, contrast=20.0, seed=2)
    es = _eigenstrain((24, 24, 24), 5)
    E = [0.0, 0.0, 0.0, 0.0, 0.0, 0.004]
    g = gfp.Grid(24, 24, 24)
    g.set_phases(lam, mu)
    g.set_eigenstrain(es)
    r = g.solve(gfp.scheme("AFB_R", "PCD", prec), E, 1e-9, 20000)
    ref = O.solve(lam, mu, "AFB_R", E, tol=1e-11, maxit=20000, disc="PCD", estar=es)
    assert r.converged and ref.converged
    tol = 1e-7 if prec == "FP64" else 1e-6
    assert _rel(g.strain(), ref.eps) <= tol
    assert _rel(r.sigma_mean, ref.sigma_mean) <= tol
    # removing the eigenstrain gives back the stiffness-only solution
    g.set_eigenstrain(None)
    r0 = g.solve(gfp.scheme("AFB_R", "PCD", prec), E, 1e-9, 20000)
    ref0 = O.solve(lam, mu, "AFB_R", E, tol=1e-11, maxit=20000, disc="PCD")
    assert _rel(r0.sigma_mean, ref0.sigma_mean) <= tol
    g.close()


def test_laminate_with_eigenstrain_closed_form(gfp):
    """Laminate along x1 with layer-wise eigenstrain: the tractions sigma_11, sigma_12, sigma_13 on the
    layer planes are uniform, which fixes the mean stress in closed form."""
    n1 = 64
    lam, mu = M.random_laminate(n1, 32, 32, seed=9)
    l1, m1 = lam[0, 0], mu[0, 0]
    es1 = _eigenstrain((n1,), 4)
    es = np.broadcast_to(es1[:, None, None, :], (6, 32, 32, n1)).copy()
    E = np.array([0.004, -0.002, 0.003, 0.001, -0.002, 0.005])
    g = gfp.Grid(n1, 32, 32)
    g.set_phases(lam, mu)
    g.set_eigenstrain(es)
    r = g.solve(gfp.scheme("AFB_R", "PCD", "FP64"), E, 1e-12, 5000)
    assert r.converged
    M_ = l1 + 2 * m1
    tr_s = es1[0] + es1[1] + es1[2]
    a = l1 * (E[1] + E[2] - tr_s) - 2 * m1 * es1[0]
    s11 = (E[0] + np.mean(a / M_)) / np.mean(1.0 / M_)
    e11 = (s11 - a) / M_
    s12 = (E[5] - np.mean(es1[5])) / np.mean(1.0 / (2 * m1))
    s13 = (E[4] - np.mean(es1[4])) / np.mean(1.0 / (2 * m1))
    tr = e11 + E[1] + E[2] - tr_s
    s22 = np.mean(l1 * tr + 2 * m1 * (E[1] - es1[1]))
    s33 = np.mean(l1 * tr + 2 * m1 * (E[2] - es1[2]))
    s23 = np.mean(2 * m1 * (E[3] - es1[3]))
    np.testing.assert_allclose(r.sigma_mean, [s11, s22, s33, s23, s13, s12], rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(g.strain()[0], np.broadcast_to(e11, (32, 32, n1)), rtol=1e-8, atol=1e-13)
    g.close()


def test_unsupported_with_eigenstrain(gfp):
    lam, mu = M.random_field(8, 8, 8, seed=1)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    g.set_eigenstrain(_eigenstrain((8, 8, 8), 1))
    with pytest.raises(gfp.GfpError) as e:
        g.effective_stiffness(gfp.scheme("AFB_R", "PCD", "FP64"), 1e-8, 100)
    assert e.value.code == -8
    with pytest.raises(ValueError):
        g.set_eigenstrain(np.zeros((6, 8, 8, 7)))
    g.close()


def test_eigenstrain_from_device_memory(gfp):
    """The eigenstrain given as a CUDA tensor (device copy) gives the same solve as from host memory."""
    torch = pytest.importorskip("torch")
    lam, mu = M.random_field(8, 8, 8, seed=4)
    es = _eigenstrain((8, 8, 8), 6)
    E = [0.001, 0.0, -0.002, 0.0, 0.0, 0.003]
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    g.set_eigenstrain(es)
    r_host = g.solve(gfp.scheme("AFB_R", "PCD", "FP64"), E, 1e-11, 5000)
    eps_host = g.strain()
    g.set_eigenstrain(torch.from_numpy(es).cuda())
    r_dev = g.solve(gfp.scheme("AFB_R", "PCD", "FP64"), E, 1e-11, 5000)
    assert r_host.iters == r_dev.iters
    np.testing.assert_array_equal(g.strain(), eps_host)
    g.close()
