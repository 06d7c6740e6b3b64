"""The paper's 1D experiments (Sec. 2.1, 3.2, 3.3, 4) on n x 1 x 1 grids through the 3D GPU path.

X1: smooth matrix-inclusion profile (eq. FiePhaIncMat, eps/l = 1/100 and 1/50) against the closed form of
    Sec. 2.1, which the finite-difference schemes reproduce at the nodes for any profile (the 1D stress is
    uniform, so E_i = S_i E_bar / <S>).
X4: Algorithm T (nodes) against Algorithm P (cell centres) on the sharp inclusion at n = 32: identical
    iterates (the half-cell phases cancel, Sec. 3.2), element by element against the oracle.
X5: Algorithm D-1D (polarization form, s^2 weights, m = n/2) against a direct solve of its own discrete
    system E = E_bar + F^+ diag(-S_m / C_H) F^- (C - C_H) E, assembled with numpy's FFT and the closed
    form S_m(omega / n) of the 1D alias sum.
Lengths: 2^a 3^b (the GPU's transform lengths) near the paper's n = 10, 50, 90.
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


def _bar(C):
    n = C.size
    return np.zeros((1, 1, n)), (0.5 * C).reshape(1, 1, n)


@pytest.mark.parametrize("op", ["F", "CD", "HC", "AFB_R"])
@pytest.mark.parametrize("eps_l", [0.01, 0.02])
def test_x1_smooth_profile_nodal_closed_form(gfp, op, eps_l):
    # CD's checkerboard mode is left uncorrected on even grids (Gamma := 0 where sin vanishes): odd lengths
    for n in ((27, 81) if op == "CD" else (16, 48, 96)):
        nu = M.phase_profile(n, n * 0.25, n * 0.75, eps_l * n, 0.0)  # lengths in voxels (h = l / n)
        C = 1.0 + 99.0 * nu
        S = 1.0 / C
        E_ref = S / S.mean()
        lam, mu = _bar(C)
        r, eps = gfp.solve(lam, mu, op, [1.0, 0, 0, 0, 0, 0], tol=1e-12, maxit=20000)
        assert r.converged
        np.testing.assert_allclose(eps[0, 0, 0], E_ref, rtol=1e-9)


@pytest.mark.parametrize("op", ["F", "HC", "AFB_R"])
def test_x4_algorithm_t_equals_algorithm_p_32(gfp, op):
    n = 32
    nu = M.phase_profile(n, n * 0.25, n * 0.75, 0.0, 0.5)  # cell centres never hit an interface
    C = 1.0 + 99.0 * nu
    lam, mu = _bar(C)
    E = [1.0, 0, 0, 0, 0, 0]
    rt, et = gfp.solve(lam, mu, op, E, tol=1e-12, maxit=20000, disc="TD")
    rp, ep = gfp.solve(lam, mu, op, E, tol=1e-12, maxit=20000, disc="PCD")
    assert rt.iters == rp.iters
    np.testing.assert_array_equal(et, ep)
    ref = O.solve(lam, mu, op, E, tol=1e-12, maxit=20000, disc="PCD")
    assert rp.iters == ref.iters
    assert np.linalg.norm(ep - ref.eps) <= 1e-10 * np.linalg.norm(ref.eps)


@pytest.mark.parametrize("n", [12, 48, 96])
def test_x5_dgo_1d_equals_direct_solve(gfp, n):
    rng = np.random.default_rng(n)
    nu = M.phase_profile(n, n * 0.25, n * 0.75, 0.0, 0.5)
    C = (1.0 + 99.0 * nu) * np.exp(0.05 * rng.standard_normal(n))
    lam, mu = _bar(C)
    r, eps = gfp.solve(lam, mu, "DGO", [1.0, 0, 0, 0, 0, 0], tol=1e-13, maxit=20000, disc="PCD")
    assert r.converged
    C_H = 0.5 * (C.min() + C.max())
    m = n // 2
    w = np.arange(n)
    Sm = np.array([sum(np.sinc(nuv + x / n) ** 2 for nuv in range(-m, m)) if x else 0.0 for x in w])
    Op = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Op[:, j] = np.fft.ifft(-Sm / C_H * np.fft.fft((C - C_H) * e)).real
    E_direct = np.linalg.solve(np.eye(n) - Op, np.ones(n))
    np.testing.assert_allclose(eps[0, 0, 0], E_direct, rtol=1e-9)
