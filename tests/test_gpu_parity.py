"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances: FP64 strain relative L2 error <= 1e-10 and identical iteration counts; mean stress
relative error <= 1e-10.
"""
import os

import numpy as np
import pytest

from oracle import gfp_oracle as O
from paper_2009_03762_gb300 import microstructure as M

pytestmark = pytest.mark.gpu

FDD = ("F", "CD", "ACD", "HC", "AHC", "AFB_R")
REL = 1e-10


@pytest.fixture(scope="module")
def gfp():
    from paper_2009_03762_gb300 import gfp as G
    G.lib()
    return G


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _compare(gfp, lam, mu, op, E, tol, maxit, **kw):
    r, eps = gfp.solve(lam, mu, op, E, tol=tol, maxit=maxit, **kw)
    ref = O.solve(lam, mu, op, E, tol=tol, maxit=maxit)
    assert r.iters == ref.iters, (r.iters, ref.iters, r.residual, ref.residual)
    assert _rel(eps, ref.eps) <= REL, _rel(eps, ref.eps)
    assert _rel(r.sigma_mean, ref.sigma_mean) <= REL
    assert abs(r.residual - ref.residual) <= 1e-6 * max(ref.residual, 1e-30) + 1e-15
    return r, ref


@pytest.mark.parametrize("op", FDD)
def test_homogeneous_one_iteration(gfp, op):
    n = 8
    lam = np.full((n, n, n), 2.0)
    mu = np.full((n, n, n), 0.7)
    E = [0.01, -0.003, 0.002, 0.001, 0.0, 0.004]
    r, eps = gfp.solve(lam, mu, op, E, tol=1e-12, maxit=10, ref=(1.0, 1.0))
    assert r.iters == 1 and r.converged
    np.testing.assert_allclose(eps, np.array(E)[:, None, None, None] * np.ones((6, n, n, n)), atol=1e-15)


@pytest.mark.parametrize("op", FDD)
@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 6, 9), (16, 4, 18)])
def test_parity_random_field(gfp, op, shape):
    n3, n2, n1 = shape
    lam, mu = M.random_field(n1, n2, n3, seed=3)
    _compare(gfp, lam, mu, op, [0.01, 0.002, -0.004, 0.003, 0.0, -0.001], 1e-9, 500)


@pytest.mark.parametrize("op", FDD)
def test_parity_fixed_iterations_ragged(gfp, op):
    """Exactly K iterations (tol = 0) on a 24 x 6 x 27 grid (radix 3 and ragged k1 tiles)."""
    lam, mu = M.random_field(24, 6, 27, seed=9)
    E = [0.0, 0.0, 0.0, 0.0, 0.0, 0.01]
    r, eps = gfp.solve(lam, mu, op, E, tol=0.0, maxit=7)
    ref = O.solve(lam, mu, op, E, max_iters_exact=7)
    assert r.iters == 7 and not r.converged
    assert _rel(eps, ref.eps) <= REL


def test_config_plain_basic_scheme_32(gfp):
    """32^3 sharp cube (edge 16), E = 1 / 10, nu = 0.3, C_H = mean of extremes, E_xx = 0.01,
    TD plain Fourier scheme, stop at eta < 1e-8; against the oracle's stored solution
    (tests/golden/make_c1.py, which calls only the oracle)."""
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "c1_plain_basic_32.npz"))
    lam, mu = M.sharp_cube(32, 16, 1.0, 10.0, 0.3)
    r, eps = gfp.solve(lam, mu, "F", [0.01, 0, 0, 0, 0, 0], tol=1e-8, maxit=20000)
    assert r.converged and r.iters == int(gold["iters"])
    e = eps.reshape(6, -1)
    assert abs(np.linalg.norm(e) - float(gold["eps_norm"])) <= REL * float(gold["eps_norm"])
    diff = e[:, gold["sample_idx"]] - gold["eps_samples"]
    assert np.abs(diff).max() <= REL * float(gold["eps_norm"]) / np.sqrt(e.shape[1])
    assert _rel(r.sigma_mean, gold["sigma_mean"]) <= REL


@pytest.mark.parametrize("op", ["AFB_R", "ACD", "CD"])
def test_config_smooth_cube_small(gfp, op):
    """Smooth log-moduli tanh cube (width 2 voxels), contrast 1e3, at 16^3 (parity size of the 128^3 case)."""
    lam, mu = M.smooth_cube(16, 8, 1e3, width=2.0)
    _compare(gfp, lam, mu, op, [0, 0, 0, 0.5, 0, 0], 1e-10, 5000)


@pytest.mark.parametrize("op", ["F", "HC", "AFB_R"])
def test_laminate_closed_form_on_gpu(gfp, op):
    lam, mu = M.random_laminate(16, 8, 8, seed=5)
    E = np.array([0.01, -0.004, 0.007, 0.003, -0.002, 0.005])
    r, eps = gfp.solve(lam, mu, op, E, tol=1e-12, maxit=3000)
    l1, m1 = lam[0, 0], mu[0, 0]
    Mm = l1 + 2 * m1
    s11 = (E[0] + np.mean(l1 / Mm) * (E[1] + E[2])) / np.mean(1 / Mm)
    s12 = E[5] / np.mean(1 / (2 * m1))
    assert r.converged
    np.testing.assert_allclose([r.sigma_mean[0], r.sigma_mean[5]], [s11, s12], rtol=1e-9)


@pytest.mark.parametrize("op", ["F", "HC", "AFB_R"])
def test_1d_matrix_inclusion_matches_paper_closed_form(gfp, op):
    """1D matrix-inclusion example of Sec. 4 on n x 1 x 1 grids (n = 18, 54, 162): the nodal strain of
    the closed form of Sec. 2.1 (tests/golden/mi1d_sharp.txt), C_I/C_M = 100 as lambda = 0, mu = C/2."""
    rows = np.loadtxt(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mi1d_sharp.txt"))
    for n in (18, 54, 162):
        sel = rows[rows[:, 0] == n]
        nu, E_ref = sel[:, 2], sel[:, 3]
        C = 1.0 + 99.0 * nu
        lam = np.zeros((1, 1, n))
        mu = (0.5 * C).reshape(1, 1, n)
        r, eps = gfp.solve(lam, mu, op, [1.0, 0, 0, 0, 0, 0], tol=1e-11, maxit=5000)
        assert r.converged
        np.testing.assert_allclose(eps[0, 0, 0], E_ref, rtol=1e-9)


def test_full_size_iterations_match_oracle_128(gfp):
    """128^3 smooth cube (config size): three iterations element by element against the oracle."""
    lam, mu = M.smooth_cube(128, 64, 10.0, width=2.0)
    E = [0, 0, 0, 0, 0, 0.5]
    r, eps = gfp.solve(lam, mu, "AFB_R", E, tol=0.0, maxit=3)
    ref = O.solve(lam, mu, "AFB_R", E, max_iters_exact=3)
    assert _rel(eps, ref.eps) <= REL


def test_deterministic_and_resume(gfp):
    lam, mu = M.random_field(16, 16, 16, seed=1)
    E = [0.01, 0, 0, 0, 0, 0]
    sch = gfp.scheme("AFB_R")
    g = gfp.Grid(16, 16, 16)
    g.set_phases(lam, mu)
    a = g.solve(sch, E, 1e-10, 500)
    ea = g.strain()
    b = g.solve(sch, E, 1e-10, 500)
    eb = g.strain()
    assert a.iters == b.iters and np.array_equal(ea, eb)
    # interrupt after 5 iterations, checkpoint, resume
    g.solve(sch, E, 0.0, 5)
    state, it = g.get_state()
    assert it == 5
    g2 = gfp.Grid(16, 16, 16)
    g2.set_phases(lam, mu)
    g2.set_state(state, it)
    c = g2.solve(sch, E, 1e-10, 500)
    assert c.iters == a.iters
    assert np.array_equal(g2.strain(), ea)


def test_launch_count(gfp):
    """gfp_result.launches counts the kernels a solve launched: tol = 0 runs exactly K FP64 iterations of
    five kernels after the strain fill, then two for the compensated mean stress; the mixed solve adds at
    least four per outer pass and two per refinement."""
    lam, mu = M.random_field(16, 16, 16, seed=3)
    g = gfp.Grid(16, 16, 16)
    g.set_phases(lam, mu)
    r = g.solve(gfp.scheme("AFB_R", "PCD", "FP64"), [0.01, 0, 0, 0, 0, 0], 0.0, 37)
    assert r.iters == 37 and r.launches == 1 + 5 * 37 + 2
    rm = g.solve(gfp.scheme("AFB_R", "PCD", "MIXED"), [0.01, 0, 0, 0, 0, 0], 1e-9, 5000)
    assert rm.converged and rm.outer >= 2
    assert rm.launches >= 1 + 4 * rm.outer + 2 * (rm.outer - 1) + 5 * rm.iters
    g.close()


def test_error_statuses(gfp):
    lam, mu = M.random_field(8, 8, 8, seed=2)
    g = gfp.Grid(8, 8, 8)
    bad = mu.copy()
    bad[0, 0, 0] = -1.0
    with pytest.raises(gfp.GfpError) as e:
        g.set_phases(lam, bad)
    assert e.value.code == -1
    g.set_phases(lam, mu)
    r = g.solve(gfp.scheme("AFB_R"), [0.01, 0, 0, 0, 0, 0], 1e-14, 2)
    assert r.status == -4 and r.iters == 2
    # the paper's 3D reference (C_H = C_I) with a soft inclusion violates 0 < c < 2 c_H and grows
    lam2, mu2 = M.sharp_cube(16, 8, 1.0, 1e-3)
    g2 = gfp.Grid(16, 16, 16)
    li, mi = M.lame(1e-3, 0.3)
    g2.set_phases(lam2, mu2, ref=(float(li), float(mi)))
    r2 = g2.solve(gfp.scheme("F"), [0.01, 0, 0, 0, 0, 0], 1e-8, 3000)
    assert r2.status == -5


@pytest.mark.parametrize("op", ["AFB_R", "F"])
def test_effective_stiffness_matches_oracle(gfp, op):
    lam, mu = M.random_field(8, 8, 8, seed=4)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    C, its, rc = g.effective_stiffness(gfp.scheme(op), 1e-11, 2000)
    Cref, itref, _ = O.effective_stiffness(lam, mu, op, tol=1e-11, maxit=2000)
    assert rc == 0 and its == itref
    np.testing.assert_allclose(C, Cref, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(C, C.T, rtol=1e-7, atol=1e-9)


def test_gradient_matches_oracle_closed_form_and_fd(gfp):
    lam, mu = M.random_field(8, 8, 8, seed=6)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    dl, dm = g.grad(gfp.scheme("AFB_R"), 0, 0, 1e-13, 5000)
    ref = O.default_reference(lam, mu)
    rI = O.solve(lam, mu, "AFB_R", [1, 0, 0, 0, 0, 0], tol=1e-13, maxit=5000, ref=ref)
    gl, gm = O.gradient_closed_form(rI.eps, rI.eps)
    np.testing.assert_allclose(dl, gl, rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(dm, gm, rtol=1e-8, atol=1e-14)
    vox = [3, 100, 311]
    fl, fm = O.gradient_fd(lam, mu, "AFB_R", 0, 0, vox, rel_step=1e-5, tol=1e-13)
    np.testing.assert_allclose(dl.ravel()[vox], fl, rtol=1e-5)
    np.testing.assert_allclose(dm.ravel()[vox], fm, rtol=1e-5)


@pytest.mark.parametrize("shape", [(32, 64, 96), (96, 32, 64), (64, 96, 32), (128, 32, 192), (192, 128, 32),
                                   (32, 192, 128), (256, 16, 32), (32, 256, 16), (16, 32, 256), (512, 8, 16),
                                   (16, 512, 8), (8, 16, 512)])
@pytest.mark.parametrize("op", ["F", "AFB_R"])
def test_parity_register_fft_sizes(gfp, shape, op):
    """Every length with a compile-time FFT plan, on every axis: three iterations element by element."""
    n3, n2, n1 = shape
    lam, mu = M.random_field(n1, n2, n3, seed=13)
    E = [0.003, -0.002, 0.004, 0.001, 0.002, 0.005]
    r, eps = gfp.solve(lam, mu, op, E, tol=0.0, maxit=3)
    ref = O.solve(lam, mu, op, E, max_iters_exact=3)
    assert _rel(eps, ref.eps) <= REL
    assert _rel(r.sigma_mean, ref.sigma_mean) <= REL


@pytest.mark.parametrize("prec,op", [("FP64", "F"), ("MIXED", "AFB_R")])
def test_autotuned_tiles_keep_parity(gfp, prec, op, tmp_path):
    """The tile autotuner changes launch shapes only: results stay at oracle parity; the cache is reused."""
    lam, mu = M.random_spheres(32, vf=0.2, rmin=3.0, rmax=5.0, contrast=20.0, seed=4)
    g = gfp.Grid(32, 32, 32)
    g.set_phases(lam, mu)
    sch = gfp.scheme(op, "PCD", prec)
    cache = str(tmp_path / "tiles.json")
    tiles = g.tune(sch, iters=2, cache=cache)
    assert len(tiles) == 3 and g.tune(sch, cache=cache) == tiles
    E = [0.0, 0.0, 0.0, 0.0, 0.0, 0.5]
    if prec == "FP64":
        r = g.solve(sch, E, 0.0, 5)
        ref = O.solve(lam, mu, op, E, max_iters_exact=5, disc="PCD")
        assert _rel(g.strain(), ref.eps) <= REL
    else:
        r = g.solve(sch, E, 1e-8, 5000)
        ref = O.solve(lam, mu, op, E, tol=1e-9, maxit=5000, disc="PCD")
        assert r.converged and _rel(r.sigma_mean, ref.sigma_mean) <= 1e-6


@pytest.mark.parametrize("op,prec", [("AFB_R", "FP64"), ("F", "FP64"), ("DGO", "FP64"), ("AFB_R", "MIXED")])
def test_zero_load_degenerate(gfp, op, prec):
    """Zero mean strain, no eigenstrain: the exact solution eps = 0 after the first iteration, as the oracle."""
    lam, mu = M.random_field(8, 8, 8, seed=3)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    r = g.solve(gfp.scheme(op, "PCD", prec), [0.0] * 6, 1e-8, 50)
    assert r.converged
    assert np.all(g.strain() == 0.0) and np.all(np.asarray(r.sigma_mean) == 0.0)
    if prec == "FP64":
        ref = O.solve(lam, mu, op, [0.0] * 6, tol=1e-8, maxit=50, disc="PCD")
        assert r.iters == ref.iters == 1
    g.close()
