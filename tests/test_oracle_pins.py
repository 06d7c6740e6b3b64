"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: closed forms, textbook
operators, brute-force real-space assemblies, library transforms and invariants.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import gfp_oracle as O
from paper_2009_03762_gb300 import microstructure as M

HERE = os.path.dirname(os.path.abspath(__file__))
FDD = ("F", "CD", "ACD", "HC", "AHC", "AFB_R", "R")


# ----------------------------------------------------------------------------- transforms
@pytest.mark.parametrize("disc", ["TD", "PCD"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 9])
def test_dft_cardinality_and_unitarity(n, disc):
    """F^+ and F^- are inverse (cardinality, App. A/B) and unitary."""
    Fp, Fm = O.dft_matrices(n, 0.7, disc)
    np.testing.assert_allclose(Fp.T @ Fm, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(Fm @ Fm.conj().T, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("disc", ["TD", "PCD"])
def test_forward3_matches_numpy_fft(disc):
    """The Rayleigh-product transform equals numpy's FFT up to the paper's ordering, scale and phase."""
    rng = np.random.default_rng(0)
    n3, n2, n1 = 5, 6, 4
    f = rng.standard_normal((n3, n2, n1))
    h = 1.0
    mats = [O.dft_matrices(nr, h, disc) for nr in (n1, n2, n3)]
    fc = O.forward3(f, mats)
    ref = np.fft.fftshift(np.fft.fftn(f)) / np.sqrt(f.size)
    if disc == "PCD":   # x_i^c = (i - 1/2) h adds e^{-i k h / 2} per axis
        for ax, nr in zip((2, 1, 0), (n1, n2, n3)):
            k = 2 * np.pi * O.kappa(nr) / (nr * h)
            sh = [1, 1, 1]
            sh[ax] = nr
            ref = ref * np.exp(-0.5j * k * h).reshape(sh)
    np.testing.assert_allclose(fc, ref, atol=1e-12)
    np.testing.assert_allclose(O.inverse3(fc, mats).real, f, atol=1e-12)
    # Parseval
    assert abs(np.sum(np.abs(fc) ** 2) - np.sum(f ** 2)) < 1e-10


# ----------------------------------------------------------------------------- symbols
def _plane_wave(qvec, pts):
    """e^{q . x} at points pts (..., 3) for a wave vector of imaginary wave numbers (x1, x2, x3)."""
    return np.exp(pts[..., 0] * qvec[0] + pts[..., 1] * qvec[1] + pts[..., 2] * qvec[2])


def _stencil_value(kind, r, qvec, x, h):
    """Evaluate a difference operator of the paper on a plane wave directly from its definition.

    kinds: FD, BD, CD, hC (eq. AppDifFinDFStn1D along axis r); AFD, ABD, ACD, AhC: the 3D
    averages over the other two axes (eqs. FBDiff2D, BDDiff2D, CDDiff2D, hCDDiff2D generalised
    to 3D as in eq. FreDifFinFBDF3D).
    """
    e = np.eye(3)
    f = lambda p: _plane_wave(qvec, np.asarray(p, float))
    def d1(kind1, p):
        if kind1 == "FD":
            return (f(p + h * e[r]) - f(p)) / h
        if kind1 == "BD":
            return (f(p) - f(p - h * e[r])) / h
        if kind1 == "CD":
            return (f(p + h * e[r]) - f(p - h * e[r])) / (2 * h)
        if kind1 == "hC":
            return (f(p + 0.5 * h * e[r]) - f(p - 0.5 * h * e[r])) / h
    if kind in ("FD", "BD", "CD", "hC"):
        return d1(kind, x)
    s, t = (r + 1) % 3, (r + 2) % 3
    if kind == "AFD":
        offs = [a * e[s] + b * e[t] for a in (0, 1) for b in (0, 1)]
        return np.mean([d1("FD", x + h * o) for o in offs])
    if kind == "ABD":
        offs = [a * e[s] + b * e[t] for a in (0, -1) for b in (0, -1)]
        return np.mean([d1("BD", x + h * o) for o in offs])
    if kind == "ACD":
        offs = [a * e[s] + b * e[t] for a in (-1, 1) for b in (-1, 1)]
        return np.mean([d1("CD", x + h * o) for o in offs])
    if kind == "AhC":
        offs = [a * e[s] + b * e[t] for a in (-0.5, 0.5) for b in (-0.5, 0.5)]
        return np.mean([d1("hC", x + h * o) for o in offs])


@pytest.mark.parametrize("scheme,a_kind,b_kind", [
    ("F", None, None), ("CD", "CD", None), ("HC", "hC", None), ("ACD", "ACD", None),
    ("AHC", "AhC", None), ("AFB_R", "AFD", "AhC")])
def test_wave_vectors_are_stencil_symbols(scheme, a_kind, b_kind):
    """q^a (and q^b) reproduce the real-space stencils applied to plane waves (modal forms)."""
    n3, n2, n1 = 5, 6, 4
    h = 1.3
    qa, qb = O.wave_vectors(scheme, n3, n2, n1, h)
    x0 = np.array([0.3, -1.1, 2.0])
    ns = (n1, n2, n3)
    for i3, i2, i1 in itertools.product(range(n3), range(n2), range(n1)):
        idx = (i1, i2, i3)
        qv = np.array([1j * 2 * np.pi * O.kappa(ns[r])[idx[r]] / (ns[r] * h) for r in range(3)])
        f0 = _plane_wave(qv, x0)
        for r in range(3):
            if a_kind is None:
                expect_a = qv[r]
            else:
                expect_a = _stencil_value(a_kind, r, qv, x0, h) / f0
            assert abs(qa[r, i3, i2, i1] - expect_a) < 1e-11
            if b_kind is not None:
                expect_b = _stencil_value(b_kind, r, qv, x0, h) / f0
                assert abs(qb[r, i3, i2, i1] - expect_b) < 1e-11
            else:
                assert abs(qb[r, i3, i2, i1] - np.conj(qa[r, i3, i2, i1])) < 1e-14


def test_conjugate_afd_is_minus_abd():
    """q^{AFD*} = -q^{ABD} (Sec. 5.3 after eq. EffNumWavConWil3D), checked on the ABD stencil."""
    n3, n2, n1 = 4, 5, 6
    qa, _ = O.wave_vectors("AFB_R", n3, n2, n1, 1.0)
    ns = (n1, n2, n3)
    x0 = np.zeros(3)
    for i3, i2, i1 in itertools.product(range(n3), range(n2), range(n1)):
        idx = (i1, i2, i3)
        qv = np.array([1j * 2 * np.pi * O.kappa(ns[r])[idx[r]] / ns[r] for r in range(3)])
        for r in range(3):
            abd = _stencil_value("ABD", r, qv, x0, 1.0)
            assert abs(np.conj(qa[r, i3, i2, i1]) + abd) < 1e-12


def test_willot_qw_equals_qfd_except_limit():
    """q^W = q^FD for mu = 2..n and lim_{mu->1} q^W = q^FD (Sec. 5.3, eq. FreDifFinFBDFR3D)."""
    for n in (6, 8, 11):
        q = O.q_fourier(n, 1.0)
        np.testing.assert_allclose(O.q1d("W", q, 1.0), O.q1d("FD", q, 1.0), atol=1e-13)
    # the limit itself: q h -> -i pi
    t = -np.pi + 1e-6
    qw = np.tanh(0.5j * t) * (np.exp(1j * t) + 1.0)
    assert abs(qw - (np.exp(-1j * np.pi) - 1.0)) < 1e-5
    qa_afb, _ = O.wave_vectors("AFB_R", 6, 6, 6, 1.0)
    qa_r, _ = O.wave_vectors("R", 6, 6, 6, 1.0)
    np.testing.assert_allclose(qa_afb, qa_r, atol=1e-13)


# ----------------------------------------------------------------------------- Green operator
def _C_apply(lam, mu, A):
    return O.stiffness_apply(lam, mu, A)


@pytest.mark.parametrize("scheme", FDD)
def test_gamma_projection_and_idempotence(scheme):
    """Gamma C_H sym(u (x) q^a) = sym(u (x) q^a) and Gamma C_H Gamma = Gamma (from eq. EquMecFunGre3D)."""
    rng = np.random.default_rng(1)
    n3, n2, n1 = 5, 4, 6
    lam_h, mu_h = 1.7, 0.9
    qa, qb = O.wave_vectors(scheme, n3, n2, n1)
    G = O.green(qa, qb, lam_h, mu_h)
    u = rng.standard_normal((3, n3, n2, n1)) + 1j * rng.standard_normal((3, n3, n2, n1))
    eps = O.sym_outer(u, qa)
    live = np.abs(np.sum(qa * qb, axis=0)) > 0
    back = O.gamma_apply(G, qa, qb, _C_apply(lam_h, mu_h, eps))
    np.testing.assert_allclose(back[:, :, live], eps[:, :, live], atol=1e-12)
    A = rng.standard_normal((3, 3, n3, n2, n1)) + 1j * rng.standard_normal((3, 3, n3, n2, n1))
    A = 0.5 * (A + np.swapaxes(A, 0, 1))
    GA = O.gamma_apply(G, qa, qb, A)
    GCGA = O.gamma_apply(G, qa, qb, _C_apply(lam_h, mu_h, GA))
    np.testing.assert_allclose(GCGA, GA, atol=1e-12)
    k0 = (n3 // 2, n2 // 2, n1 // 2)
    assert np.all(GA[(slice(None), slice(None)) + k0] == 0)


@pytest.mark.parametrize("scheme", FDD)
def test_gamma_real_and_even(scheme):
    """The literal complex Gamma of every pairing is real and even in k (interior modes)."""
    n = 7
    lam_h, mu_h = 1.2, 0.8
    qa, qb = O.wave_vectors(scheme, n, n, n)
    G = O.green(qa, qb, lam_h, mu_h)
    mats = []
    for (i, j) in O.VOIGT:
        B = np.zeros((3, 3, n, n, n))
        B[i, j] = 1.0
        B[j, i] = 1.0
        mats.append(O.gamma_apply(G, qa, qb, B))
    mats = np.array(mats)
    assert np.abs(mats.imag).max() < 1e-13
    # kappa -> -kappa is index m+kappa -> m-kappa; for odd n the range is symmetric
    flipped = mats[..., ::-1, ::-1, ::-1]
    np.testing.assert_allclose(mats.real, flipped.real, atol=1e-13)


def test_gamma_fourier_is_textbook_isotropic_operator():
    """For the plain Fourier scheme Gamma equals the isotropic Gamma^0 of Moulinec-Suquet (1998):
    Gamma_khij = (d_ki x_h x_j + d_hi x_k x_j + d_kj x_h x_i + d_hj x_k x_i)/(4 mu |x|^2)
                 - (lam + mu)/(mu (lam + 2 mu)) x_i x_j x_k x_h / |x|^4."""
    n = 5
    lam_h, mu_h = 2.3, 0.7
    qa, qb = O.wave_vectors("F", n, n, n)
    G = O.green(qa, qb, lam_h, mu_h)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3, n, n, n))
    A = 0.5 * (A + np.swapaxes(A, 0, 1))
    got = O.gamma_apply(G, qa, qb, A).real
    xi = (qa / 1j).real
    d = np.eye(3)
    x2 = np.sum(xi * xi, axis=0)
    x2s = np.where(x2 > 0, x2, 1.0)
    c = (lam_h + mu_h) / (mu_h * (lam_h + 2 * mu_h))
    ref = np.zeros_like(got)
    for k, h_, i, j in itertools.product(range(3), repeat=4):
        g = ((d[k, i] * xi[h_] * xi[j] + d[h_, i] * xi[k] * xi[j] + d[k, j] * xi[h_] * xi[i]
              + d[h_, j] * xi[k] * xi[i]) / (4 * mu_h * x2s)
             - c * xi[i] * xi[j] * xi[k] * xi[h_] / x2s ** 2)
        ref[k, h_] += g * A[i, j]
    ref[:, :, x2 == 0] = 0.0
    np.testing.assert_allclose(got, ref, atol=1e-13)


# ----------------------------------------------------------------------------- whole solver
@pytest.mark.parametrize("scheme", FDD + ("DGO",))
def test_homogeneous_medium_converges_in_one_iteration(scheme):
    n = 4
    lam = np.full((n, n, n), 2.5)
    mu = np.full((n, n, n), 1.1)
    E = np.array([0.01, -0.02, 0.005, 0.003, -0.004, 0.002])
    r = O.solve(lam, mu, scheme, E, tol=1e-12, ref=(1.0, 0.5))
    assert r.iters == 1
    np.testing.assert_allclose(r.eps, E[:, None, None, None] * np.ones((1, n, n, n)), atol=1e-15)


def _laminate_closed_form(lam1, mu1, E):
    """Exact mean stress of a laminate along x1 (T constant across the layers, Sec. 2.1, the 1D equilibrium argument
    generalised: sigma_11, sigma_12, sigma_13 uniform; eps_22, eps_33, eps_23 uniform)."""
    E11, E22, E33, E23, E13, E12 = E
    M_ = lam1 + 2 * mu1
    s11 = (E11 + np.mean(lam1 / M_) * (E22 + E33)) / np.mean(1.0 / M_)
    s12 = E12 / np.mean(1.0 / (2 * mu1))
    s13 = E13 / np.mean(1.0 / (2 * mu1))
    e11 = (s11 - lam1 * (E22 + E33)) / M_
    tr = e11 + E22 + E33
    s22 = np.mean(lam1 * tr + 2 * mu1 * E22)
    s33 = np.mean(lam1 * tr + 2 * mu1 * E33)
    s23 = np.mean(2 * mu1 * E23)
    return np.array([s11, s22, s33, s23, s13, s12]), e11


@pytest.mark.parametrize("scheme,n1", [("F", 7), ("F", 8), ("HC", 8), ("AHC", 8), ("AFB_R", 8),
                                      ("R", 6), ("CD", 7), ("ACD", 7), ("DGO", 6)])
def test_laminate_exact_effective_response(scheme, n1):
    lam, mu = M.random_laminate(n1, 3, 4, seed=5)
    E = np.array([0.01, -0.004, 0.007, 0.003, -0.002, 0.005])
    # the DGO's stress form has equilibrium as its fixed point; its polarization form is pinned below
    kw = dict(dgo_form="stress") if scheme == "DGO" else {}
    r = O.solve(lam, mu, scheme, E, tol=1e-12, maxit=3000, **kw)
    assert r.converged
    ref, e11 = _laminate_closed_form(lam[0, 0], mu[0, 0], E)
    np.testing.assert_allclose(r.sigma_mean, ref, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(r.eps[0], np.broadcast_to(e11, r.eps[0].shape), rtol=1e-8, atol=1e-12)


def _laminate_eigenstrain_closed_form(lam1, mu1, es, E):
    """Exact response of a laminate along x1 with a layer-wise eigenstrain es (6, n1), stress
    T = C[E - E_*] (generalization at the end of Sec. 6).  The tractions on the layer planes,
    sigma_11, sigma_12, sigma_13, are uniform; eps_22, eps_33, eps_23 equal their means.
    Returns the 6 mean stresses and the fields eps_11, eps_12 across the layers."""
    E11, E22, E33, E23, E13, E12 = E
    M_ = lam1 + 2 * mu1
    tr_s = es[0] + es[1] + es[2]
    a = lam1 * (E22 + E33 - tr_s) - 2 * mu1 * es[0]          # sigma_11 = M eps_11 + a
    s11 = (E11 + np.mean(a / M_)) / np.mean(1.0 / M_)
    e11 = (s11 - a) / M_
    s12 = (E12 - np.mean(es[5])) / np.mean(1.0 / (2 * mu1))   # sigma_12 = 2 mu (eps_12 - es_12)
    s13 = (E13 - np.mean(es[4])) / np.mean(1.0 / (2 * mu1))
    e12 = s12 / (2 * mu1) + es[5]
    tr = e11 + E22 + E33 - tr_s
    s22 = np.mean(lam1 * tr + 2 * mu1 * (E22 - es[1]))
    s33 = np.mean(lam1 * tr + 2 * mu1 * (E33 - es[2]))
    s23 = np.mean(2 * mu1 * (E23 - es[3]))
    return np.array([s11, s22, s33, s23, s13, s12]), e11, e12


@pytest.mark.parametrize("scheme", ["F", "HC", "AFB_R"])
def test_laminate_with_eigenstrain_closed_form(scheme):
    """Eigenstrain generalization (Sec. 6): a laminate with layer-wise moduli and eigenstrain."""
    n1 = 8
    lam, mu = M.random_laminate(n1, 3, 4, seed=7)
    rng = np.random.Generator(np.random.PCG64(11))
    es1 = rng.uniform(-0.01, 0.01, size=(6, n1))
    es = np.broadcast_to(es1[:, None, None, :], (6, 4, 3, n1)).copy()
    E = np.array([0.004, -0.002, 0.003, 0.001, -0.002, 0.005])
    r = O.solve(lam, mu, scheme, E, tol=1e-12, maxit=3000, estar=es)
    assert r.converged
    ref, e11, e12 = _laminate_eigenstrain_closed_form(lam[0, 0], mu[0, 0], es1, E)
    np.testing.assert_allclose(r.sigma_mean, ref, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(r.eps[0], np.broadcast_to(e11, r.eps[0].shape), rtol=1e-8, atol=1e-13)
    np.testing.assert_allclose(r.eps[5], np.broadcast_to(e12, r.eps[5].shape), rtol=1e-8, atol=1e-13)


def test_uniform_eigenstrain_is_a_shift_of_the_mean_strain():
    """A uniform eigenstrain E0 solves like the mean strain E_bar - E0 shifted by E0:
    eps(E_bar; E_* = E0) = eps(E_bar - E0) + E0, with the same stresses, iterate by iterate."""
    lam, mu = M.random_field(6, 5, 4, seed=3)
    E = np.array([0.01, -0.003, 0.002, 0.004, 0.0, -0.001])
    E0 = np.array([0.002, 0.001, -0.004, 0.0, 0.003, 0.001])
    es = np.broadcast_to(E0[:, None, None, None], (6, 4, 5, 6)).copy()
    for scheme in ("AFB_R", "CD"):
        a = O.solve(lam, mu, scheme, E, estar=es, max_iters_exact=6)
        b = O.solve(lam, mu, scheme, E - E0, max_iters_exact=6)
        np.testing.assert_allclose(a.eps, b.eps + E0[:, None, None, None], rtol=0, atol=1e-14)
        np.testing.assert_allclose(a.sigma_mean, b.sigma_mean, rtol=1e-13, atol=1e-15)


def _sym_grad_spectral(disp, symbols):
    """sym(grad u) with per-axis difference symbols applied by numpy's FFT: symbols[r] is a function of
    (theta1, theta2, theta3) on the FFT grid giving the symbol of the derivative along x_(r+1)."""
    n3, n2, n1 = disp.shape[1:]
    t3, t2, t1 = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(n) for n in (n3, n2, n1)], indexing="ij")
    uh = [np.fft.fftn(disp[i]) for i in range(3)]
    q = [symbols[r](t1, t2, t3) for r in range(3)]
    G = np.empty((3, 3, n3, n2, n1))
    for i in range(3):
        for j in range(3):
            G[i, j] = np.fft.ifftn(q[j] * uh[i]).real       # d u_i / d x_j
    return 0.5 * (G + G.transpose(1, 0, 2, 3, 4))


def _afd_symbols():
    """AFD (eq. FreDifFinFBDF3D): forward difference along r averaged (e^{i theta} + 1)/2 over the
    other two axes."""
    fd = lambda t: np.exp(1j * t) - 1.0
    av = lambda t: 0.5 * (np.exp(1j * t) + 1.0)
    return [lambda t1, t2, t3: fd(t1) * av(t2) * av(t3),
            lambda t1, t2, t3: fd(t2) * av(t3) * av(t1),
            lambda t1, t2, t3: fd(t3) * av(t1) * av(t2)]


def test_displacement_afb_r_reproduces_strain_3d():
    """The displacement u^p = F^+ u_check of Algorithm T with AFB/R: its AFD difference gives back the
    strain fluctuation exactly (any grid), sym(q^AFD (x) u) = eps - E_bar."""
    lam, mu = M.random_field(6, 5, 4, seed=6)
    E = np.array([0.01, -0.004, 0.002, 0.003, -0.002, 0.001])
    r = O.solve(lam, mu, "AFB_R", E, tol=1e-11, maxit=2000)
    S = _sym_grad_spectral(r.disp, _afd_symbols())
    Ef = O.voigt_to_tensor(r.eps) - O.voigt_to_tensor(E)[:, :, None, None, None]
    np.testing.assert_allclose(S, Ef, rtol=0, atol=1e-14)
    assert abs(r.disp.mean()) < 1e-16


@pytest.mark.parametrize("scheme", ["F", "AHC", "ACD"])
def test_displacement_reproduces_strain_odd_grid(scheme):
    """Schemes without the half-voxel phase: on odd grids (no Nyquist mode) sym(q^a (x) u^p) gives back
    the strain fluctuation; q^a = i k (F), i 2 sin(theta/2) cos cos (AHC), i sin(theta) cos cos (ACD)."""
    lam, mu = M.random_field(5, 7, 3, seed=8)
    E = np.array([0.01, -0.004, 0.002, 0.003, -0.002, 0.001])
    r = O.solve(lam, mu, scheme, E, tol=1e-11, maxit=4000)
    if scheme == "F":
        f, a = (lambda t: 1j * t), (lambda t: 1.0)
    elif scheme == "AHC":
        f, a = (lambda t: 2j * np.sin(0.5 * t)), (lambda t: np.cos(0.5 * t))
    else:
        f, a = (lambda t: 1j * np.sin(t)), (lambda t: np.cos(t))
    sym = [lambda t1, t2, t3: f(t1) * a(t2) * a(t3),
           lambda t1, t2, t3: f(t2) * a(t3) * a(t1),
           lambda t1, t2, t3: f(t3) * a(t1) * a(t2)]
    S = _sym_grad_spectral(r.disp, sym)
    Ef = O.voigt_to_tensor(r.eps) - O.voigt_to_tensor(E)[:, :, None, None, None]
    np.testing.assert_allclose(S, Ef, rtol=0, atol=1e-13)


def _load_golden_1d():
    rows = np.loadtxt(os.path.join(HERE, "golden", "mi1d_sharp.txt"))
    out = {}
    for n in (10, 50, 90):
        sel = rows[rows[:, 0] == n]
        out[n] = (sel[:, 2], sel[:, 3])
    return out


@pytest.mark.parametrize("scheme", ["F", "HC", "AHC", "AFB_R", "R"])
def test_1d_matrix_inclusion_matches_paper_closed_form(scheme):
    """1D MI example of Sec. 4 (n = 10, 50, 90): all these wave numbers give the nodal closed form."""
    gold = _load_golden_1d()
    for n, (nu, E_ref) in gold.items():
        C = 1.0 + 99.0 * nu
        lam = np.zeros((1, 1, n))
        mu = (0.5 * C).reshape(1, 1, n)
        r = O.solve(lam, mu, scheme, [1.0, 0, 0, 0, 0, 0], tol=1e-11, maxit=2000)
        assert r.converged
        np.testing.assert_allclose(r.eps[0, 0, 0], E_ref, rtol=1e-10)


def test_td_and_pcd_fdd_give_identical_iterates():
    """Algorithm P on the same sampled moduli equals Algorithm T ("independent of s", Sec. 3.2)."""
    lam, mu = M.random_field(6, 5, 4, seed=2)
    for scheme in ("F", "AFB_R", "ACD"):
        a = O.solve(lam, mu, scheme, [0.01, 0, 0, 0.002, 0, 0], tol=1e-10, disc="TD")
        b = O.solve(lam, mu, scheme, [0.01, 0, 0, 0.002, 0, 0], tol=1e-10, disc="PCD")
        assert a.iters == b.iters
        np.testing.assert_allclose(a.eps, b.eps, atol=1e-13)


# ----------------------------------------------------------------------------- dense real-space solves
def _shift(n3, n2, n1, d):
    """Periodic shift matrix S with (S f)[x] = f[x + d] on the flattened (n3, n2, n1) grid."""
    N = n1 * n2 * n3
    idx = np.arange(N).reshape(n3, n2, n1)
    src = np.roll(idx, shift=(-d[2], -d[1], -d[0]), axis=(0, 1, 2)).ravel()
    S = np.zeros((N, N))
    S[np.arange(N), src] = 1.0
    return S


def _stencil_matrices(kind, n3, n2, n1):
    """Real-space difference matrices D_r (r = x1, x2, x3) of the paper's stencils, h = 1."""
    e = np.eye(3, dtype=int)
    Sh = lambda d: _shift(n3, n2, n1, tuple(int(v) for v in d))
    mats = []
    for r in range(3):
        s, t = (r + 1) % 3, (r + 2) % 3
        if kind == "CD":
            D = 0.5 * (Sh(e[r]) - Sh(-e[r]))
        elif kind == "ACD":
            D = sum(0.125 * (Sh(e[r] + a * e[s] + b * e[t]) - Sh(-e[r] + a * e[s] + b * e[t]))
                    for a in (-1, 1) for b in (-1, 1))
        elif kind == "AFD":
            D = sum(0.25 * (Sh(e[r] + a * e[s] + b * e[t]) - Sh(a * e[s] + b * e[t]))
                    for a in (0, 1) for b in (0, 1))
        elif kind == "ABD":
            D = sum(0.25 * (Sh(a * e[s] + b * e[t]) - Sh(-e[r] + a * e[s] + b * e[t]))
                    for a in (0, -1) for b in (0, -1))
        mats.append(D)
    return mats


def _fourier_diff_matrices(n):
    """Textbook periodic spectral differentiation matrix for odd n on [0, n) (Trefethen 2000, ch. 3):
    D_ij = (pi/n) (-1)^{i-j} / sin(pi (i-j)/n), D_ii = 0."""
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (np.pi / n) * (-1.0) ** (i - j) / np.sin(np.pi * (i - j) / n)
    I = np.eye(n)
    return [np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I))]


def _dense_equilibrium_strain(lam, mu, E, grad, div):
    """Solve div_b C (E_bar + sym grad_a u) = 0 for u (minimum-norm least squares), return eps."""
    N = lam.size
    l = lam.ravel()
    m_ = mu.ravel()

    def strain_from_u(U):          # U: (3N, cols)
        cols = U.shape[1]
        u = U.reshape(3, N, cols)
        H = np.array([[grad[j] @ u[i] for j in range(3)] for i in range(3)])   # H_ij = d_j u_i
        return 0.5 * (H + np.swapaxes(H, 0, 1))

    def stress(eps):
        tr = eps[0, 0] + eps[1, 1] + eps[2, 2]
        s = 2 * m_[:, None] * eps
        for i in range(3):
            s[i, i] = s[i, i] + l[:, None] * tr
        return s

    def divergence(s):
        return np.concatenate([sum(div[j] @ s[i, j] for j in range(3)) for i in range(3)])

    K = divergence(stress(strain_from_u(np.eye(3 * N))))
    Eb = O.voigt_to_tensor(np.asarray(E, float))[:, :, None, None] * np.ones((1, 1, N, 1))
    rhs = -divergence(stress(Eb))
    u, *_ = np.linalg.lstsq(K, rhs, rcond=None)
    eps = Eb + strain_from_u(u)
    return np.stack([eps[i, j, :, 0] for (i, j) in O.VOIGT])


@pytest.mark.parametrize("scheme,grad_kind,div_kind,n", [
    ("CD", "CD", "CD", 4), ("ACD", "ACD", "ACD", 4), ("AFB_R", "AFD", "ABD", 4), ("AHC", "AFD", "ABD", 4),
    ("F", "F", "F", 5)])
def test_fixed_point_equals_dense_real_space_solve(scheme, grad_kind, div_kind, n):
    """The iterated fixed point equals a direct solve of the real-space stencil equations
    (Sec. 5.3 stencils; for F the spectral differentiation matrix, odd n), brute force at n^3."""
    lam, mu = M.random_field(n, n, n, seed=11)
    E = np.array([0.01, 0.0, -0.003, 0.0, 0.002, 0.004])
    r = O.solve(lam, mu, scheme, E, tol=1e-13, maxit=5000)
    assert r.converged
    if grad_kind == "F":
        grad = div = _fourier_diff_matrices(n)
    else:
        grad = _stencil_matrices(grad_kind, n, n, n)
        div = _stencil_matrices(div_kind, n, n, n)
    eps = _dense_equilibrium_strain(lam, mu, E, grad, div)
    np.testing.assert_allclose(r.eps.reshape(6, -1), eps, atol=1e-11)


# ----------------------------------------------------------------------------- DGO
@pytest.mark.parametrize("power", [1, 2])
def test_dgo_weights_partition_of_unity(power):
    """S_m(x) = sum_{nu=-m}^{m-1} sinc^p(pi (nu + x)) -> 1 for p = 1 and p = 2 (alias-sum weights)."""
    errs = []
    for m in (4, 16, 64, 256):
        Sm = sum(O.sinc_weight(np.array([nu * 16 + 6]), 16)[0] ** power for nu in range(-m, m))
        errs.append(abs(Sm - 1.0))
    assert errs[-1] < errs[0] and errs[-1] < 2e-3


@pytest.mark.parametrize("power", [1, 2])
def test_dgo_1d_closed_form(power):
    """In 1D Gamma_H(k) = -1/C_H for all k, so Gamma^c_omega = -S_m(omega/n)/C_H, Gamma^c_0 = 0."""
    n = 8
    lam_h, mu_h = 0.0, 2.0
    G = O.dgo_operator(1, 1, n, 1.0, lam_h, mu_h, power=power)
    g11 = G[0, 0, 0, 0, 0, :]
    om = np.arange(n)
    Sm = np.array([sum((np.sin(np.pi * (nu + w / n)) / (np.pi * (nu + w / n))) ** power for nu in range(-4, 4))
                   for w in om[1:]])
    np.testing.assert_allclose(g11[1:], -Sm / (lam_h + 2 * mu_h), atol=1e-14)
    assert g11[0] == 0.0


@pytest.mark.parametrize("power", [1, 2])
def test_dgo_on_axis_closed_form_and_symmetry(power):
    """Gamma^c(omega1, 0, 0) = Gamma_H(e1) S_m(omega1/n); Gamma^c(n - omega) = Gamma^c(omega), real."""
    n = 6
    lam_h, mu_h = 1.3, 0.6
    G = O.dgo_operator(n, n, n, 1.0, lam_h, mu_h, power=power)
    e1 = np.array([[1.0], [0.0], [0.0]])
    Gh = O.green_hat_iso(e1, lam_h, mu_h)[0]
    for w in range(1, n):
        Sm = sum((np.sin(np.pi * (nu + w / n)) / (np.pi * (nu + w / n))) ** power for nu in range(-3, 3))
        for p, (i, j) in enumerate(O.VOIGT):
            B = np.zeros((3, 3))
            B[i, j] = B[j, i] = 1.0
            Bk = B @ e1[:, 0]
            ref = -0.5 * (np.outer(Gh @ Bk, e1[:, 0]) + np.outer(e1[:, 0], Gh @ Bk)) * Sm
            np.testing.assert_allclose(G[p][:, :, 0, 0, w], ref, atol=1e-13)
    idx = (-np.arange(n)) % n
    np.testing.assert_allclose(G, G[..., idx, :, :][..., :, idx, :][..., :, :, idx], atol=1e-13)


def test_dgo_polarization_1d_equals_direct_solve():
    """1D DGO, polarization form: the fixed point solves E = E_bar + F^+ diag(-S_m / C_H) F^- (C - C_H) E,
    assembled here with numpy's FFT and the closed-form 1D operator, and solved directly."""
    n = 10
    rng = np.random.default_rng(4)
    C = np.exp(rng.uniform(np.log(0.5), np.log(30.0), n))
    lam = np.zeros((1, 1, n))
    mu = (0.5 * C).reshape(1, 1, n)
    r = O.solve(lam, mu, "DGO", [1.0, 0, 0, 0, 0, 0], tol=1e-14, maxit=5000)
    assert r.converged
    C_H = 0.5 * (C.min() + C.max())
    w = np.arange(n)
    Sm = np.array([sum((np.sin(np.pi * (nu + x / n)) / (np.pi * (nu + x / n))) ** 2 for nu in range(-5, 5))
                   if x else 0.0 for x in w])
    # column j of the operator: E_bar-free part applied to unit vectors
    Op = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Op[:, j] = np.fft.ifft(-Sm / C_H * np.fft.fft((C - C_H) * e)).real
    E = np.linalg.solve(np.eye(n) - Op, np.ones(n))
    np.testing.assert_allclose(r.eps[0, 0, 0], E, rtol=1e-11)


# ----------------------------------------------------------------------------- gradient
def test_gradient_closed_form_matches_finite_differences():
    lam, mu = M.random_field(4, 4, 4, seed=7)
    I, J = 0, 0
    scheme = "AFB_R"
    ref = O.default_reference(lam, mu)
    EI = np.zeros(6); EI[I] = 1.0
    EJ = np.zeros(6); EJ[J] = 1.0
    rI = O.solve(lam, mu, scheme, EI, tol=1e-14, maxit=20000, ref=ref)
    rJ = O.solve(lam, mu, scheme, EJ, tol=1e-14, maxit=20000, ref=ref)
    gl, gm = O.gradient_closed_form(rI.eps, rJ.eps)
    vox = [0, 17, 42]
    fl, fm = O.gradient_fd(lam, mu, scheme, I, J, vox, rel_step=1e-5, tol=1e-14)
    np.testing.assert_allclose(gl.ravel()[vox], fl, rtol=1e-5)
    np.testing.assert_allclose(gm.ravel()[vox], fm, rtol=1e-5)


def test_paper_increment_stop_rule_runs():
    lam, mu = M.random_field(4, 4, 4, seed=1)
    r = O.solve(lam, mu, "AFB_R", [0.01, 0, 0, 0, 0, 0], tol=1e-12, stop_rule=1, maxit=500)
    assert r.converged and r.iters > 2


@pytest.mark.parametrize("scheme", ["AFB_R", "ACD"])
def test_increment_criterion_from_the_displacement_iterates(scheme):
    """The paper's stopping quantity of iteration k (Algorithms T-3D / P-3D), sum over the modes of
    |du^(k) - du^(k-1)|, rebuilt from the displacement fields u^p the oracle returns after k - 1, k and
    k + 1 iterations: du^(k) - du^(k-1) = u_(k+1) - 2 u_k + u_(k-1) in real space, numpy's unitary FFT,
    the Euclidean norm of each mode's vector, summed (a non-cubic grid with an odd axis)."""
    lam, mu = M.random_field(5, 4, 6, seed=8)
    E = [0.01, -0.002, 0.003, 0.001, 0.0, 0.002]
    ref = O.solve(lam, mu, scheme, E, tol=0.0, maxit=7, stop_rule=1, max_iters_exact=7)
    assert np.isinf(ref.history[0])
    disp = {k: O.solve(lam, mu, scheme, E, max_iters_exact=k).disp for k in range(1, 8)}
    for k in range(2, 7):
        d2 = disp[k + 1] - 2.0 * disp[k] + disp[k - 1]
        F = np.fft.fftn(d2, axes=(1, 2, 3), norm="ortho")
        crit = np.sum(np.sqrt(np.sum(np.abs(F) ** 2, axis=0)))
        assert abs(crit - ref.history[k - 1]) <= 1e-12 * ref.history[k - 1]


# ----------------------------------------------------------------------------- DGO off-axis pins
def _voigt_stiffness(lam_h, mu_h):
    """6x6 map from tensor components (11,22,33,23,13,12) of a strain to those of lam tr I + 2 mu eps."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam_h
    C[np.arange(6), np.arange(6)] += 2.0 * mu_h
    return C


def _dgo_matrix(G, w1, w2, w3):
    """The oracle's Gamma^c(omega) as a 6x6 map on tensor components (basis p has unit entries at (i,j), (j,i))."""
    Mx = np.zeros((6, 6))
    for p in range(6):
        out = G[p][:, :, w3, w2, w1]
        Mx[:, p] = [out[i, j] for (i, j) in O.VOIGT]
    return Mx


def _axis_alias_sum(n, w, power):
    """S(omega) = sum_{nu=-m}^{m-1} sinc^p((nu n + omega)/n), m = n/2 (numpy's normalised sinc)."""
    m = max(1, n // 2)
    return sum(np.sinc((nu * n + w) / n) ** power for nu in range(-m, m))


@pytest.mark.parametrize("power", [1, 2])
def test_dgo_off_axis_trace_and_eigenvalues(power):
    """-Gamma^c(omega) C_H = sum_nu w_nu P(k_nu), P(k) the C_H-orthogonal projection onto the compatible strains
    sym(u (x) k) (rank 3; Sec. 5.4 isotropic G_H).  Hence its trace is 3 prod_r S_r(omega_r) at every omega != 0
    (an axis pairing mistake on a non-cubic grid changes S_r), and with the squared weights its eigenvalues lie in
    [0, prod_r S_r] within [0, 1]; with the printed weights s (which change sign) they leave [0, 1], so the
    contraction argument of the Green-operator iteration fails for them (the oracle's weight reading)."""
    n1, n2, n3 = 4, 6, 8
    lam_h, mu_h = 1.3, 0.6
    G = O.dgo_operator(n3, n2, n1, 1.0, lam_h, mu_h, power=power)
    C = _voigt_stiffness(lam_h, mu_h)
    lo, hi = np.inf, -np.inf
    for w3, w2, w1 in itertools.product(range(n3), range(n2), range(n1)):
        if w1 == w2 == w3 == 0:
            assert np.all(_dgo_matrix(G, 0, 0, 0) == 0.0)
            continue
        A = -_dgo_matrix(G, w1, w2, w3) @ C
        S = _axis_alias_sum(n1, w1, power) * _axis_alias_sum(n2, w2, power) * _axis_alias_sum(n3, w3, power)
        assert abs(np.trace(A) - 3.0 * S) < 1e-12
        ev = np.linalg.eigvals(A).real
        lo, hi = min(lo, ev.min()), max(hi, ev.max())
        if power == 2:
            assert ev.min() > -1e-12 and ev.max() < S + 1e-12
    if power == 2:
        assert hi <= 1.0
    else:
        assert lo < -0.1 and hi > 1.1


def test_dgo_generic_omega_equals_projection_sum():
    """At a generic off-axis omega on a non-cubic grid, Gamma^c(omega) = -sum_nu w_nu P(k_nu) C_H^{-1}, with P(k) built
    here by least squares in the C_H energy metric (not from the Green tensor), k_nu,r = 2 pi (nu_r n_r + omega_r)/n_r
    and w_nu = prod_r sinc^2, nu_r in [-n_r/2, n_r/2 - 1] (Algorithm D-3D with the squared weights the oracle reads)."""
    n1, n2, n3 = 4, 6, 8
    lam_h, mu_h = 0.9, 1.4
    G = O.dgo_operator(n3, n2, n1, 1.0, lam_h, mu_h, power=2)
    C = _voigt_stiffness(lam_h, mu_h)
    D = np.diag([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])     # a : b over the full symmetric tensors
    ns = (n1, n2, n3)
    for om in ((1, 2, 3), (3, 5, 1), (2, 1, 6)):
        ref = np.zeros((6, 6))
        for nu in itertools.product(*[range(-n // 2, n // 2) for n in ns]):
            j = [nu[r] * ns[r] + om[r] for r in range(3)]
            w = np.prod([np.sinc(j[r] / ns[r]) ** 2 for r in range(3)])
            k = np.array([2.0 * np.pi * j[r] / ns[r] for r in range(3)])
            B = np.zeros((6, 3))                     # u -> tensor components of sym(u (x) k)
            for p, (a, b) in enumerate(O.VOIGT):
                B[p, a] += 0.5 * k[b]
                B[p, b] += 0.5 * k[a]
            W = D @ C
            P = B @ np.linalg.solve(B.T @ W @ B, B.T @ W)
            ref -= w * P @ np.linalg.inv(C)
        np.testing.assert_allclose(_dgo_matrix(G, *om), ref, atol=1e-12)


def _axis_alias_sum_sym(n, w, power):
    """S+(omega) = sum_{nu=-m}^{m} sinc^p((nu n + omega)/n), m = n/2: the symmetric alias range."""
    m = max(1, n // 2)
    return sum(np.sinc((nu * n + w) / n) ** power for nu in range(-m, m + 1))


@pytest.mark.parametrize("power", [1, 2])
def test_dgo_symmetric_range_1d_closed_form(power):
    """1D, alias range [-m, m]: Gamma_H(k) = -1/C_H for every k, so the Hermitian part of the alias sum is
    Gamma^c_omega = -(S+(omega) + S+(n - omega)) / (2 C_H); Gamma^c_0 = 0."""
    n = 8
    lam_h, mu_h = 0.0, 2.0
    G = O.dgo_operator(1, 1, n, 1.0, lam_h, mu_h, power=power, alias_range="symmetric")
    g11 = G[0, 0, 0, 0, 0, :]
    ref = [-(_axis_alias_sum_sym(n, w, power) + _axis_alias_sum_sym(n, n - w, power)) / (2.0 * (lam_h + 2 * mu_h))
           for w in range(1, n)]
    np.testing.assert_allclose(g11[1:], ref, atol=1e-14)
    assert g11[0] == 0.0
    # the printed range differs from it by boundary terms
    Gp = O.dgo_operator(1, 1, n, 1.0, lam_h, mu_h, power=power)
    assert np.abs(Gp[0, 0, 0, 0, 0, 1:] - g11[1:]).max() > 1e-3


def test_dgo_symmetric_range_even_trace_eigenvalues():
    """3D, 4 x 6 x 8, s^2 weights, alias range [-m, m] in its Hermitian part: Gamma^c(n - omega) = Gamma^c(omega);
    -Gamma^c C_H is half the sum of two positive combinations of rank-3 projections, so its trace is
    3/2 (prod_r S+_r(omega_r) + prod_r S+_r(n_r - omega_r)) and its eigenvalues lie in [0, 1]."""
    n1, n2, n3 = 4, 6, 8
    lam_h, mu_h = 1.3, 0.6
    G = O.dgo_operator(n3, n2, n1, 1.0, lam_h, mu_h, power=2, alias_range="symmetric")
    idx = [(-np.arange(n)) % n for n in (n3, n2, n1)]
    np.testing.assert_allclose(G, G[..., idx[0], :, :][..., :, idx[1], :][..., :, :, idx[2]], atol=1e-13)
    C = _voigt_stiffness(lam_h, mu_h)
    for w3, w2, w1 in itertools.product(range(n3), range(n2), range(n1)):
        if w1 == w2 == w3 == 0:
            continue
        A = -_dgo_matrix(G, w1, w2, w3) @ C
        Sp = _axis_alias_sum_sym(n1, w1, 2) * _axis_alias_sum_sym(n2, w2, 2) * _axis_alias_sum_sym(n3, w3, 2)
        Sm = (_axis_alias_sum_sym(n1, (n1 - w1) % n1, 2) * _axis_alias_sum_sym(n2, (n2 - w2) % n2, 2)
              * _axis_alias_sum_sym(n3, (n3 - w3) % n3, 2))
        assert abs(np.trace(A) - 1.5 * (Sp + Sm)) < 1e-12
        ev = np.linalg.eigvals(A).real
        assert ev.min() > -1e-12 and ev.max() < 1.0 + 1e-12


def test_dgo_alias_ranges_agree_as_m_grows():
    """The two alias ranges differ by the terms nu = m and nu = -m - 1, of size sinc^2 ~ 1/(pi m)^2: in 1D the
    difference falls by about 16 when m grows by 4 (s^2 weights).  Both sums tend to the full series, 1; what the
    truncation leaves out is at most sum_{|nu| > m} 1/(pi (nu -+ 1/2))^2 < 2/(pi^2 m)."""
    n = 6
    d = []
    for m in (2, 8, 32):
        Gp = O.dgo_operator(1, 1, n, 1.0, 0.0, 0.5, m=m, power=2)[0, 0, 0, 0, 0, 1:]
        Gs = O.dgo_operator(1, 1, n, 1.0, 0.0, 0.5, m=m, power=2, alias_range="symmetric")[0, 0, 0, 0, 0, 1:]
        d.append(np.abs(Gp - Gs).max())
        assert np.all(-Gs <= 1.0 + 1e-12) and np.all(-Gs >= 1.0 - 2.0 / (np.pi ** 2 * m))
    assert d[1] < d[0] / 8 and d[2] < d[1] / 8


@pytest.mark.parametrize("rng", ["printed", "symmetric"])
def test_dgo_stress_form_1d_reaches_exact_solution(rng):
    """1D, printed stress form E_check += Gamma^c T_check with s^2 weights: at its fixed point
    S(omega) F(C E)(omega) = 0 with S > 0 at every omega != 0, so the stress C E is uniform and
    E_i = E_bar / (C_i <1/C>) (the 1D matrix-inclusion solution of Sec. 2)."""
    n = 10
    rng_ = np.random.default_rng(6)
    C = np.exp(rng_.uniform(np.log(1.0), np.log(3.0), n))
    lam = np.zeros((1, 1, n))
    mu = (0.5 * C).reshape(1, 1, n)
    r = O.solve(lam, mu, "DGO", [1.0, 0, 0, 0, 0, 0], tol=1e-13, maxit=5000, dgo_form="stress", dgo_range=rng)
    assert r.converged
    np.testing.assert_allclose(r.eps[0, 0, 0], 1.0 / (C * np.mean(1.0 / C)), rtol=1e-11)


def _permute_sym(E6, perm):
    """Tensor components of E'_ij = E_{perm[i] perm[j]}."""
    T = O.voigt_to_tensor(np.asarray(E6, np.float64))
    return O.tensor_to_voigt(T[np.ix_(perm, perm)])


@pytest.mark.parametrize("scheme", ["DGO", "AFB_R", "F"])
@pytest.mark.parametrize("axis", [1, 2])
def test_laminate_along_x2_and_x3_non_cubic(scheme, axis):
    """Laminates along x2 and along x3 of a 4 x 6 x 8 grid have the exact layered response (traction continuity,
    in-plane strains uniform), obtained from the x1 closed form by relabelling the axes.  On a non-cubic grid this
    pins the per-axis lengths and alias ranges of the operators off the x1 axis."""
    n1, n2, n3 = 4, 6, 8
    nax = (n1, n2, n3)[axis]
    rng = np.random.default_rng(21 + axis)
    prof_l = np.exp(rng.uniform(np.log(0.5), np.log(20.0), nax))
    prof_m = np.exp(rng.uniform(np.log(0.5), np.log(20.0), nax))
    shape = [1, 1, 1]
    shape[2 - axis] = nax
    lam = np.broadcast_to(prof_l.reshape(shape), (n3, n2, n1)).copy()
    mu = np.broadcast_to(prof_m.reshape(shape), (n3, n2, n1)).copy()
    E = np.array([0.01, -0.004, 0.007, 0.003, -0.002, 0.005])
    kw = dict(dgo_form="stress") if scheme == "DGO" else {}
    r = O.solve(lam, mu, scheme, E, tol=1e-12, maxit=5000, **kw)
    assert r.converged
    perm = [axis] + [a for a in range(3) if a != axis]     # laminate frame: its axis 0 is the layering axis
    s_lam, _ = _laminate_closed_form(prof_l, prof_m, _permute_sym(E, perm))
    inv = np.argsort(perm)
    np.testing.assert_allclose(r.sigma_mean, _permute_sym(s_lam, inv), rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("form,power,grows", [("stress", 1, True), ("polarization", 1, True),
                                              ("stress", 2, False), ("polarization", 2, False)])
def test_dgo_printed_weights_diverge_on_two_phase_cube(form, power, grows):
    """The DGO weight and form readings on a 6^3 two-phase cube (edge 3, contrast 10, C_H = 1/2 (min + max)): with the printed weights s the
    iteration grows in the printed stress form and in the polarization form alike; with s^2 both decrease
    monotonically in the long run (the polarization form reaches 1e-10)."""
    ind = M.cube_indicator(6, 3)
    chi = 10.0
    lam = 1.0 * (1.0 + ind * (chi - 1.0))
    mu = 0.7 * (1.0 + ind * (chi - 1.0))
    r = O.solve(lam, mu, "DGO", [0.01, 0, 0, 0, 0, 0], tol=1e-10, maxit=200, dgo_form=form, dgo_power=power)
    h = np.array(r.history)
    if grows:
        assert h[-1] > 1e3 * h.min() and h[-1] > h[0]
    else:
        assert h[-1] == h.min() and h[-1] < 1e-4 * h[0]
        if form == "polarization":
            assert r.converged


@pytest.mark.parametrize("scheme", ["AFB_R", "F", "DGO"])
def test_zero_load_is_solved_in_one_iteration(scheme):
    """No mean strain and no eigenstrain: the stress is identically zero, which is equilibrium; the solve
    stops after its first iteration with eps = 0 and residual 0 (a zero reference norm is no division)."""
    lam, mu = M.random_field(4, 4, 4, seed=1)
    r = O.solve(lam, mu, scheme, [0.0] * 6, tol=1e-8, maxit=10)
    assert r.converged and r.iters == 1 and r.residual == 0.0
    assert np.all(r.eps == 0.0) and np.all(r.sigma_mean == 0.0)
