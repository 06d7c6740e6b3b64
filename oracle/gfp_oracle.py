"""FP64 CPU oracle of the Green-function-preconditioned (GFP) fixed-point solver.

TEST INFRASTRUCTURE ONLY. This module is the plain, slow, literal statement of what
the solver computes, used to check the CUDA path. Only the tests, the smoke check and
the CPU-baseline leg of the benchmark may import it; the product path never does, and
it shares no code with the CUDA library (its inputs come from the seeded generators in
paper_2009_03762_gb300.microstructure, which hold none of the method's arithmetic).

Everything is numpy float64 / complex128 and follows the paper (Khorrami, Mianroodi,
Shanthraj, Svendsen, "Development and comparison of spectral algorithms for numerical
modeling of the quasi-static mechanical behavior of inhomogeneous materials"):

* the discrete Fourier transforms are the paper's unitary matrices F^{+-}, applied axis by
  axis as the Rayleigh product (Sec. 5.2 eqs. DisFouSca3D/DisFouMat3D; App. A for TD,
  Sec. 3.2 eq. DisFouPC1D and App. B for PCD) -- an O(n^4) dense transform, no FFT;
* the effective wave vectors q^a, q^b are the modal symbols of the difference stencils
  (Sec. 3.1 eqs. FreDifFinFBDF1D, FreDifFinCDDF1D; Sec. 5.3 eqs. FreDifFinFBDF3D,
  FreDifFinFBDFR3D, EffNumWavConWil3D), evaluated with complex exponentials;
* the Green operator is the literal complex 3x3 inverse of G_H^{-1}(q^a, q^b)
  (Sec. 5.2 eq. EquMecFunGre3D), set to zero where q^a . q^b = 0 (Sec. 3.1, zero modes);
* the basic scheme of Algorithms T-3D / P-3D is the fixed-point map of the Lippmann-Schwinger
  form of Sec. 5.2: the displacement coefficients u_check are corrected by G_H (T_check q^b)
  until the divergence T_check q^b vanishes (`_fdd_step`); the strain is E_bar + F^+ sym(u_check (x) q^a);
* Algorithm D-3D's discrete Green operator Gamma^c is the alias sum of the continuous isotropic
  Gamma_H over the wave numbers k_{nu n + omega} (Sec. 5.4); `_solve_dgo` states the weights and
  the update form it uses by default.

Pins (tests/test_oracle_pins.py) cover every function here; the alias sum off the coordinate axes
is pinned by an independent construction from C_H-orthogonal projections onto compatible strains.

Readings where the paper is silent or garbled:
* stopping rule: the default is the equilibrium residual
  eta = ||T(k) q^b(k)||_2 / ||T(k=0)||_F over all modes (unitary DFT, so this equals
  ||div^b T|| / (sqrt(N) ||mean T||)); the paper's own rule (L1 norm of the difference of
  successive increments) is available as stop_rule=1.  For Algorithm D the equilibrium
  residual does not vanish at its fixed point, so the default there is the strain
  increment eta_D = ||Delta E||_2 / (sqrt(N) ||E_bar||_F).
* iteration count: one iteration = one evaluation of the stress and of eta; a
  homogeneous medium therefore stops after 1 iteration.
* reference medium: half the sum of the grid minimum and maximum of each Lame constant
  unless given.
* symbols that vanish mathematically (e.g. sinh(q h) at the Nyquist mode) are set to an
  exact zero when their modulus is below 1e-12/h (the smallest non-zero symbol on grids
  up to 10^4 points is far larger).
"""
from __future__ import annotations

import numpy as np

VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
SCHEMES = ("F", "CD", "ACD", "HC", "AHC", "AFB_R", "R", "DGO")
_ZERO = 1e-12


# --------------------------------------------------------------------------------------
# 1D index maps and discrete Fourier matrices (Sec. 3.1 eq. FieFouAppTra1D; App. A;
# Sec. 3.2 eq. DisFouPC1D; App. B; Algorithm D-1D for the omega-indexed matrices)
# --------------------------------------------------------------------------------------
def kappa(n):
    """kappa = mu - 1 - m for mu = 1..n, m = floor(n/2): -m..n-1-m."""
    m = n // 2
    return np.arange(1, n + 1) - 1 - m


def nodes(n, h, disc):
    """TD nodes x_i = (i - 1) h, PCD cell centres x_i^c = (i - 1/2) h, i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return (i - 1.0) * h if disc == "TD" else (i - 0.5) * h


def dft_matrices(n, h, disc="TD", index="kappa"):
    """Unitary F^+_{mu i} = n^{-1/2} e^{+q_mu x_i}, F^-_{mu i} = n^{-1/2} e^{-q_mu x_i}.

    index="kappa": q_mu = i k_{mu-1-m} (Algorithms T, P); index="omega": wave numbers
    k_omega, omega = 0..n-1 (Algorithm D).  k_kappa = 2 pi kappa / l with l = n h.
    """
    l = n * h
    idx = kappa(n) if index == "kappa" else np.arange(n)
    k = 2.0 * np.pi * idx / l
    x = nodes(n, h, disc)
    phase = np.outer(k, x)
    return np.exp(1j * phase) / np.sqrt(n), np.exp(-1j * phase) / np.sqrt(n)


def _apply_axis(M, f, axis):
    """g[..., mu, ...] = sum_i M[mu, i] f[..., i, ...] along `axis`."""
    g = np.tensordot(M, f, axes=([1], [axis]))
    return np.moveaxis(g, 0, axis)


def forward3(f, mats):
    """f_check = F^-_{mu1 i1} F^-_{mu2 i2} F^-_{mu3 i3} f_{i1 i2 i3} (Rayleigh product, eq. DisFouMat3D).

    Arrays are indexed [..., i3, i2, i1]; mats = ((F1p, F1m), (F2p, F2m), (F3p, F3m)).
    """
    g = _apply_axis(mats[0][1], f, f.ndim - 1)
    g = _apply_axis(mats[1][1], g, f.ndim - 2)
    return _apply_axis(mats[2][1], g, f.ndim - 3)


def inverse3(fc, mats):
    """f_i = F^+_{mu1 i1} F^+_{mu2 i2} F^+_{mu3 i3} f_check_mu (sum over mu)."""
    g = _apply_axis(mats[0][0].T, fc, fc.ndim - 1)
    g = _apply_axis(mats[1][0].T, g, fc.ndim - 2)
    return _apply_axis(mats[2][0].T, g, fc.ndim - 3)


# --------------------------------------------------------------------------------------
# Effective wave numbers (modal symbols of the difference stencils)
# --------------------------------------------------------------------------------------
def q_fourier(n, h):
    """q_mu = i k_{mu-1-m} (plain Fourier, 'F')."""
    return 1j * 2.0 * np.pi * kappa(n) / (n * h)


def q1d(kind, q, h):
    """1D symbols: FD, BD (eq. FreDifFinFBDF1D), CD, hC (eq. FreDifFinCDDF1D), F, W (eq. FreDifFinFBDFR3D)."""
    if kind == "F":
        return q.copy()
    if kind == "FD":
        return (np.exp(q * h) - 1.0) / h
    if kind == "BD":
        return (1.0 - np.exp(-q * h)) / h
    if kind == "CD":
        return np.sinh(q * h) / h
    if kind == "hC":
        return 2.0 * np.sinh(0.5 * q * h) / h
    if kind == "W":
        # Willot's q^W = h^-1 tanh(q h / 2)(e^{q h} + 1); indeterminate at q h = -i pi,
        # where its limit q^FD is used (Sec. 5.3 after eq. FreDifFinFBDFR3D).
        out = np.empty_like(q)
        sing = np.abs(np.abs(q * h) - np.pi) < 1e-12
        ok = ~sing
        out[ok] = np.tanh(0.5 * q[ok] * h) * (np.exp(q[ok] * h) + 1.0) / h
        out[sing] = (np.exp(q[sing] * h) - 1.0) / h
        return out
    raise ValueError(kind)


def _clean(a, h):
    a = np.array(a, dtype=np.complex128)
    a[np.abs(a) < _ZERO / h] = 0.0
    return a


def wave_vectors(scheme, n3, n2, n1, h=1.0):
    """(q^a, q^b) as arrays of shape (3, n3, n2, n1), component r = 0,1,2 for x1, x2, x3.

    3D averaged symbols (eq. FreDifFinFBDF3D), with (s, t) the other two axes of r:
      AFD_r = 1/4 q^FD_r (e^{q_s h} + 1)(e^{q_t h} + 1)
      ACD_r = q^CD_r cosh(q_s h) cosh(q_t h)
      AhC_r = q^hC_r cosh(q_s h / 2) cosh(q_t h / 2)
      R_r   = 1/4 q^W_r (e^{q_s h} + 1)(e^{q_t h} + 1)           (eq. FreDifFinFBDFR3D)
    Pairings (eq. EffNumWavConWil3D): conjugate q^b = q^{a*} for F, CD, ACD, hC, AhC;
    AFB/R = (AFD, AhC); R = (R, AhC).
    """
    ns = (n1, n2, n3)
    qs = [q_fourier(nr, h) for nr in ns]
    shape = (n3, n2, n1)

    def bc(v, r):
        sh = [1, 1, 1]
        sh[2 - r] = ns[r]
        return np.broadcast_to(v.reshape(sh), shape)

    def vec(fr, avg):
        out = np.empty((3,) + shape, dtype=np.complex128)
        for r in range(3):
            s, t = (r + 1) % 3, (r + 2) % 3
            out[r] = bc(fr(qs[r]), r) * bc(avg(qs[s]), s) * bc(avg(qs[t]), t)
        return out

    one = lambda q: np.ones_like(q)
    if scheme == "F":
        qa = vec(lambda q: q1d("F", q, h), one)
        qb = np.conj(qa)
    elif scheme == "CD":
        qa = vec(lambda q: q1d("CD", q, h), one)
        qb = np.conj(qa)
    elif scheme == "HC":
        qa = vec(lambda q: q1d("hC", q, h), one)
        qb = np.conj(qa)
    elif scheme == "ACD":
        qa = vec(lambda q: q1d("CD", q, h), lambda q: np.cosh(q * h))
        qb = np.conj(qa)
    elif scheme == "AHC":
        qa = vec(lambda q: q1d("hC", q, h), lambda q: np.cosh(0.5 * q * h))
        qb = np.conj(qa)
    elif scheme == "AFB_R":
        qa = vec(lambda q: 0.25 * q1d("FD", q, h), lambda q: np.exp(q * h) + 1.0)
        qb = vec(lambda q: q1d("hC", q, h), lambda q: np.cosh(0.5 * q * h))
    elif scheme == "R":
        qa = vec(lambda q: 0.25 * q1d("W", q, h), lambda q: np.exp(q * h) + 1.0)
        qb = vec(lambda q: q1d("hC", q, h), lambda q: np.cosh(0.5 * q * h))
    else:
        raise ValueError(scheme)
    return _clean(qa, h), _clean(qb, h)


# --------------------------------------------------------------------------------------
# Green operator of the homogeneous reference medium (eq. EquMecFunGre3D)
# --------------------------------------------------------------------------------------
def green(qa, qb, lam_h, mu_h):
    """G_H(q^a, q^b) = [ -mu_H (q^a.q^b) I - mu_H q^a (x) q^b - lam_H q^b (x) q^a ]^{-1} per mode.

    Returns (..., 3, 3); modes with q^a . q^b = 0 (including k = 0) get G_H = 0.
    """
    qa_ = np.moveaxis(qa, 0, -1)
    qb_ = np.moveaxis(qb, 0, -1)
    dot = np.sum(qa_ * qb_, axis=-1)
    Ginv = (-mu_h * dot[..., None, None] * np.eye(3)
            - mu_h * qa_[..., :, None] * qb_[..., None, :]
            - lam_h * qb_[..., :, None] * qa_[..., None, :])
    sing = np.abs(dot) == 0.0
    Ginv[sing] = np.eye(3)
    G = np.linalg.inv(Ginv)
    G[sing] = 0.0
    return G


def sym_outer(u, q):
    """sym(u (x) q) for vector fields u, q of shape (3, ...): returns (3, 3, ...)."""
    o = u[:, None] * q[None, :]
    return 0.5 * (o + np.swapaxes(o, 0, 1))


def matvec(T, q):
    """(T q)_i = sum_j T_ij q_j for T (3, 3, ...), q (3, ...)."""
    return np.einsum("ij...,j...->i...", T, q)


def gamma_apply(G, qa, qb, A):
    """Gamma A := -sym( G_H (A q^b) (x) q^a ), so that Algorithm T's increment is -Gamma T."""
    v = matvec(A, qb)
    Gv = np.einsum("...ij,j...->i...", G, v)
    return -sym_outer(Gv, qa)


def stiffness_apply(lam, mu, E):
    """T = C E with C = lambda I (x) I + mu (I box I + I triangle I): T = lambda tr(E) I + 2 mu E."""
    tr = E[0, 0] + E[1, 1] + E[2, 2]
    T = 2.0 * mu * E
    for i in range(3):
        T[i, i] = T[i, i] + lam * tr
    return T


def voigt_to_tensor(v):
    """Components (11,22,33,23,13,12) -> symmetric 3x3 (tensor components, no factor 2)."""
    v = np.asarray(v)
    T = np.empty((3, 3) + v.shape[1:], dtype=v.dtype)
    for p, (i, j) in enumerate(VOIGT):
        T[i, j] = v[p]
        T[j, i] = v[p]
    return T


def tensor_to_voigt(T):
    return np.stack([T[i, j] for (i, j) in VOIGT])


def default_reference(lam, mu):
    """lambda_H, mu_H = 1/2 (min + max) over the grid (reading of Sec. 4's C_H = 1/2 (C_M + C_I))."""
    return 0.5 * (lam.min() + lam.max()), 0.5 * (mu.min() + mu.max())


# --------------------------------------------------------------------------------------
# Discrete Green operator of Algorithm D-3D
# --------------------------------------------------------------------------------------
def sinc_weight(j, n):
    """s_j = sinc(pi j / n), with the exact zeros s_j = 0 for j = 0 mod n, j != 0 (eq. RepFieSerForPieCon1D)."""
    j = np.asarray(j, dtype=np.int64)
    x = np.pi * j / n
    out = np.ones(j.shape)
    nz = j != 0
    out[nz] = np.sin(x[nz]) / x[nz]
    out[(j % n == 0) & nz] = 0.0
    return out


def green_hat_iso(k, lam_h, mu_h):
    """Continuous isotropic G_H(k) = (mu_H |k|^2)^{-1} [I - (1+lam/mu)/(1+(1+lam/mu)) k^ (x) k^]."""
    k_ = np.moveaxis(k, 0, -1)
    k2 = np.sum(k_ * k_, axis=-1)
    r = 1.0 + lam_h / mu_h
    c = r / (1.0 + r)
    kk = k_[..., :, None] * k_[..., None, :] / k2[..., None, None]
    return (np.eye(3) - c * kk) / (mu_h * k2)[..., None, None]


def dgo_operator(n3, n2, n1, h, lam_h, mu_h, m=None, power=1, alias_range="printed"):
    """Gamma^c_omega for omega in [0,n1) x [0,n2) x [0,n3), the alias sum of Algorithm D-3D:

      Gamma^c_0 = 0,
      Gamma^c_omega = sum_{nu_r = -m_r}^{m_r - 1} prod_r s_{nu_r n_r + omega_r} Gamma_H(k_{nu n + omega}),
      Gamma_H(k) A = -sym[ G_H(k) A (k (x) k) ] = -sym( G_H(k) (A k) (x) k ).

    Returned as the action on the six symmetric basis tensors: array (6, 3, 3, n3, n2, n1);
    basis p = (11, 22, 33, 23, 13, 12) with unit entries at (i, j) and (j, i).
    m defaults to n_r / 2 on every axis (m = n/2, the paper's choice); an axis with n_r = 1
    uses m_r = 1 so that its range [-m_r, m_r - 1] contains nu_r = 0.
    alias_range = "symmetric": nu_r runs over [-m_r, m_r] instead.  That sum is not even in omega
    (omega -> n - omega maps the term nu to -nu - 1, outside the range at nu = m), and the increment
    of a real strain field is the real part of its inverse transform, i.e. the operator's Hermitian
    part; so this variant returns 1/2 (Sigma(omega) + Sigma(n - omega)), the reading the Nyquist
    modes of the finite-difference schemes take as well.
    """
    ns = (n1, n2, n3)
    ms = tuple(max(1, nr // 2 if m is None else m) for nr in ns)
    hi = tuple(mr + 1 if alias_range == "symmetric" else mr for mr in ms)
    shape = (n3, n2, n1)
    om = [np.arange(nr) for nr in ns]
    basis = []
    for (i, j) in VOIGT:
        B = np.zeros((3, 3))
        B[i, j] = 1.0
        B[j, i] = 1.0
        basis.append(B)
    out = np.zeros((6, 3, 3) + shape)
    om_grid = [np.broadcast_to(om[0][None, None, :], shape), np.broadcast_to(om[1][None, :, None], shape),
               np.broadcast_to(om[2][:, None, None], shape)]
    zero = (om_grid[0] == 0) & (om_grid[1] == 0) & (om_grid[2] == 0)
    for n3v in range(-ms[2], hi[2]):
        for n2v in range(-ms[1], hi[1]):
            for n1v in range(-ms[0], hi[0]):
                nu = (n1v, n2v, n3v)
                j = [nu[r] * ns[r] + om_grid[r] for r in range(3)]
                w = (sinc_weight(j[0], n1) * sinc_weight(j[1], n2) * sinc_weight(j[2], n3)) ** power
                k = np.stack([2.0 * np.pi * j[r] / (ns[r] * h) for r in range(3)]).astype(np.float64)
                k2 = (k * k).sum(axis=0)
                live = (w != 0.0) & (k2 > 0.0)
                if not live.any():
                    continue
                kl = k[:, live]
                G = green_hat_iso(kl, lam_h, mu_h)
                for p, B in enumerate(basis):
                    Bk = np.einsum("ij,j...->i...", B, kl)
                    GBk = np.einsum("...ij,j...->i...", G, Bk)
                    out[p][:, :, live] += w[live] * (-sym_outer(GBk, kl))
    out[:, :, :, zero] = 0.0
    if alias_range == "symmetric":
        i3, i2, i1 = [(-np.arange(nr)) % nr for nr in (n3, n2, n1)]
        out = 0.5 * (out + out[..., i3, :, :][..., :, i2, :][..., :, :, i1])
    return out


def dgo_apply(Gc, A):
    """Delta E = Gamma^c A for A given as a symmetric (3, 3, ...) complex field."""
    coeff = tensor_to_voigt(A)
    return np.einsum("pij...,p...->ij...", Gc, coeff)


# --------------------------------------------------------------------------------------
# Algorithms T-3D / P-3D / D-3D
# --------------------------------------------------------------------------------------
class Result:
    def __init__(self, eps, iters, residual, history, sigma_mean, converged, disp=None):
        self.eps = eps                  # (6, n3, n2, n1) tensor components (11,22,33,23,13,12)
        self.disp = disp                # (3, n3, n2, n1) periodic displacement u^p = F^+ u_check (Alg. T/P)
        self.iters = iters
        self.residual = residual
        self.history = history
        self.sigma_mean = sigma_mean    # (6,) tensor components
        self.converged = converged


def _ratio(num, den):
    """A residual num / den; with a zero reference (zero mean strain and no eigenstrain: the stress vanishes
    identically) a zero numerator is a converged state (0) and a non-zero one cannot be normalised (inf)."""
    if den > 0.0:
        return num / den
    return 0.0 if num == 0.0 else np.inf


def _fdd_step(u, Ebar_f, T0, lam, mu, qa, qb, G, mats):
    """One evaluation of the fixed-point map u_check -> u_check + G_H (T_check q^b) (Sec. 5.2).

    The compatible strain fluctuation of the current coefficients is F^+ sym(u_check (x) q^a), the
    stress is T^(0) + C : (that fluctuation) with T^(0) = C : E_bar, its transform T_check = F^- T,
    the discrete divergence T_check q^b, and the displacement correction G_H (T_check q^b).
    Returns (strain, stress, T_check, T_check q^b, correction).
    """
    Et = inverse3(sym_outer(u, qa), mats).real
    T = T0 + stiffness_apply(lam, mu, Et)
    Tc = forward3(T, mats)
    Tq = matvec(Tc, qb)
    du = np.einsum("...ij,j...->i...", G, Tq)
    return Ebar_f + Et, T, Tc, Tq, du


def solve(lam, mu, scheme, E_macro, tol=1e-8, maxit=1000, disc="TD", h=1.0, ref=None,
          stop_rule=0, dgo_m=None, dgo_table=None, max_iters_exact=None, dgo_form="polarization",
          dgo_power=2, estar=None, dgo_range="printed"):
    """Solve the periodic cell problem with Algorithm T-3D (disc='TD'), P-3D (disc='PCD') or D-3D (DGO).

    lam, mu: (n3, n2, n1) voxel Lame fields (already sampled at x_i or x_i^c).
    E_macro: 6 tensor components (11,22,33,23,13,12) of the prescribed mean strain.
    max_iters_exact: if set, run exactly that many iterations regardless of tol.
    estar: optional eigenstrain field, (6, n3, n2, n1) tensor components in the same order.  The
    stress-strain relation becomes T = C[E - E_*] and the initial stress of the algorithm
    T^(0) = C_i [E_bar - E_*i] (the generalization stated at the end of Sec. 6); the iteration is
    otherwise unchanged.  Not defined here for Algorithm D.
    """
    lam = np.asarray(lam, np.float64)
    mu = np.asarray(mu, np.float64)
    n3, n2, n1 = lam.shape
    N = lam.size
    lam_h, mu_h = default_reference(lam, mu) if ref is None else ref
    Ebar = voigt_to_tensor(np.asarray(E_macro, np.float64))
    Ebar_f = Ebar[:, :, None, None, None] * np.ones((1, 1, n3, n2, n1))
    if estar is None:
        T0 = stiffness_apply(lam, mu, Ebar_f)
    else:
        T0 = stiffness_apply(lam, mu, Ebar_f - voigt_to_tensor(np.asarray(estar, np.float64)))
    if scheme == "DGO":
        if estar is not None:
            raise ValueError("eigenstrain is not defined for Algorithm D here")
        return _solve_dgo(lam, mu, T0, Ebar, N, h, lam_h, mu_h, tol, maxit, dgo_m, dgo_table, max_iters_exact,
                          dgo_form, dgo_power, dgo_range)
    mats = [dft_matrices(nr, h, disc) for nr in (n1, n2, n3)]
    qa, qb = wave_vectors(scheme, n3, n2, n1, h)
    G = green(qa, qb, lam_h, mu_h)
    k0 = (n3 // 2, n2 // 2, n1 // 2)           # kappa = 0 sits at mu = m + 1
    u = np.zeros((3, n3, n2, n1), dtype=np.complex128)
    du_prev = None
    history = []
    it = 0
    eps = Ebar_f.copy()
    while True:
        it += 1
        eps, T, Tc, Tq, du = _fdd_step(u, Ebar_f, T0, lam, mu, qa, qb, G, mats)
        T0n = np.sqrt(np.sum(np.abs(Tc[(slice(None), slice(None)) + k0]) ** 2))
        eta = _ratio(np.sqrt(np.sum(np.abs(Tq) ** 2)), T0n)
        if stop_rule == 1:
            crit = np.inf if du_prev is None else np.sum(np.sqrt(np.sum(np.abs(du - du_prev) ** 2, axis=0)))
        else:
            crit = eta
        history.append(crit)
        converged = crit < tol
        if max_iters_exact is not None:
            if it >= max_iters_exact:
                break
        elif converged or it >= maxit:
            break
        u = u + du
        du_prev = du
    sig_mean = tensor_to_voigt(T.mean(axis=(-3, -2, -1)))
    # the displacement coefficients u_check that produced eps (the last increment is not added at exit)
    disp = inverse3(u, mats).real
    return Result(tensor_to_voigt(eps), it, history[-1], history, sig_mean, bool(converged), disp)


def _solve_dgo(lam, mu, T0, Ebar, N, h, lam_h, mu_h, tol, maxit, dgo_m, dgo_table, max_iters_exact,
               dgo_form="polarization", dgo_power=2, dgo_range="printed"):
    """Algorithm D-3D with the omega-indexed PCD transforms F^{c+-} (x_i^c = (i - 1/2) h).

    Readings of the weights and the update form:
    dgo_form = "stress": Delta E = Gamma^c T, E += Delta E, the update of Algorithm D-3D.
    dgo_form = "polarization" (default): the form the footnote to Algorithm D-1D ascribes to
    Eloh2019, E_check = Gamma^c [(C - C_H) E]_check, E = E_bar + F^{c+} E_check.
    dgo_power = 1: the weights s of Algorithm D-3D; dgo_power = 2 (default): weights s^2, the
    consistent operator of Brisard2010 on which Eloh2019 builds (the factor (-1)^nu s of the basis
    phi^El, eq. DisPieCon1D, enters once from the trial and once from the test function).
    With s, -Gamma^c C_H is a sum of projections with weights of both signs, so its eigenvalues
    leave [0, 1] and no contraction bound holds: on a 6^3 two-phase cube at contrast 10 both forms
    grow (at contrast 4 they still converge).  With s^2 the eigenvalues lie in [0, 1] and both
    forms converge there; the polarization form reproduces the paper's finding that the DGO
    response is stiffer than AFB/R at high contrast.
    Residual: eta_D = ||E_new - E_old||_2 / (sqrt(N) ||E_bar||_F) (unitary transforms).
    In both forms the iterate returned includes the increment of the last iteration: Algorithm D-3D
    adds Delta E_check to E_check inside the loop body, before the while test.
    dgo_range: the alias range of dgo_operator ("printed" [-m, m-1] or "symmetric" [-m, m]).
    """
    n3, n2, n1 = lam.shape
    mats = [dft_matrices(nr, h, "PCD", index="omega") for nr in (n1, n2, n3)]
    Gc = dgo_operator(n3, n2, n1, h, lam_h, mu_h, dgo_m, dgo_power, dgo_range) if dgo_table is None else dgo_table
    Ec = np.zeros((3, 3, n3, n2, n1), dtype=np.complex128)
    Ebar_f = Ebar[:, :, None, None, None] * np.ones((1, 1, n3, n2, n1))
    enorm = np.sqrt(np.sum(Ebar ** 2)) * np.sqrt(N)
    history = []
    it = 0
    while True:
        it += 1
        Et = inverse3(Ec, mats).real
        eps = Ebar_f + Et
        if dgo_form == "stress":
            T = T0 + stiffness_apply(lam, mu, Et)
            dE = dgo_apply(Gc, forward3(T, mats))
            Ec_new = Ec + dE
        else:
            tau = stiffness_apply(lam - lam_h, mu - mu_h, eps)
            Ec_new = dgo_apply(Gc, forward3(tau, mats))
            dE = Ec_new - Ec
        eta = _ratio(np.sqrt(np.sum(np.abs(dE) ** 2)), enorm)
        history.append(eta)
        converged = eta < tol
        stop = (it >= max_iters_exact) if max_iters_exact is not None else (converged or it >= maxit)
        Ec = Ec_new
        if stop:
            eps = Ebar_f + inverse3(Ec, mats).real
            break
    T = stiffness_apply(lam, mu, eps)
    sig_mean = tensor_to_voigt(T.mean(axis=(-3, -2, -1)))
    return Result(tensor_to_voigt(eps), it, history[-1], history, sig_mean, bool(converged))


def sigma_mean_voigt(res):
    """Macroscopic stress of a solve, tensor components (11,22,33,23,13,12)."""
    return res.sigma_mean


def effective_stiffness(lam, mu, scheme, tol=1e-10, maxit=5000, **kw):
    """C_eff (6x6, Voigt): column J is the mean stress under the Voigt unit strain e_J (shear 1/2)."""
    C = np.zeros((6, 6))
    iters = []
    fields = []
    for J in range(6):
        E = np.zeros(6)
        E[J] = 1.0 if J < 3 else 0.5
        r = solve(lam, mu, scheme, E, tol=tol, maxit=maxit, **kw)
        C[:, J] = r.sigma_mean
        iters.append(r.iters)
        fields.append(r.eps)
    return C, iters, fields


def gradient_closed_form(eps_I, eps_J):
    """d C_eff,IJ / d lambda_i = (1/N) tr eps^I tr eps^J,  d / d mu_i = (2/N) eps^I : eps^J.

    Valid at a converged solution because the compatible fluctuation of one load is orthogonal to
    the equilibrated stress of the other (Gamma real and symmetric), so C_eff,IJ = <eps^I : C : eps^J>.
    """
    N = eps_I[0].size
    trI = eps_I[0] + eps_I[1] + eps_I[2]
    trJ = eps_J[0] + eps_J[1] + eps_J[2]
    dd = eps_I[0] * eps_J[0] + eps_I[1] * eps_J[1] + eps_I[2] * eps_J[2] + 2.0 * (
        eps_I[3] * eps_J[3] + eps_I[4] * eps_J[4] + eps_I[5] * eps_J[5])
    return trI * trJ / N, 2.0 * dd / N


def ceff_entry(lam, mu, scheme, I, J, tol, maxit=10000, ref=None, **kw):
    E = np.zeros(6)
    E[J] = 1.0 if J < 3 else 0.5
    r = solve(lam, mu, scheme, E, tol=tol, maxit=maxit, ref=ref, **kw)
    return r.sigma_mean[I]


def gradient_fd(lam, mu, scheme, I, J, voxels, rel_step=1e-6, tol=1e-13, maxit=20000, **kw):
    """Central finite differences of C_eff,IJ with respect to lambda and mu at the given flat voxel indices.

    The reference medium is frozen at the unperturbed one so that only C(x) changes.
    """
    ref = default_reference(lam, mu)
    gl, gm = [], []
    for v in voxels:
        idx = np.unravel_index(v, lam.shape)
        for field, out in ((0, gl), (1, gm)):
            vals = []
            for sgn in (+1.0, -1.0):
                l2, m2 = lam.copy(), mu.copy()
                base = (l2 if field == 0 else m2)[idx]
                step = rel_step * base
                if field == 0:
                    l2[idx] = base + sgn * step
                else:
                    m2[idx] = base + sgn * step
                vals.append(ceff_entry(l2, m2, scheme, I, J, tol, maxit, ref=ref, **kw))
            out.append((vals[0] - vals[1]) / (2.0 * step))
    return np.array(gl), np.array(gm)
