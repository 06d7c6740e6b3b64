"""Adjoint sensitivities through torch.autograd (GfpCeff) and the 128^3 lognormal workload."""
import numpy as np
import pytest

from oracle import gfp_oracle as O
from paper_2009_03762_gb300 import microstructure as M

pytestmark = pytest.mark.gpu


def test_autograd_backward_matches_oracle_closed_form():
    import torch
    from paper_2009_03762_gb300 import gfp
    lam, mu = M.random_field(8, 8, 8, seed=31)
    dev = torch.device("cuda", 0)
    lt = torch.tensor(lam, dtype=torch.float64, device=dev, requires_grad=True)
    mt = torch.tensor(mu, dtype=torch.float64, device=dev, requires_grad=True)
    for (I, J) in ((0, 0), (0, 1), (3, 3)):
        c = gfp.ceff_entry(lt, mt, I, J, "AFB_R", tol=1e-13, maxit=10000)
        gl, gm = torch.autograd.grad(c, (lt, mt))
        ref = O.default_reference(lam, mu)
        EI = np.zeros(6); EI[I] = 1.0 if I < 3 else 0.5
        EJ = np.zeros(6); EJ[J] = 1.0 if J < 3 else 0.5
        rI = O.solve(lam, mu, "AFB_R", EI, tol=1e-13, maxit=10000, ref=ref)
        rJ = O.solve(lam, mu, "AFB_R", EJ, tol=1e-13, maxit=10000, ref=ref)
        ol, om = O.gradient_closed_form(rI.eps, rJ.eps)
        np.testing.assert_allclose(gl.cpu().numpy(), ol, rtol=1e-7, atol=1e-13)
        np.testing.assert_allclose(gm.cpu().numpy(), om, rtol=1e-7, atol=1e-13)
        assert abs(c.item() - rJ.sigma_mean[I]) <= 1e-9 * abs(rJ.sigma_mean[I]) + 1e-14


def test_gradient_32_lognormal_matches_oracle_gradient():
    """The adjoint configuration scaled to 32^3 (cube of edge 16, contrast 10, lognormal(0.1) Lame fields):
    dC_1111/dlambda and /dmu of every voxel from gfp_grad against the oracle's gradient (its closed-form
    contraction of its own converged fields), 1e-7 relative."""
    from paper_2009_03762_gb300 import gfp
    n = 32
    lam, mu = M.sharp_cube(n, 16, 1.0, 10.0)
    lam, mu = M.lognormal_perturb(lam, mu, sigma=0.1, seed=5)
    ref = O.default_reference(lam, mu)
    g = gfp.Grid(n, n, n)
    g.set_phases(lam, mu, ref=ref)
    dl, dm = g.grad(gfp.scheme("AFB_R"), 0, 0, 1e-13, 20000)
    r = O.solve(lam, mu, "AFB_R", [1.0, 0, 0, 0, 0, 0], tol=1e-13, maxit=20000, ref=ref)
    assert r.converged
    ol, om = O.gradient_closed_form(r.eps, r.eps)
    np.testing.assert_allclose(dl, ol, rtol=1e-7, atol=1e-7 * np.abs(ol).max())
    np.testing.assert_allclose(dm, om, rtol=1e-7, atol=1e-7 * np.abs(om).max())
    g.close()


def test_adjoint_128_lognormal_against_finite_differences():
    """128^3 cube (edge 64, contrast 10) with lognormal(0.1) Lame fields: dC_1111/dmu and /dlambda from the
    adjoint contraction against central differences (relative step 1e-6, FP64) on 16 seeded voxels."""
    from paper_2009_03762_gb300 import gfp
    n = 128
    lam, mu = M.sharp_cube(n, 64, 1.0, 10.0)
    lam, mu = M.lognormal_perturb(lam, mu, sigma=0.1, seed=5)
    ref = (0.5 * (lam.min() + lam.max()), 0.5 * (mu.min() + mu.max()))
    g = gfp.Grid(n, n, n)
    g.set_phases(lam, mu, ref=ref)
    sch = gfp.scheme("AFB_R")
    dl, dm = g.grad(sch, 0, 0, 1e-12, 20000)
    rng = np.random.default_rng(16)
    vox = rng.choice(lam.size, size=16, replace=False)
    E = [1.0, 0, 0, 0, 0, 0]
    errs = []
    for v in vox:
        idx = np.unravel_index(v, lam.shape)
        for field, grad in ((0, dl), (1, dm)):
            vals = []
            base = (lam if field == 0 else mu)[idx]
            hstep = 1e-6 * base
            for sgn in (1.0, -1.0):
                l2, m2 = lam.copy(), mu.copy()
                (l2 if field == 0 else m2)[idx] = base + sgn * hstep
                g.set_phases(l2, m2, ref=ref)
                # a fixed iteration count keeps the perturbed maps smooth (the difference then cancels the
                # iteration error); 600 iterations are far below the 1e-12 residual for this cell
                r = g.solve(sch, E, 0.0, 600)
                vals.append(r.sigma_mean[0])
            fd = (vals[0] - vals[1]) / (2 * hstep)
            errs.append(abs(fd - grad[idx]) / abs(grad[idx]))
    # A one-voxel perturbation moves C_1111 by ~1e-6 / N ~ 5e-13 relative; the FP64 solve forms the mean
    # stress by a compensated real-space sum (the k = 0 value of the transform rounds at ~4e-16, which
    # alone would put ~1e-3 of noise on a central difference), so every voxel must agree to 1e-3.
    assert max(errs) <= 1e-3, errs
