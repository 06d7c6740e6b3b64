"""The allocation-free entry point gfp_solve_noalloc against the regular gfp_solve.

Some callers cannot allocate GPU memory (their device memory is owned by a host framework's pool,
or cudaMalloc's device-wide synchronisation is not acceptable where they run), so the library offers
one solve whose scratch is a fixed device array inside the library.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2009_03762_gb300 import microstructure as M

pytestmark = pytest.mark.gpu
REL = 1e-10


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def test_noalloc_matches_regular_solve_on_two_calls():
    import torch
    from paper_2009_03762_gb300 import gfp
    gfp.lib()
    dev = torch.device("cuda", 0)
    cases = [((16, 24, 18), "AFB_R", [0.01, 0.0, -0.002, 0.0, 0.003, 0.0]),
             ((32, 32, 32), "ACD", [0.0, 0.0, 0.0, 0.5, 0.0, 0.0])]
    for (n3, n2, n1), op, E in cases:     # two calls in a row share the library's scratch
        lam, mu = M.random_spheres((n1, n2, n3), vf=0.2, rmin=2.0, rmax=4.0, contrast=10.0, seed=n1)
        ref_r, ref_eps = gfp.solve(lam, mu, op, E, tol=1e-9, maxit=3000)
        assert ref_r.converged
        lam_t = torch.from_numpy(lam).to(dev)
        mu_t = torch.from_numpy(mu).to(dev)
        eps_t = torch.empty((6, n3, n2, n1), dtype=torch.float64, device=dev)
        rc, r = gfp.solve_noalloc(lam_t, mu_t, eps_t, gfp.scheme(op), E, tol=1e-9, maxit=3000)
        torch.cuda.synchronize()
        assert rc == 0 and r.iters == ref_r.iters, (rc, r.iters, r.residual, ref_r.iters, ref_r.residual)
        assert _rel(eps_t.cpu().numpy(), ref_eps) <= REL
        assert _rel(r.sigma_mean, ref_r.sigma_mean) <= REL


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2009_03762_gb300 import gfp
    dev = torch.device("cuda", 0)
    lam_t = torch.ones((64, 64, 64), dtype=torch.float64, device=dev)
    eps_t = torch.empty((6, 64, 64, 64), dtype=torch.float64, device=dev)
    with pytest.raises(gfp.GfpError) as e:
        gfp.solve_noalloc(lam_t, lam_t, eps_t, gfp.scheme("AFB_R"), [0.01, 0, 0, 0, 0, 0])
    assert e.value.code == -2
    assert b"scratch" in gfp.lib().gfp_last_error_detail()


def test_noalloc_call_allocates_no_device_memory():
    """After a first call (which looks up the scratch's device address and loads the kernels it uses), a
    repeated call leaves both the device's free memory and torch's allocator untouched."""
    import torch
    from paper_2009_03762_gb300 import gfp
    dev = torch.device("cuda", 0)
    n3, n2, n1 = 16, 24, 18
    lam, mu = M.random_spheres((n1, n2, n3), vf=0.2, rmin=2.0, rmax=4.0, contrast=10.0, seed=5)
    lam_t = torch.from_numpy(lam).to(dev)
    mu_t = torch.from_numpy(mu).to(dev)
    eps_t = torch.empty((6, n3, n2, n1), dtype=torch.float64, device=dev)
    E = [0.01, 0.0, 0.0, 0.0, 0.0, 0.002]
    rc0, r0 = gfp.solve_noalloc(lam_t, mu_t, eps_t, gfp.scheme("AFB_R"), E, tol=1e-9, maxit=3000)
    torch.cuda.synchronize()
    first = eps_t.cpu().numpy()
    free0, alloc0 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_allocated(dev)
    rc1, r1 = gfp.solve_noalloc(lam_t, mu_t, eps_t, gfp.scheme("AFB_R"), E, tol=1e-9, maxit=3000)
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_allocated(dev)
    assert rc0 == rc1 == 0 and r0.iters == r1.iters
    assert (free1, alloc1) == (free0, alloc0)
    np.testing.assert_array_equal(eps_t.cpu().numpy(), first)


def test_noalloc_rejects_mismatched_shapes_before_the_call():
    import torch
    from paper_2009_03762_gb300 import gfp
    dev = torch.device("cuda", 0)
    lam_t = torch.ones((8, 8, 8), dtype=torch.float64, device=dev)
    short = torch.ones((8, 8, 4), dtype=torch.float64, device=dev)
    eps_t = torch.empty((6, 8, 8, 8), dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        gfp.solve_noalloc(lam_t, short, eps_t, gfp.scheme("AFB_R"), [0.01, 0, 0, 0, 0, 0])
    with pytest.raises(ValueError):
        gfp.solve_noalloc(lam_t, lam_t, eps_t[:3], gfp.scheme("AFB_R"), [0.01, 0, 0, 0, 0, 0])
