"""Failure detection without a GPU fault: a bounded device wait that is made to run out reports
GFP_ERR_DEVICE_TIMEOUT and leaves the CUDA context usable."""
import numpy as np
import pytest

from oracle import gfp_oracle as O
from paper_2009_03762_gb300 import microstructure as M

pytestmark = pytest.mark.gpu


def test_tma_wait_timeout_is_reported_and_context_survives():
    from paper_2009_03762_gb300 import gfp
    L = gfp.lib()
    lam, mu = M.random_field(32, 32, 32, seed=8)
    g = gfp.Grid(32, 32, 32)
    g.set_phases(lam, mu)
    g.set_tiles(gfp.FP64, [0, 8, -4])           # TMA-fed z-pass, 4 columns
    sch = gfp.scheme("AFB_R")
    E = [0.01, 0, 0, 0, 0, 0]
    assert L.gfp_set_fault_injection(1, 1) == 0
    try:
        r = g.solve(sch, E, 1e-8, 3)
    except gfp.GfpError as e:
        r = None
        code = e.code
    finally:
        assert L.gfp_set_fault_injection(1, 0) == 0
    assert (r.status if r is not None else code) == -6
    # the context is intact: the same grid solves correctly afterwards
    r2 = g.solve(sch, E, 0.0, 3)
    ref = O.solve(lam, mu, "AFB_R", E, max_iters_exact=3)
    assert r2.iters == 3
    assert np.linalg.norm(g.strain() - ref.eps) / np.linalg.norm(ref.eps) <= 1e-10
    assert L.gfp_set_fault_injection(7, 1) == -1
    assert L.gfp_set_fault_injection(1, 64) == -1
