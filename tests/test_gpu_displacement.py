"""Displacement output u^p = F^+ u_check (the primary unknown of Algorithms T/P) recovered on the GPU
from the strain, against the oracle's accumulated displacement and the AFD difference relation."""
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


@pytest.mark.parametrize("op,shape", [("AFB_R", (8, 8, 8)), ("AFB_R", (6, 9, 12)), ("AFB_R", (32, 32, 32)),
                                      ("AHC", (9, 3, 27)), ("ACD", (9, 3, 27)), ("F", (9, 3, 27)),
                                      ("CD", (27, 9, 3)), ("HC", (3, 27, 9))])
def test_displacement_matches_oracle(gfp, op, shape):
    """Four iterations, then the displacement of that state, element by element."""
    n3, n2, n1 = shape
    lam, mu = M.random_field(n1, n2, n3, seed=23)
    E = [0.004, -0.002, 0.003, 0.001, -0.001, 0.002]
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    sch = gfp.scheme(op, "PCD", "FP64")
    g.solve(sch, E, 0.0, 4)
    u = g.displacement(sch)
    ref = O.solve(lam, mu, op, E, max_iters_exact=4)
    assert _rel(g.strain(), ref.eps) <= REL
    assert _rel(u, ref.disp) <= REL, _rel(u, ref.disp)
    g.close()


def test_displacement_laminate_forward_difference(gfp):
    """AFB/R on a laminate along x1 (64 layers): the forward differences of u_1 and u_2 along x1 give back
    eps_11 - E_11 and 2 (eps_12 - E_12) exactly; zero-mean displacement."""
    lam, mu = M.random_laminate(64, 32, 32, seed=3)
    E = np.array([0.004, -0.002, 0.003, 0.001, -0.002, 0.005])
    g = gfp.Grid(64, 32, 32)
    g.set_phases(lam, mu)
    sch = gfp.scheme("AFB_R", "PCD", "FP64")
    r = g.solve(sch, E, 1e-12, 20000)
    assert r.converged
    u = g.displacement(sch)
    eps = g.strain()
    d1 = np.roll(u[0], -1, axis=2) - u[0]
    d2 = np.roll(u[1], -1, axis=2) - u[1]
    np.testing.assert_allclose(d1, eps[0] - E[0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(d2, 2 * (eps[5] - E[5]), rtol=0, atol=1e-14)
    assert abs(u.mean()) < 1e-15
    g.close()


def test_displacement_errors(gfp):
    lam, mu = M.random_field(8, 8, 8, seed=1)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    with pytest.raises(gfp.GfpError) as e:
        g.displacement(gfp.scheme("AFB_R"))   # no solve yet
    assert e.value.code == -1
    with pytest.raises(ValueError):
        g.displacement(gfp.scheme("AFB_R"), out=np.empty((3, 8, 8, 7)))
    g.close()


def test_displacement_into_device_memory(gfp):
    """The displacement written to a CUDA tensor equals the host copy."""
    torch = pytest.importorskip("torch")
    lam, mu = M.random_field(8, 8, 8, seed=2)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    sch = gfp.scheme("AFB_R", "PCD", "FP64")
    g.solve(sch, [0.002, 0, 0, 0, 0, 0.001], 1e-10, 5000)
    u_host = g.displacement(sch)
    u_dev = torch.empty((3, 8, 8, 8), dtype=torch.float64, device="cuda")
    g.displacement(sch, out=u_dev)
    np.testing.assert_array_equal(u_dev.cpu().numpy(), u_host)
    g.close()
