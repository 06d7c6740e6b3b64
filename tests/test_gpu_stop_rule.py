"""The paper's stopping rule on the GPU (stop_rule = 1): the L1 norm over the modes of the difference of
successive displacement increments, sum_mu |du^(it) - du^(it-1)| (Algorithms T-3D / P-3D), against the
oracle's literal evaluation of it (complex G_H per mode, unitary transforms)."""
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


@pytest.mark.parametrize("op,shape", [("AFB_R", (16, 12, 8)), ("AHC", (12, 12, 12)), ("CD", (9, 27, 9)),
                                      ("ACD", (27, 9, 9)), ("AFB_R", (32, 32, 32))])
def test_increment_rule_matches_oracle(gfp, op, shape):
    n1, n2, n3 = shape
    lam, mu = M.random_field(n1, n2, n3, seed=n1 + n2)
    E = [0.01, -0.002, 0.0, 0.003, 0.0, 0.001]
    tol = 1e-9
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    r = g.solve(gfp.scheme(op, "TD", "FP64", stop_rule=1), E, tol, 5000, history=True)
    ref = O.solve(lam, mu, op, E, tol=tol, maxit=5000, stop_rule=1)
    assert r.converged and ref.converged
    assert r.iters == ref.iters, (r.iters, ref.iters)
    h = np.asarray(r.history[:r.iters])
    assert np.isinf(h[0]) and np.isinf(ref.history[0])
    # the criterion is a difference of successive increments: its rounding floor is that of the
    # increments themselves, about 1e-16 of the early criterion values
    np.testing.assert_allclose(h[1:], ref.history[1:], rtol=1e-8, atol=1e-13 * np.max(ref.history[1:]))
    eps = g.strain()
    assert np.linalg.norm(eps - ref.eps) <= 1e-10 * np.linalg.norm(ref.eps)
    assert abs(r.residual - ref.residual) <= 1e-8 * ref.residual + 1e-13 * np.max(ref.history[1:])
    g.close()


def test_increment_rule_unsupported_combinations(gfp):
    lam, mu = M.random_field(8, 8, 8, seed=4)
    g = gfp.Grid(8, 8, 8)
    g.set_phases(lam, mu)
    for op, prec in (("F", "FP64"), ("HC", "FP64"), ("AFB_R", "MIXED"), ("DGO", "FP64")):
        with pytest.raises(gfp.GfpError) as e:
            g.solve(gfp.scheme(op, "PCD", prec, stop_rule=1), [0.01, 0, 0, 0, 0, 0], 1e-8, 100, raise_on_error=True)
        assert e.value.code == -8
    g.close()
