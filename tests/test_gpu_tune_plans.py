"""Radix schedules of the shared-memory Stockham passes chosen by the autotuner (gfp_tune) and set
explicitly (gfp_set_plans): any valid schedule gives the oracle's iterates; invalid ones are refused."""
import functools

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


SHAPE = (48, 54, 24)  # n1, n2, n3: lengths without a register-FFT plan


def _cell():
    n1, n2, n3 = SHAPE
    return M.random_field(n1, n2, n3, seed=17)


@functools.lru_cache(maxsize=None)
def _oracle(op, E):
    lam, mu = _cell()
    return O.solve(lam, mu, op, list(E), tol=1e-10, maxit=3000, disc="PCD")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def test_tuned_radix_schedules_are_valid_and_keep_the_iterates(gfp, tmp_path):
    lam, mu = _cell()
    n1, n2, n3 = SHAPE
    E = [0.01, -0.002, 0.0, 0.001, 0.0, 0.002]
    sch = gfp.scheme("AFB_R", "PCD", "FP64")
    ref = _oracle("AFB_R", tuple(E))
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    before = g.get_plans(gfp.FP64)
    cache = str(tmp_path / "tune.json")
    g.tune(sch, iters=2, cache=cache)
    after = g.get_plans(gfp.FP64)
    for p, n in zip(after, SHAPE):
        assert int(np.prod(p)) == n and all(r in (2, 3, 4, 8, 16) for r in p)
    r = g.solve(sch, E, 1e-10, 3000)
    assert r.converged and r.iters == ref.iters
    assert _rel(g.strain(), ref.eps) <= 1e-10
    # the cache restores the same schedules on a fresh grid
    g2 = gfp.Grid(n1, n2, n3)
    g2.set_phases(lam, mu)
    assert g2.get_plans(gfp.FP64) == before
    g2.tune(sch, cache=cache)
    assert g2.get_plans(gfp.FP64) == after
    g.close()
    g2.close()


@pytest.mark.parametrize("plans", [[[3, 4, 4], [3, 2, 3, 3], [2, 4, 3]], [[2, 8, 3], [3, 3, 3, 2], [3, 8]],
                                   [[16, 3], [2, 3, 3, 3], [8, 3]]])
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_explicit_radix_schedules_match_oracle(gfp, plans, prec):
    lam, mu = _cell()
    n1, n2, n3 = SHAPE
    E = [0.0, 0.0, 0.0, 0.0, 0.0, 0.5]
    ref = _oracle("ACD", tuple(E))
    g = gfp.Grid(n1, n2, n3)
    g.set_phases(lam, mu)
    g.set_plans(gfp.FP64 if prec == "FP64" else gfp.MIXED, plans)
    r = g.solve(gfp.scheme("ACD", "PCD", prec), E, 1e-10, 3000)
    assert r.converged
    if prec == "FP64":
        assert r.iters == ref.iters
        assert _rel(g.strain(), ref.eps) <= 1e-10
    else:
        assert _rel(r.sigma_mean, ref.sigma_mean) <= 1e-6
    g.close()


def test_invalid_radix_schedules_are_refused(gfp):
    n1, n2, n3 = SHAPE
    g = gfp.Grid(n1, n2, n3)
    lam, mu = _cell()
    g.set_phases(lam, mu)
    good = g.get_plans(gfp.FP64)
    for bad in ([[16, 4], good[1], good[2]], [good[0], [6, 9], good[2]], [good[0], good[1], [2] * 13]):
        with pytest.raises(gfp.GfpError) as e:
            g.set_plans(gfp.FP64, bad)
        assert e.value.code == -1
    assert g.get_plans(gfp.FP64) == good
    g.close()
