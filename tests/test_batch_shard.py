"""Host logic of the sharded batched homogenization on CPU: two gloo ranks split the cells by cost and
every rank receives the full C_eff.  The local solve is a stub returning seeded per-cell matrices (no GPU)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2009_03762_gb300 import gfp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _expected(i):
    rng = np.random.default_rng(1000 + i)
    return rng.standard_normal((6, 6)), rng.integers(1, 500, size=6)


def _stub_solver(cells, sch, tol, maxit):
    ids = [int(lam.flat[0]) for lam, mu in cells]   # make_cell stores the cell index in lam
    C = np.array([_expected(i)[0] for i in ids]).reshape(-1, 6, 6)
    it = np.array([_expected(i)[1] for i in ids]).reshape(-1, 6)
    return C, it, 0


def _worker(rank, world, port, costs, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2009_03762_gb300 import gfp as G
    dist.init_process_group("gloo")
    make_cell = lambda i: (np.full((2, 2, 2), float(i)), np.ones((2, 2, 2)))
    C, its, rc = G.solve_batch_sharded(make_cell, costs, None, solver=_stub_solver)
    out[rank] = (C, its, rc, G.batch_shard(costs, rank, world))
    dist.destroy_process_group()


def test_batch_shard_is_disjoint_covering_and_balanced():
    costs = [64 ** 3, 96 ** 3, 128 ** 3, 64 ** 3, 128 ** 3, 96 ** 3, 96 ** 3, 64 ** 3, 128 ** 3]
    for world in (1, 2, 3, 4):
        parts = [gfp.batch_shard(costs, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)


def test_two_gloo_ranks_gather_the_full_batch():
    world = 2
    costs = [64 ** 3, 96 ** 3, 128 ** 3, 64 ** 3, 128 ** 3, 96 ** 3, 96 ** 3]
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    exp_C = np.array([_expected(i)[0] for i in range(len(costs))])
    exp_it = np.array([_expected(i)[1] for i in range(len(costs))])
    for r in range(world):
        C, its, rc, mine = out[r]
        assert rc == 0
        np.testing.assert_array_equal(C, exp_C)
        np.testing.assert_array_equal(its, exp_it)
    assert sorted(out[0][3] + out[1][3]) == list(range(len(costs)))
    assert not set(out[0][3]) & set(out[1][3])
