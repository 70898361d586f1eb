"""The domain decomposition's exchange schedule across processes (Sec. 4: counts and
ghost particles, the global v_max, collision partners of ghosts, migration) on CPU
with the gloo backend, two and three ranks.  Each rank's result is checked against
what the global particle set says it must be."""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _gas(n, seed, Lx):
    rng = np.random.default_rng(seed)
    rows = np.zeros((n, 8))
    rows[:, 0] = np.arange(n)
    rows[:, 1] = rng.random(n) * Lx
    rows[:, 2:4] = rng.random((n, 2)) * 0.25
    rows[:, 4:7] = rng.normal(0, 1, (n, 3))
    rows[:, 7] = rng.integers(0, n, n)
    return rows


def _worker(rank, world, port, periodic, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1310_3437_gb300 import domains as dm

    n, Lx, d0, dt = 3000, 8.0, 0.01, 0.05
    allrows = _gas(n, 5 + world, Lx)
    X = dm.slab_bounds(Lx, world)
    mine = allrows[dm.owner_of(allrows[:, 1], X) == rank]
    D = dm.DomainRank(rank, world, X, mine, periodic, Lx, d0, dt)
    res = {}
    # phase 2: the global maximum speed and the reach
    v = allrows[:, 4:7]
    want_v2 = float(((v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]).max())
    res["vmax2"] = (D.global_vmax2(), want_v2)
    R = dm.reach(D.global_vmax2(), d0, dt)
    # phase 1: the ghosts are every particle of the others within R of this slab
    g = D.exchange_ghosts(R)
    near = dm.slab_distance(allrows[:, 1], X, rank, periodic, Lx) < R
    others = dm.owner_of(allrows[:, 1], X) != rank
    res["ghost_ids"] = (sorted(g[:, 0].astype(int).tolist()),
                        sorted(allrows[near & others, 0].astype(int).tolist()))
    res["ghost_rows_exact"] = bool(np.array_equal(
        g[np.argsort(g[:, 0])], allrows[near & others][np.argsort(allrows[near & others, 0])]))
    res["counts"] = (D.counts_sent, D.counts_received)
    # phase 3: the owners' choices reach every copy of their particles
    choice = {int(i): (int(i) * 7 + 1) % n for i in D.rows[:, 0]}
    got = D.exchange_choices(choice)
    res["choices"] = all(got[int(i)] == (int(i) * 7 + 1) % n for i in g[:, 0]) and \
        len(got) == len(g)
    # phase 4: stream, wrap or reflect at the ends, migrate
    x = D.rows[:, 1] + D.rows[:, 4] * 0.3
    x = np.mod(x, Lx) if periodic else np.abs(x) - 2.0 * np.maximum(np.abs(x) - Lx, 0.0)
    D.rows[:, 1] = x
    D.migrate()
    res["owned_after"] = sorted(D.rows[:, 0].astype(int).tolist())
    res["in_slab"] = bool((dm.owner_of(D.rows[:, 1], X) == rank).all())
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, False), (3, True), (3, False)])
def test_exchange_schedule_gloo(world, periodic):
    port = 29600 + (os.getpid() % 500) + 7 * world + (1 if periodic else 0)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, periodic, out), nprocs=world, join=True)
    owned = []
    for r in range(world):
        res = out[r]
        assert res["vmax2"][0] == res["vmax2"][1]
        got, want = res["ghost_ids"]
        assert got == want and len(want) > 0
        assert res["ghost_rows_exact"]
        sent, received = res["counts"]  # of the ghost exchange: counts first
        for src, c in received.items():
            assert out[src]["counts"][0][r] == c
        assert sum(received.values()) == len(want)
        assert res["choices"]
        assert res["in_slab"]
        owned += res["owned_after"]
    # every particle is owned by exactly one rank after the migration
    assert sorted(owned) == list(range(3000))
