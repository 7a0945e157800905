"""Replica ensembles split over ranks (host logic of the N > 1 path), on CPU.

Two gloo ranks each simulate their share of a small ensemble with the oracle;
the per-replica results gathered on rank 0 must be bit-identical to one
process simulating the whole ensemble, and the timing aggregate must be the
slowest rank's time over the units of all ranks.
"""
import multiprocessing
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2604_14307_gb300 import inputs as I
from paper_2604_14307_gb300 import replicas as RP

STEPS = 2


def ensemble():
    """Five uneven boxes with one 162-site sphere each (shape of the batched
    single-colloid workload, small enough for the oracle)."""
    return I.batched_single_sphere(n_rep=5, precision=I.P32, seed=3, Ls=(6, 8))


def per_replica(system, st):
    so, bo = system.solvent_offsets(), system.body_offsets()
    sid = system.stream_ids()
    return {int(sid[r]): (st.x[so[r]:so[r + 1]].copy(), st.v[so[r]:so[r + 1]].copy(),
                          st.P[bo[r]:bo[r + 1]].copy(), st.Lm[bo[r]:bo[r + 1]].copy())
            for r in range(system.n_rep)}


def run_oracle(system):
    st = I.initial_state(system)
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st)
    O.step(osys, ost, STEPS)
    st.x, st.v, st.P, st.Lm = ost.x, ost.v, ost.P, ost.Lm
    return per_replica(system, st)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = RP.local_system(ensemble(), world, rank)
        out = run_oracle(local)
        parts = [None] * world
        dist.all_gather_object(parts, out)
        agg = RP.aggregate_timing(ms_local=10.0 + 5.0 * rank, units_local=100.0 * (rank + 1))
        if rank == 0:
            q.put((parts, agg))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_is_a_balanced_partition():
    rng = np.random.default_rng(0)
    costs = rng.integers(1, 100, size=37).astype(float)
    for world in (1, 2, 3, 8):
        parts = RP.shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [costs[p].sum() for p in parts]
        assert max(loads) - min(loads) <= costs.max()       # LPT bound
        assert parts == RP.shard(costs, world)              # same split on every rank
    assert RP.shard([5.0, 5.0], 4)[2:] == [[], []]


def test_subset_starts_from_the_same_state():
    full = ensemble()
    a = per_replica(full, I.initial_state(full))
    for ids in ([3, 1], [4], [0, 2]):
        sub = full.subset(ids)
        b = per_replica(sub, I.initial_state(sub))
        for sid, arrs in b.items():
            for u, w in zip(arrs, a[sid]):
                assert np.array_equal(u, w)


def test_two_gloo_ranks_reproduce_the_single_process_ensemble():
    O.build()
    ref = run_oracle(ensemble())
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts, agg = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = {}
    for part in parts:
        assert not (set(part) & set(got))                    # every replica on one rank only
        got.update(part)
    assert sorted(got) == sorted(ref)
    for sid in ref:
        for u, w in zip(got[sid], ref[sid]):
            assert np.array_equal(u, w), sid
    assert agg["ms"] == 15.0 and agg["units"] == 300.0
    assert agg["per_s"] == pytest.approx(300.0 / 0.015)
