"""Sharding of a chemistry step over ranks, on CPU processes with the gloo backend (no GPU).

Two ranks split a field of cells by predicted cost, advance their shares with the FP64 oracle
(the per-cell computation is independent of the partition), gather the results and max-reduce
their step times; the gathered field must equal the unpartitioned computation bit for bit.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_23993_gb300.shard import gather_field, max_over_ranks, partition_by_cost


def test_partition_is_a_balanced_cover():
    rng = np.random.default_rng(0)
    cost = np.concatenate([np.ones(950), rng.integers(2, 400, 50)]).astype(float)
    for world in (1, 2, 3, 8):
        parts = partition_by_cost(cost, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(cost.size))
        loads = np.array([cost[p].sum() for p in parts])
        # LPT bound: the largest load exceeds the mean by at most the largest unit
        assert loads.max() <= cost.sum() / world + cost.max()
        assert all(np.all(np.diff(p) > 0) for p in parts)
    assert partition_by_cost(cost, 2)[0].tolist() == partition_by_cost(cost, 2)[0].tolist()


def _field():
    import synth
    mech = synth.h2_air_mechanism(0)
    T, p, Y, hot = synth.slab_field(mech, n=4, slab=(1, 2))   # 64 cells, a hot slab of 32
    return mech, T, p, Y, hot


def _advance(mech, T, p, Y, idx):
    import oracle
    rho, e = oracle.state_from_TpY(mech, T[idx], p[idx], Y[:, idx])
    T1, _, Y1, _ = oracle.advance(mech, rho, e, T[idx], Y[:, idx], 1e-8)
    return np.column_stack([T1, Y1.T])


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mech, T, p, Y, hot = _field()
        cost = np.where(hot, 300.0, 1.0)               # predicted substeps
        parts = partition_by_cost(cost, world)
        local = _advance(mech, T, p, Y, parts[rank])
        full = gather_field(local, parts, T.size, dist)
        t = max_over_ranks(1.0 + rank, dist)
        if rank == 0:
            np.save(out_path, full)
            assert t == float(world)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo_step_equals_unpartitioned(tmp_path):
    out = str(tmp_path / "full.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    full = np.load(out)
    mech, T, p, Y, hot = _field()
    ref = _advance(mech, T, p, Y, np.arange(T.size))
    assert np.array_equal(full, ref)
    # the two shares carry equal predicted cost
    parts = partition_by_cost(np.where(hot, 300.0, 1.0), 2)
    assert abs(hot[parts[0]].sum() - hot[parts[1]].sum()) <= 1
