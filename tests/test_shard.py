"""State sharding on the CPU: the partition (a host-only C-ABI call), the slice
arrays, and the variable-length all-gather over two gloo ranks. The device side
(slices iterated and exchanged on a GPU) is in test_shard_gpu.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_2401_04068_gb300 as g
from paper_2401_04068_gb300 import build as pbuild
from workloads import banded_imdp, random_imdp



@pytest.fixture(scope="module", autouse=True)
def _library():
    return pbuild.build()  # incremental; the partition call needs no device


def _work(m):
    sp, cp = m.stateptr, m.colptr
    nnz = cp[sp[1:]] - cp[sp[:-1]]
    return 20.0 * nnz + 12.0 * np.diff(sp) + 20.0


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_partition_covers_and_balances(parts):
    m = banded_imdp(3000, 3, 3000 * 3 * 60 + 1, seed=5)
    b = g.imdp_partition_states(m.n_states, m.stateptr, m.colptr, parts)
    assert b[0] == 0 and b[-1] == m.n_states and np.all(np.diff(b) > 0)
    w = _work(m)
    per = np.array([w[b[i]:b[i + 1]].sum() for i in range(parts)])
    # each part within one state's work of the ideal share
    assert np.max(np.abs(per - w.sum() / parts)) <= w.max() + 1e-9


def test_partition_uneven_states_and_limits():
    # one heavy state among light ones: every part still gets a state
    m = random_imdp(12, max_actions=3, seed=3)
    b = g.imdp_partition_states(m.n_states, m.stateptr, m.colptr, 12)
    assert np.array_equal(b, np.arange(13))
    with pytest.raises(g.ImdpError) as e:
        g.imdp_partition_states(m.n_states, m.stateptr, m.colptr, 13)
    assert e.value.status == g.IMDP_EINVAL
    with pytest.raises(g.ImdpError):
        g.imdp_partition_states(m.n_states, m.stateptr, m.colptr, 0)


def test_slice_arrays_reassemble_the_model():
    m = banded_imdp(500, 2, 500 * 2 * 20 + 1, seed=4)
    b = g.imdp_partition_states(m.n_states, m.stateptr, m.colptr, 3)
    sps, cps, rvs, los, ups = [], [], [], [], []
    col_off = ent_off = 0
    for i in range(3):
        sp, cp, rv, lo, up = g.slice_arrays(m, b[i], b[i + 1])
        assert sp[0] == 0 and sp[-1] == len(cp) - 1 and cp[0] == 0 and cp[-1] == len(rv)
        sps.append(sp[:-1] + col_off)
        cps.append(cp[:-1] + ent_off)
        col_off += len(cp) - 1
        ent_off += len(rv)
        rvs.append(rv), los.append(lo), ups.append(up)
    assert np.array_equal(np.concatenate(sps + [[col_off]]), m.stateptr)
    assert np.array_equal(np.concatenate(cps + [[ent_off]]), m.colptr)
    assert np.array_equal(np.concatenate(rvs), m.rowval)
    assert np.array_equal(np.concatenate(los), m.lower) and np.array_equal(np.concatenate(ups), m.upper)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gather_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2401_04068_gb300.sharded import gather_slices
        lengths = [5, 3]
        full = torch.arange(1, 9, dtype=torch.int64) * (1 << 40) + 7  # 8 words, 64-bit values survive
        bounds = np.concatenate([[0], np.cumsum(lengths)])
        own = full[bounds[rank]:bounds[rank + 1]].clone()
        parts = gather_slices(own, lengths, rank)
        out[rank] = torch.cat(parts).tolist()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gather_slices_two_gloo_ranks_uneven():
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_gather_main, args=(2, port, out), nprocs=2, start_method="spawn")
    want = (np.arange(1, 9, dtype=np.int64) * (1 << 40) + 7).tolist()
    assert out[0] == want and out[1] == want


class _ChainSlice:
    """A CPU stand-in for one slice: value iteration of a Markov chain (the
    lower == upper special case of Eq. 2) on raw integer words, owned rows only."""

    def __init__(self, P, goal, bounds, part, eps_raw, cap):
        self.P, self.goal, self.bounds, self.part = P, goal, bounds, part
        self.s0, self.s1 = bounds[part], bounds[part + 1]
        self.infinite, self.eps_raw, self.horizon = True, eps_raw, cap

    def reset(self):
        n = self.P.shape[0]
        self.V = np.where(np.isin(np.arange(n), self.goal), 1 << 40, 0).astype(np.int64)
        self.prev = self.V.copy()
        self.k = 0

    def step(self):
        self.prev = self.V.copy()
        new = self.V.copy()
        for s in range(self.s0, self.s1):
            if s not in self.goal:
                new[s] = int(np.rint(self.P[s] @ self.V.astype(np.float64)))
        self.V = new
        self.k += 1
        return torch.from_numpy(self.V[self.s0:self.s1].copy())

    def residual(self):
        d = np.abs(self.V[self.s0:self.s1] - self.prev[self.s0:self.s1])
        return torch.tensor([int(d.max()) if d.size else 0], dtype=torch.int64)

    def sync(self):
        pass

    def put(self, slices):
        for r, x in enumerate(slices):
            if r != self.part:
                self.V[self.bounds[r]:self.bounds[r + 1]] = x.numpy()


def _chain(n=60, seed=3):
    # a random walk on 0..n-2 that leaks a tenth of its mass per step into the
    # absorbing state n-1 (value 0): values converge geometrically
    rng = np.random.default_rng(seed)
    P = np.zeros((n, n))
    for s in range(n - 1):
        nb = [max(0, s - 1), s, min(n - 2, s + 1)]
        w = rng.random(3) + 0.1
        for j, x in zip(nb, 0.9 * w / w.sum()):
            P[s, j] += x
        P[s, n - 1] += 0.1
    P[n - 1, n - 1] = 1.0
    return P, np.array([n // 2], np.int64)


def _drive_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2401_04068_gb300.sharded import drive, gather_slices_and_residual
        P, goal = _chain()
        bounds = [0, 23, 60]
        runner = _ChainSlice(P, goal, bounds, rank, eps_raw=1 << 12, cap=100000)
        k = drive(runner, lambda own, res, lens, r: gather_slices_and_residual(own, res, lens, r),
                  np.diff(bounds), rank)
        out[rank] = (k, runner.V.tolist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_infinite_horizon_stops_with_the_unsharded_run():
    # two gloo ranks drive the sharded loop: the residual of each slice rides in
    # its all-gather block, every rank takes the maximum and stops after the
    # same iteration as one process iterating the whole chain, with the same words
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_drive_main, args=(2, port, out), nprocs=2, start_method="spawn")
    P, goal = _chain()
    whole = _ChainSlice(P, goal, [0, 60], 0, eps_raw=1 << 12, cap=100000)
    whole.reset()
    while True:
        whole.step()
        if int(whole.residual()[0]) < (1 << 12):
            break
    assert out[0][0] == out[1][0] == whole.k > 5
    assert out[0][1] == out[1][1] == whole.V.tolist()
