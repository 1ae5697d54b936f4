"""State-sharded finite-horizon value iteration: one model split over the ranks
of a process group (one GPU per rank).

Every rank owns a contiguous range of states (``imdp_partition_states``, about
equal work per rank), holds the columns of those states only
(``imdp_create_csc_slice``) and runs one session on that slice. After each
Bellman step (Eq. 2) the ranks all-gather their owned values, so that every
slice holds the complete V_k before step k + 1; the per-state problems are
independent within an iteration (Sec. 4), so the result equals the unsharded
one word for word. The exchange moves the raw 64-bit iterates (8 bytes per
state and step) through ``torch.distributed`` (NCCL between GPUs).
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence

import numpy as np

from . import _binding as B


def gather_slices(own, lengths: Sequence[int], rank: int, group=None) -> List:
    """All-gather variable-length 1-D int64 tensors: rank r contributes ``own``
    (``lengths[r]`` words); returns every rank's slice (views of one buffer).
    Slices are padded to the longest one, as all-gather moves equal blocks."""
    import torch
    import torch.distributed as dist
    world = len(lengths)
    width = max(int(x) for x in lengths)
    buf = torch.zeros(width, dtype=torch.int64, device=own.device)
    buf[: own.numel()] = own
    parts = [torch.empty(width, dtype=torch.int64, device=own.device) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return [parts[r][: int(lengths[r])] for r in range(world)]


class SliceRunner:
    """One slice of a state-sharded problem, stepped one iteration at a time.

    ``m``: the whole model's host CSC arrays (n_states, stateptr, colptr, rowval,
    lower, upper); ``bounds``: the partition; ``spec_kw``: the finite-horizon
    specification (``make_spec`` keywords, identical on every rank)."""

    def __init__(self, m, bounds: Sequence[int], part: int, spec_kw: dict, dtype=B.IMDP_F64, stream=None,
                 device=None):
        import torch
        if spec_kw.get("infinite_time"):
            raise ValueError("state-sharded iteration runs finite horizons only")
        self.bounds = [int(b) for b in bounds]
        self.part = part
        self.s0, self.s1 = self.bounds[part], self.bounds[part + 1]
        self.stream = stream
        self.horizon = int(spec_kw.get("horizon", 100))
        self.model = B.create_model_slice(m, self.s0, self.s1, dtype, stream)
        self.spec = B.make_spec(**spec_kw)
        self.session = B.imdp_session_create([self.model], [self.spec], stream=stream)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.own = torch.empty(self.s1 - self.s0, dtype=torch.int64, device=dev)
        self.k = 0

    def reset(self):
        B.imdp_session_reset(self.session, self.stream)
        self.k = 0

    def step(self):
        """One Bellman iteration of the owned states; returns V_k on them (raw words)."""
        B.imdp_session_step(self.session, 1, self.stream)
        self.k += 1
        B.imdp_session_values_get(self.session, 0, self.k, self.s0, self.s1, self.own, self.stream)
        return self.own

    def put(self, slices: Sequence):
        """Write the other parts' V_k (``slices[r]`` for part r) into this slice."""
        for r, x in enumerate(slices):
            if r != self.part and x.numel():
                B.imdp_session_values_put(self.session, 0, self.k, self.bounds[r], self.bounds[r + 1], x,
                                          self.stream)

    def read(self, V_out, k_out=None):
        return B.imdp_session_read(self.session, 0, V_out, k_out, stream=self.stream)

    def close(self):
        self.session.close()
        self.model.close()


def run_sharded(m, spec_kw: dict, rank: int, world: int, group=None, dtype=B.IMDP_F64, stream=None,
                exchange: Optional[Callable] = None):
    """Finite-horizon value iteration of model ``m`` sharded over ``world`` ranks;
    returns (V as a host float64 array, iterations). ``exchange(own, lengths,
    rank)`` defaults to an all-gather over ``group``."""
    import torch
    bounds = B.imdp_partition_states(m.n_states, m.stateptr, m.colptr, world)
    runner = SliceRunner(m, bounds, rank, spec_kw, dtype, stream)
    lengths = np.diff(bounds)
    ex = exchange or (lambda own, lens, r: gather_slices(own, lens, r, group))
    try:
        runner.reset()
        for _ in range(runner.horizon):
            own = runner.step()
            if world > 1:
                if stream is not None:
                    stream.synchronize()  # `own` is complete before the exchange reads it
                slices = ex(own, lengths, rank)
                if stream is not None:
                    stream.wait_stream(torch.cuda.current_stream())  # the exchange ran on torch's stream
                runner.put(slices)
        V = np.zeros(m.n_states)
        k = [0]
        runner.read(V, k)
        if stream is not None:
            stream.synchronize()
        torch.cuda.synchronize()
        return V, k[0]
    finally:
        runner.close()
