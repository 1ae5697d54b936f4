"""State-sharded value iteration: one model split over the ranks of a process
group (one GPU per rank).

Every rank owns a contiguous range of states (``imdp_partition_states``, about
equal work per rank), holds the columns of those states only
(``imdp_create_csc_slice``) and runs one session on that slice. After each
Bellman step (Eq. 2) the ranks all-gather their owned values, so that every
slice holds the complete V_k before step k + 1; the per-state problems are
independent within an iteration (Sec. 4), so the result equals the unsharded
one word for word. The exchange moves the raw 64-bit iterates (8 bytes per
state and step) through ``torch.distributed`` (NCCL between GPUs).

An infinite horizon stops on the maximum Bellman residual over all states, so
each rank appends the residual of its own states (one word) to its block of the
all-gather: every rank then holds every slice's residual, takes their maximum
(the all-reduce(max) of the residual, with no collective of its own) and stops
after the same iteration as the unsharded run.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import _binding as B

_I64_MAX = (1 << 63) - 1


def gather_slices(own, lengths: Sequence[int], rank: int, group=None) -> List:
    """All-gather variable-length 1-D int64 tensors: rank r contributes ``own``
    (``lengths[r]`` words); returns every rank's slice (views of one buffer).
    Slices are padded to the longest one, as all-gather moves equal blocks."""
    slices, _ = gather_slices_and_residual(own, None, lengths, rank, group)
    return slices


def gather_slices_and_residual(own, residual, lengths: Sequence[int], rank: int,
                               group=None) -> Tuple[List, Optional[int]]:
    """As gather_slices; with ``residual`` (a one-word int64 tensor: this rank's
    maximum |V_k - V_{k-1}| as a raw word) also returns the maximum over all
    ranks, carried in one extra word of every block."""
    import torch
    import torch.distributed as dist
    world = len(lengths)
    width = max(int(x) for x in lengths) + (1 if residual is not None else 0)
    buf = torch.zeros(width, dtype=torch.int64, device=own.device)
    buf[: own.numel()] = own
    if residual is not None:
        # raw residuals lie in [0, 2^63]: 2^63 reads as a negative int64, and any
        # residual that large fails every threshold below 1, as its clamp does
        r = residual.reshape(1)
        buf[width - 1:] = torch.where(r < 0, torch.full_like(r, _I64_MAX), r)
    parts = [torch.empty(width, dtype=torch.int64, device=own.device) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    slices = [parts[r][: int(lengths[r])] for r in range(world)]
    if residual is None:
        return slices, None
    return slices, int(max(int(p[width - 1]) for p in parts))


class SliceRunner:
    """One slice of a state-sharded problem, stepped one iteration at a time.

    ``m``: the whole model's host CSC arrays (n_states, stateptr, colptr, rowval,
    lower, upper); ``bounds``: the partition; ``spec_kw``: the specification
    (``make_spec`` keywords, identical on every rank); ``launch``: launch
    configuration keywords of the slice's session (``imdp_session_set_launch``;
    None: by rule)."""

    def __init__(self, m, bounds: Sequence[int], part: int, spec_kw: dict, dtype=B.IMDP_F64, stream=None,
                 device=None, launch: Optional[dict] = None):
        import torch
        self.bounds = [int(b) for b in bounds]
        self.part = part
        self.s0, self.s1 = self.bounds[part], self.bounds[part + 1]
        self.stream = stream
        self.infinite = bool(spec_kw.get("infinite_time"))
        h = int(spec_kw.get("horizon", 100))
        self.horizon = (h if h > 0 else 1000000) if self.infinite else h
        self.model = B.create_model_slice(m, self.s0, self.s1, dtype, stream)
        self.spec = B.make_spec(**spec_kw)
        self.session = B.imdp_session_create([self.model], [self.spec], stream=stream)
        if launch:
            B.imdp_session_set_launch(self.session, stream=stream, **launch)
        self.eps_raw = B.imdp_session_stop_threshold(self.session, 0) if self.infinite else None
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.own = torch.empty(self.s1 - self.s0, dtype=torch.int64, device=dev)
        self.res = torch.zeros(1, dtype=torch.int64, device=dev)
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

    def residual(self):
        """max |V_k - V_{k-1}| over the owned states (one raw word, device)."""
        B.imdp_session_residual(self.session, 0, self.k, self.s0, self.s1, self.res, self.stream)
        return self.res

    def put(self, slices: Sequence):
        """Write the other parts' V_k (``slices[r]`` for part r) into this slice."""
        for r, x in enumerate(slices):
            if r != self.part and x.numel():
                if self.stream is not None:
                    x.record_stream(self.stream)  # read there after the exchange's stream lets go of it
                B.imdp_session_values_put(self.session, 0, self.k, self.bounds[r], self.bounds[r + 1], x,
                                          self.stream)

    def sync(self):
        """Order the exchange after this step on the device: the exchange runs on
        torch's current stream, which waits for the slice's stream (the host does
        not block; a residual read on the host waits by itself)."""
        if self.stream is not None:
            import torch
            torch.cuda.current_stream().wait_stream(self.stream)

    def wait(self):
        """Block the host until the slice's work is done."""
        if self.stream is not None:
            self.stream.synchronize()

    def read(self, V_out, k_out=None):
        return B.imdp_session_read(self.session, 0, V_out, k_out, stream=self.stream, check=False)

    def close(self):
        self.session.close()
        self.model.close()


def drive(runner, exchange: Callable, lengths: Sequence[int], rank: int) -> int:
    """The sharded iteration loop, independent of where the runner computes:
    step, exchange the owned values (and, for an infinite horizon, the residuals),
    stop at the horizon or on the all-slice residual test. Returns the
    iterations performed. ``exchange(own, residual_or_None, lengths, rank)``
    returns (slices, maximum residual or None)."""
    runner.reset()
    for _ in range(runner.horizon):
        own = runner.step()
        res = runner.residual() if runner.infinite else None
        runner.sync()  # the exchange reads `own` and the residual after the step writes them
        slices, rmax = exchange(own, res, lengths, rank)
        runner.put(slices)
        if runner.infinite and rmax < runner.eps_raw:
            break
    return runner.k


def run_sharded(m, spec_kw: dict, rank: int, world: int, group=None, dtype=B.IMDP_F64, stream=None,
                exchange: Optional[Callable] = None):
    """Value iteration of model ``m`` sharded over ``world`` ranks; returns (V as
    a host float64 array, iterations). ``exchange(own, residual, lengths, rank)``
    defaults to the all-gather over ``group``."""
    import torch
    bounds = B.imdp_partition_states(m.n_states, m.stateptr, m.colptr, world)
    runner = SliceRunner(m, bounds, rank, spec_kw, dtype, stream)
    lengths = np.diff(bounds)

    def default_exchange(own, res, lens, r):
        slices, rmax = gather_slices_and_residual(own, res, lens, r, group)
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())  # the exchange ran on torch's stream
        return slices, rmax

    try:
        k = drive(runner, exchange or default_exchange, lengths, rank)
        V = np.zeros(m.n_states)
        kk = [0]
        runner.read(V, kk)
        runner.wait()
        torch.cuda.synchronize()
        assert kk[0] == k
        return V, k
    finally:
        runner.close()
