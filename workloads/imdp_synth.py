"""Seeded synthetic IMDP generators.

The paper's 35 benchmark models (Appendix B table) are abstractions of linear
and non-linear systems; their files are not available, so these generators
reproduce their *shapes* (states, actions, transitions) and structure:

* every model has ``n_domain`` grid states plus one absorbing out-of-domain
  sink (the "+1" in every row of the table: 6 = 5 + 1, 241 = 240 + 1, ...);
* column (s, a) has a contiguous window of destination states around
  ``s + drift(a)`` (a Gaussian transition kernel on a 1-D grid) plus the sink,
  which takes the mass that leaves the domain;
* nominal probabilities are normalised Gaussian weights; the bounds are
  ``lower = p (1 - eps u1)``, ``upper = min(1, p (1 + eps u2))`` with
  ``u ~ U(0, 1)``, so every column is feasible by construction;
* the reachability target is a block of grid states in the middle of the
  domain; the sink is absorbing and is not a target.

Everything is drawn from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class IMDPInput:
    """A CSC IMDP plus a reachability target.

    stateptr (n+1), colptr (m+1), rowval (nnz, strictly increasing per column),
    lower/upper (nnz, float64).  ``goal`` holds target state indices (0-based)
    and ``sink`` the absorbing out-of-domain state(s)."""
    n_states: int
    stateptr: np.ndarray
    colptr: np.ndarray
    rowval: np.ndarray
    lower: np.ndarray
    upper: np.ndarray
    goal: np.ndarray
    sink: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    model_state_offsets: Optional[np.ndarray] = None  # for block-diagonal batches

    @property
    def n_cols(self) -> int:
        return int(self.colptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.rowval.size)

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.stateptr, self.colptr, self.rowval, self.lower, self.upper))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _split_total(rng, total: int, parts: int, spread: float, lo: int, hi: int) -> np.ndarray:
    """Integer sizes in [lo, hi] summing exactly to ``total`` (when feasible)."""
    mean = total / parts
    raw = mean * (1.0 + spread * (rng.random(parts) * 2.0 - 1.0))
    k = np.clip(np.floor(raw).astype(np.int64), lo, hi)
    diff = int(total - k.sum())
    order = rng.permutation(parts)
    i = 0
    guard = 0
    while diff != 0 and guard < 64:
        step = 1 if diff > 0 else -1
        room = (hi - k[order]) if step > 0 else (k[order] - lo)
        take = np.minimum(room, abs(diff) // parts + 1)
        take = np.where(np.cumsum(take) <= abs(diff), take, 0)
        if take.sum() == 0:
            # place the remainder one by one
            for j in order:
                if diff == 0:
                    break
                if lo <= k[j] + step <= hi:
                    k[j] += step
                    diff -= step
            guard += 1
            continue
        k[order] += step * take
        diff -= step * int(take.sum())
        i += 1
        guard += 1
    return k


def _banded_core(rng, n_models: int, n_domain, n_actions, kk: np.ndarray, eps: np.ndarray,
                 goal_frac: float = 0.1):
    """Vectorised generator for ``n_models`` models.

    n_domain, n_actions: scalars (all models alike) or one value per model;
    kk: in-domain window length per grid column (models in order, then states,
    then actions); eps: one value per model.  Returns the concatenated
    block-diagonal CSC arrays."""
    nd = np.broadcast_to(np.asarray(n_domain, dtype=np.int64), (n_models,))
    na = np.broadcast_to(np.asarray(n_actions, dtype=np.int64), (n_models,))
    cols_m = nd * na
    colbase = np.zeros(n_models + 1, dtype=np.int64)
    np.cumsum(cols_m, out=colbase[1:])
    N = int(colbase[-1])
    model = np.repeat(np.arange(n_models), cols_m)
    local = np.arange(N) - colbase[model]
    na_c = na[model]
    nd_c = nd[model]
    state = local // na_c
    action = local % na_c
    kk = np.asarray(kk, dtype=np.int64)
    sigma = np.maximum(kk / 4.0, 0.5)
    # actions shift the kernel left/centre/right; jitter keeps columns distinct
    drift = (action - (na_c - 1) / 2.0) * np.maximum(kk / 3.0, 1.0)
    centre = state + drift + rng.normal(0.0, 0.25, N) * sigma
    start = np.clip(np.round(centre - kk / 2.0).astype(np.int64), 0, nd_c - kk)
    # entries per column: window + sink
    cnt = kk + 1
    colstart = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(cnt, out=colstart[1:])
    tot = int(colstart[-1])
    col_of = np.repeat(np.arange(N), cnt)
    pos_in = np.arange(tot) - colstart[col_of]
    is_sink = pos_in == kk[col_of]
    dest = start[col_of] + pos_in
    w = np.exp(-0.5 * ((dest - centre[col_of]) / sigma[col_of]) ** 2)
    w[is_sink] = 0.0
    wsum = np.add.reduceat(w, colstart[:-1])
    dist = np.minimum(centre, (nd_c - 1) - centre)
    leak = 1e-3 + 0.3 * np.exp(-np.maximum(dist, 0.0) / sigma)
    p = np.where(is_sink, leak[col_of], w / wsum[col_of] * (1.0 - leak[col_of]))
    u1 = rng.random(tot)
    u2 = rng.random(tot)
    e = eps[model][col_of]
    lower = p * (1.0 - e * u1)
    upper = np.minimum(1.0, p * (1.0 + e * u2))
    # local -> global destination indices; the sink is the last state of each model
    sbase = np.zeros(n_models + 1, dtype=np.int64)
    np.cumsum(nd + 1, out=sbase[1:])
    base = sbase[model][col_of]
    rowval = np.where(is_sink, base + nd_c[col_of], base + dest).astype(np.int32)

    # insert each model's sink column (self-loop, lower = upper = 1)
    ins_at = colstart[colbase[1:]]  # positions (before insertion) at model ends
    sinks = sbase[:-1] + nd
    rowval = np.insert(rowval, ins_at, sinks.astype(np.int32))
    lower = np.insert(lower, ins_at, 1.0)
    upper = np.insert(upper, ins_at, 1.0)
    cnt_all = np.insert(cnt, colbase[1:], 1)
    colptr = np.zeros(cnt_all.size + 1, dtype=np.int64)
    np.cumsum(cnt_all, out=colptr[1:])
    acts = np.repeat(na, nd + 1)
    acts[sinks] = 1
    stateptr = np.zeros(acts.size + 1, dtype=np.int64)
    np.cumsum(acts, out=stateptr[1:])
    # target block in the middle of each model's domain
    g = np.maximum(1, np.round(goal_frac * nd).astype(np.int64))
    g0 = (nd - g) // 2
    gbase = np.zeros(n_models + 1, dtype=np.int64)
    np.cumsum(g, out=gbase[1:])
    gm = np.repeat(np.arange(n_models), g)
    goal = sbase[gm] + g0[gm] + (np.arange(int(gbase[-1])) - gbase[gm])
    if colptr[-1] >= 2**31:
        raise ValueError("model too large for int32 column pointers")
    return IMDPInput(
        n_states=int(sbase[-1]),
        stateptr=stateptr.astype(np.int32),
        colptr=colptr.astype(np.int32),
        rowval=rowval,
        lower=lower,
        upper=upper,
        goal=goal.astype(np.int32),
        sink=sinks.astype(np.int32),
        model_state_offsets=sbase,
    )


def banded_imdp(n_domain: int, n_actions: int, nnz: int, eps: float = 0.05, spread: float = 0.5,
                seed: int = 0, goal_frac: float = 0.1) -> IMDPInput:
    """One model with ``n_domain + 1`` states, ``n_actions`` actions per grid state
    and exactly ``nnz`` transitions (including the sink self-loop)."""
    rng = _rng(seed)
    cols = n_domain * n_actions
    inner = nnz - 1 - cols  # minus the sink column, minus one sink entry per column
    if inner < cols or inner > cols * n_domain:
        raise ValueError("nnz out of range for this shape")
    kk = _split_total(rng, inner, cols, spread, 1, n_domain)
    return _banded_core(rng, 1, n_domain, n_actions, kk, np.array([eps]), goal_frac)


def banded_batch(n_models: int, n_domain: int, n_actions: int, nnz_per_model: int, eps: float = 0.05,
                 spread: float = 0.5, seed: int = 0, stress_frac: float = 0.0, stress_eps: float = 1e-4,
                 goal_frac: float = 0.1) -> IMDPInput:
    """``n_models`` independent models of the same shape as one block-diagonal IMDP
    (no transition crosses a model boundary).  A fraction ``stress_frac`` of the
    models gets very narrow intervals (``stress_eps``)."""
    rng = _rng(seed)
    cols = n_domain * n_actions
    inner = nnz_per_model - 1 - cols
    if inner < cols or inner > cols * n_domain:
        raise ValueError("nnz out of range for this shape")
    kk = np.concatenate([_split_total(rng, inner, cols, spread, 1, n_domain) for _ in range(min(n_models, 8))])
    reps = -(-n_models // min(n_models, 8))
    kk = np.tile(kk, reps)[: n_models * cols]
    # shuffle sizes between models' columns while keeping each model's total
    eps_m = np.full(n_models, eps)
    if stress_frac > 0:
        eps_m[rng.random(n_models) < stress_frac] = stress_eps
    return _banded_core(rng, n_models, n_domain, n_actions, kk, eps_m, goal_frac)


def _split_models(big: IMDPInput, n_models: int) -> List[IMDPInput]:
    """Cut a block-diagonal IMDP into its independent models (local indices)."""
    out = []
    sb = big.model_state_offsets
    gi = np.searchsorted(big.goal, sb)
    for i in range(n_models):
        s0, s1 = int(sb[i]), int(sb[i + 1])
        c0, c1 = int(big.stateptr[s0]), int(big.stateptr[s1])
        e0, e1 = int(big.colptr[c0]), int(big.colptr[c1])
        out.append(IMDPInput(
            n_states=s1 - s0,
            stateptr=(big.stateptr[s0:s1 + 1] - c0).astype(np.int32),
            colptr=(big.colptr[c0:c1 + 1] - e0).astype(np.int32),
            rowval=(big.rowval[e0:e1] - s0).astype(np.int32),
            lower=big.lower[e0:e1].copy(),
            upper=big.upper[e0:e1].copy(),
            goal=(big.goal[gi[i]:gi[i + 1]] - s0).astype(np.int32),
            sink=np.array([s1 - 1 - s0], np.int32),
            model_state_offsets=np.array([0, s1 - s0], np.int64),
        ))
    return out


def shaped_models(n_domain: np.ndarray, n_actions: np.ndarray, kbar: np.ndarray, eps: np.ndarray,
                  seed: int = 0, chunk: int = 128, threads: int = 0) -> List[IMDPInput]:
    """Independent banded models of per-model shape: ``n_domain[i] + 1`` states,
    ``n_actions[i]`` actions, in-domain windows of about ``kbar[i]`` entries
    (each column's length drawn uniformly within +-50 % of it, clipped to
    [1, n_domain[i]]).  Models are generated in chunks of ``chunk`` with one
    PCG64 stream per chunk (spawned from ``seed``), so the result does not
    depend on ``threads``; numpy releases the GIL in the array work, so a
    thread pool shortens generation of large sets."""
    n = len(n_domain)
    nd = np.asarray(n_domain, np.int64)
    na = np.asarray(n_actions, np.int64)
    kb = np.asarray(kbar, np.float64)
    ep = np.asarray(eps, np.float64)
    bounds = list(range(0, n, chunk)) + [n]
    seqs = np.random.SeedSequence(seed).spawn(len(bounds) - 1)

    def one(ci):
        a, b = bounds[ci], bounds[ci + 1]
        rng = np.random.Generator(np.random.PCG64(seqs[ci]))
        cols = nd[a:b] * na[a:b]
        kc = np.repeat(kb[a:b], cols) * (1.0 + 0.5 * (rng.random(int(cols.sum())) * 2.0 - 1.0))
        kk = np.clip(np.round(kc).astype(np.int64), 1, np.repeat(nd[a:b], cols))
        big = _banded_core(rng, b - a, nd[a:b], na[a:b], kk, ep[a:b])
        return _split_models(big, b - a)

    nchunks = len(bounds) - 1
    if threads and threads > 1 and nchunks > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=threads) as ex:
            parts = list(ex.map(one, range(nchunks)))
    else:
        parts = [one(ci) for ci in range(nchunks)]
    return [m for part in parts for m in part]


def uneven_batch(n_models: int = 10000, seed: int = 7, threads: int = 0):
    """Heterogeneous batch: states ~ U{6..961}, actions ~ U{1..4}, mean
    in-domain window ~ U{2..min(400, states - 1)}, eps in {0.05, 0.1} and
    horizon K ~ U{50..500} per problem (the spread of the table's rows from
    linear_5 to cartpole_960).  Returns (models, horizons)."""
    rng = _rng(seed)
    states = rng.integers(6, 962, n_models)
    nd = states - 1
    na = rng.integers(1, 5, n_models)
    kbar = rng.integers(2, np.minimum(400, nd) + 1)
    eps = rng.choice([0.05, 0.1], n_models)
    horizons = rng.integers(50, 501, n_models).astype(np.int32)
    return shaped_models(nd, na, kbar, eps, seed=seed + 1, threads=threads), horizons


def served_stream(n_requests: int, seed: int = 8, repeat_frac: float = 0.3, threads: int = 0):
    """Request stream for serving: states ~ log-U[50, 4000], actions ~ U{1..3},
    mean window ~ log-U[3, 700] (capped at the domain), K ~ U{100..500}; a
    fraction ``repeat_frac`` of requests re-query an earlier request's model
    with another target block and adversary.  Returns (models, requests) with
    requests as tuples (model index, horizon, pessimistic, goal)."""
    rng = _rng(seed)
    is_new = rng.random(n_requests) >= repeat_frac
    is_new[0] = True
    n_new = int(is_new.sum())
    states = np.exp(rng.uniform(np.log(50), np.log(4000), n_new)).astype(np.int64)
    nd = states - 1
    na = rng.integers(1, 4, n_new)
    kbar = np.minimum(np.exp(rng.uniform(np.log(3), np.log(700), n_new)), nd)
    eps = rng.choice([0.05, 0.1], n_new)
    models = shaped_models(nd, na, kbar, eps, seed=seed + 1, threads=threads)
    reqs = []
    j = -1
    for i in range(n_requests):
        K = int(rng.integers(100, 501))
        if is_new[i]:
            j += 1
            reqs.append((j, K, True, models[j].goal))
        else:
            mi = int(rng.integers(0, j + 1))
            n = models[mi].n_states - 1
            g = max(1, n // 10)
            g0 = int(rng.integers(0, n - g + 1))
            reqs.append((mi, K, bool(rng.random() < 0.5), np.arange(g0, g0 + g, dtype=np.int32)))
    return models, reqs


def random_imdp(n_states: int, max_actions: int = 3, density: float = 0.6, seed: int = 0,
                exact_grid: int = 0, lower_equals_upper: bool = False) -> IMDPInput:
    """Small unstructured IMDP for brute-force checks.  With ``exact_grid > 0``
    every bound is a multiple of 1/exact_grid (exact in binary when the grid is a
    power of two), so exact-rational checkers see the same numbers."""
    rng = _rng(seed)
    acts = rng.integers(1, max_actions + 1, size=n_states)
    stateptr = np.zeros(n_states + 1, dtype=np.int64)
    np.cumsum(acts, out=stateptr[1:])
    rows: List[np.ndarray] = []
    los: List[np.ndarray] = []
    ups: List[np.ndarray] = []
    colptr = [0]
    for _ in range(int(stateptr[-1])):
        mask = rng.random(n_states) < density
        if not mask.any():
            mask[rng.integers(n_states)] = True
        r = np.nonzero(mask)[0]
        p = rng.random(r.size) + 0.05
        p /= p.sum()
        if exact_grid:
            # integer masses summing exactly to exact_grid
            q = np.floor(p * exact_grid).astype(np.int64)
            q[rng.integers(r.size)] += exact_grid - q.sum()
            lo_i = np.maximum(q - rng.integers(0, 3, r.size), 0)
            up_i = np.minimum(q + rng.integers(0, 3, r.size), exact_grid)
            if lower_equals_upper:
                lo_i = up_i = q
            lo, up = lo_i / exact_grid, up_i / exact_grid
        else:
            lo = p * (1 - 0.3 * rng.random(r.size))
            up = np.minimum(1.0, p * (1 + 0.3 * rng.random(r.size)))
            if lower_equals_upper:
                lo = up = p
        rows.append(r.astype(np.int32))
        los.append(lo)
        ups.append(up)
        colptr.append(colptr[-1] + r.size)
    goal = np.array([n_states - 1], dtype=np.int32)
    return IMDPInput(n_states, stateptr.astype(np.int32), np.array(colptr, dtype=np.int32),
                     np.concatenate(rows), np.concatenate(los).astype(np.float64),
                     np.concatenate(ups).astype(np.float64), goal)


def concat_block_diagonal(models: List[IMDPInput]) -> IMDPInput:
    """Concatenate independent models into one block-diagonal IMDP."""
    s_off = np.cumsum([0] + [m.n_states for m in models])
    c_off = np.cumsum([0] + [m.n_cols for m in models])
    e_off = np.cumsum([0] + [m.nnz for m in models])
    stateptr = np.concatenate([m.stateptr[:-1] + c for m, c in zip(models, c_off)] + [[c_off[-1]]])
    colptr = np.concatenate([m.colptr[:-1] + e for m, e in zip(models, e_off)] + [[e_off[-1]]])
    rowval = np.concatenate([m.rowval + s for m, s in zip(models, s_off)])
    goal = np.concatenate([m.goal + s for m, s in zip(models, s_off)])
    sink = np.concatenate([m.sink + s for m, s in zip(models, s_off)])
    return IMDPInput(int(s_off[-1]), stateptr.astype(np.int32), colptr.astype(np.int32),
                     rowval.astype(np.int32), np.concatenate([m.lower for m in models]),
                     np.concatenate([m.upper for m in models]), goal.astype(np.int32), sink.astype(np.int32),
                     model_state_offsets=np.asarray(s_off, dtype=np.int64))


# Synthetic stand-ins for the paper's benchmark shapes (Appendix B table).
# Query for all of them: maximum pessimistic finite-time reachability, K = 200
# (Sec. 5), unless a test says otherwise.
CONFIGS = {
    # linear_5_states_*_0.1_sigma: 6 states, 1 action, 31 transitions
    "linear5": dict(kind="single", n_domain=5, n_actions=1, nnz=31, eps=0.1, seed=0),
    # pendulum_1_layer_240_states_0.05_sigma: 241 states, 1 action, 26321 transitions; 4096 of them
    "pendulum240_x4096": dict(kind="batch", n_models=4096, n_domain=240, n_actions=1, nnz=26321,
                              eps=0.05, seed=1, stress_frac=0.1),
    # cartpole_1_layer_3840_states_0.1_sigma: 3841 states, 1 action, 8614913 transitions
    "cartpole3840": dict(kind="single", n_domain=3840, n_actions=1, nnz=8614913, eps=0.1, seed=4),
    # harrier_25920_states: 25921 states, 1 action, 18574307 transitions
    "harrier": dict(kind="single", n_domain=25920, n_actions=1, nnz=18574307, eps=0.05, seed=5),
    # pimdp_2: 42634 states, 3 actions, 48106480 transitions (the paper's largest model)
    "pimdp2": dict(kind="single", n_domain=42633, n_actions=3, nnz=48106480, eps=0.05, seed=6),
    # dense: every column lists every grid state (plus the sink), as a dense
    # IntervalProbabilities matrix of Sec. 3.1 would; 4096 states, 2 actions
    "dense4096": dict(kind="single", n_domain=4095, n_actions=2, nnz=4095 * 2 * 4095 + 4095 * 2 + 1, eps=0.05,
                      seed=8),
}


def make_config(name: str, **overrides) -> IMDPInput:
    c = dict(CONFIGS[name])
    c.update(overrides)
    if c.pop("kind") == "batch":
        return banded_batch(c["n_models"], c["n_domain"], c["n_actions"], c["nnz"], eps=c["eps"],
                            seed=c["seed"], stress_frac=c.get("stress_frac", 0.0))
    return banded_imdp(c["n_domain"], c["n_actions"], c["nnz"], eps=c["eps"], seed=c["seed"])
