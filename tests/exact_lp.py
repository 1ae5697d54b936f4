"""Exact-rational reference computations used to pin the oracle.

Independent of O-maximization: the inner problem of Eq. 3,
``opt_{p in Gamma} sum_i v_i p_i`` over ``{lower <= p <= upper, sum p = 1}``
(Sec. 2, definition of Gamma_{s,a}), is solved here by enumerating the
vertices of that polytope.  A vertex has every coordinate at one of its
bounds except at most one, which is then fixed by the simplex constraint, so
enumerating (free index, bound pattern) pairs visits every vertex.  The LP
optimum is attained at a vertex.

Also here: the two O-maximization procedures printed in Sec. 4 (sequential and
cumulative-sum form), restated in exact rationals so a test can check that
they agree with each other and with the LP optimum.
"""
from __future__ import annotations

from fractions import Fraction as Fr
from itertools import product
from typing import List, Sequence, Tuple


def lp_vertex_opt(v: Sequence[Fr], lo: Sequence[Fr], up: Sequence[Fr], minimize: bool) -> Fr:
    k = len(v)
    best = None
    cands = []
    for free in [None] + list(range(k)):
        others = [i for i in range(k) if i != free]
        for pattern in product((0, 1), repeat=len(others)):
            p = [None] * k
            s = Fr(0)
            for i, b in zip(others, pattern):
                p[i] = up[i] if b else lo[i]
                s += p[i]
            if free is None:
                if s != 1:
                    continue
            else:
                pf = 1 - s
                if pf < lo[free] or pf > up[free]:
                    continue
                p[free] = pf
            cands.append(sum(vi * pi for vi, pi in zip(v, p)))
    if not cands:
        raise ValueError("infeasible column")
    best = min(cands) if minimize else max(cands)
    return best


def omax_sequential(order: Sequence[int], lo: Sequence[Fr], up: Sequence[Fr]) -> List[Fr]:
    """Sequential procedure of Sec. 4 (exact)."""
    p = list(lo)
    rem = 1 - sum(lo)
    for o in order:
        gap = up[o] - lo[o]
        if gap < rem:
            p[o] += gap
            rem -= gap
        else:
            p[o] += rem
            break
    return p


def omax_prefix(order: Sequence[int], lo: Sequence[Fr], up: Sequence[Fr]) -> List[Fr]:
    """Cumulative-sum form of Sec. 4 (exact): each position's remaining budget is
    rem minus the inclusive prefix of gaps plus its own gap."""
    p = list(lo)
    rem = 1 - sum(lo)
    gaps = [up[o] - lo[o] for o in order]
    cum = []
    acc = Fr(0)
    for g in gaps:
        acc += g
        cum.append(acc)
    for i, o in enumerate(order):
        rem_state = max(rem - cum[i] + gaps[i], Fr(0))
        p[o] += gaps[i] if gaps[i] < rem_state else rem_state
    return p


def exact_value_iteration(n: int, cols: List[List[Tuple[int, Fr, Fr]]], stateptr: Sequence[int],
                          goal: Sequence[int], K: int, pessimistic: bool, maximize: bool,
                          avoid: Sequence[int] = (), reward=None, discount=None):
    """Eq. 2 in exact rationals with the LP solved by vertex enumeration.
    cols[j] = [(dest, lower, upper), ...].  Returns the list V_0..V_K and the
    per-iteration list of optimal action sets (set of local indices)."""
    goal = set(goal)
    avoid = set(avoid)
    if reward is None:
        V = [Fr(1) if s in goal else Fr(0) for s in range(n)]
    else:
        V = [Fr(r) for r in reward]
    hist = [V]
    argsets = []
    for _ in range(K):
        Vn = []
        acts = []
        for s in range(n):
            if reward is None and s in goal:
                Vn.append(Fr(1)); acts.append(set()); continue
            if reward is None and s in avoid:
                Vn.append(Fr(0)); acts.append(set()); continue
            qs = []
            for j in range(stateptr[s], stateptr[s + 1]):
                d = [e[0] for e in cols[j]]
                qs.append(lp_vertex_opt([V[x] for x in d], [e[1] for e in cols[j]], [e[2] for e in cols[j]],
                                        minimize=pessimistic))
            best = max(qs) if maximize else min(qs)
            acts.append({i for i, q in enumerate(qs) if q == best})
            Vn.append(best if reward is None else Fr(reward[s]) + Fr(discount) * best)
        V = Vn
        hist.append(V)
        argsets.append(acts)
    return hist, argsets


def columns_from_csc(colptr, rowval, lower, upper, exact_values=None):
    """Exact rational columns from CSC arrays.  ``exact_values`` (optional) maps
    entry index -> (Fraction lower, Fraction upper); otherwise the binary value of
    each float is used exactly."""
    cols = []
    for j in range(len(colptr) - 1):
        c = []
        for i in range(colptr[j], colptr[j + 1]):
            if exact_values is not None:
                lo, up = exact_values[i]
            else:
                lo, up = Fr(float(lower[i])), Fr(float(upper[i]))
            c.append((int(rowval[i]), lo, up))
        cols.append(c)
    return cols
