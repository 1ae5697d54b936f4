"""Pins for the CPU oracle against what the paper and the mathematics fix.

Nothing here re-types the oracle's own formulae: the expected values come from
(a) the LP definition of the inner problem solved by vertex enumeration in exact
rationals, (b) textbook reductions (lower == upper gives an MDP / Markov chain,
solved with dense numpy matrix products), (c) closed forms (gambler's ruin,
geometric reward sums), and (d) invariants of robust value iteration.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from exact_lp import (columns_from_csc, exact_value_iteration, lp_vertex_opt, omax_prefix,
                      omax_sequential)
from workloads import banded_imdp, random_imdp

MODES = [(True, True), (True, False), (False, True), (False, False)]  # (pessimistic, maximize)


def _om(m):
    return oracle.OracleIMDP(m.n_states, m.stateptr, m.colptr, m.rowval, m.lower, m.upper)


def _om_dict(d):
    return oracle.OracleIMDP(d["n_states"], d["stateptr"], d["colptr"], d["rowval"], d["lower"], d["upper"])


# --------------------------------------------------------------------------- worked example (Sec. 3.1)

def test_worked_example_first_step_by_hand(worked_example):
    # V_1 for goal {state 3}, pessimistic, maximize, worked out from Eq. 2 with the
    # LP of Eq. 3: state 1 keeps 1/5 of the mass on the goal under a1 (1/10 under
    # a2); state 2 keeps 3/10 under a1 and 2/5 under a2.
    ex = worked_example
    st, V, k, res, pol = oracle.value_iteration(_om_dict(ex), oracle.OracleSpec(horizon=1, reach=ex["goal"]),
                                                policy=True)
    assert st == "ok" and k == 1
    np.testing.assert_allclose(V, [0.2, 0.4, 1.0], atol=1e-15)
    assert list(pol[0]) == [0, 1, -1]


@pytest.mark.parametrize("pess,maxi", MODES)
def test_worked_example_matches_exact_lp(worked_example, pess, maxi):
    ex = worked_example
    cols = columns_from_csc(ex["colptr"], ex["rowval"], ex["lower"], ex["upper"], exact_values=ex["exact"])
    K = 12
    hist, argsets = exact_value_iteration(ex["n_states"], cols, ex["stateptr"], ex["goal"], K, pess, maxi)
    for k in (1, 2, 3, 5, 12):
        st, V, kk, res, pol = oracle.value_iteration(
            _om_dict(ex), oracle.OracleSpec(horizon=k, reach=ex["goal"], pessimistic=pess, maximize=maxi),
            policy=True)
        assert st == "ok" and kk == k
        np.testing.assert_allclose(V, [float(x) for x in hist[k]], rtol=0, atol=1e-14)
        np.testing.assert_allclose(res, [float(a - b) for a, b in zip(hist[k], hist[k - 1])], atol=1e-14)
        # policy column t is the optimal action of iteration k - t
        for t in range(k):
            for s in range(ex["n_states"]):
                opts = argsets[k - t - 1][s]
                if not opts:
                    assert pol[t][s] == -1
                elif len(opts) == 1:
                    assert pol[t][s] in opts


def test_worked_example_full_horizon(worked_example):
    ex = worked_example
    cols = columns_from_csc(ex["colptr"], ex["rowval"], ex["lower"], ex["upper"], exact_values=ex["exact"])
    hist, _ = exact_value_iteration(ex["n_states"], cols, ex["stateptr"], ex["goal"], ex["horizon"], True, True)
    st, V, k, res, _ = oracle.value_iteration(_om_dict(ex), oracle.OracleSpec(horizon=ex["horizon"],
                                                                              reach=ex["goal"]))
    assert k == 100
    np.testing.assert_allclose(V, [float(x) for x in hist[100]], atol=1e-14)
    # hand-derived second step, from the LP by vertex enumeration
    assert hist[1] == [Fr(1, 5), Fr(2, 5), Fr(1)]
    assert hist[2] == [Fr(21, 50), Fr(29, 50), Fr(1)]


# --------------------------------------------------------------------------- the O-maximization procedure

def _rand_column(rng, k, den=64):
    q = rng.multinomial(den, np.ones(k) / k)
    lo = np.maximum(q - rng.integers(0, 4, k), 0)
    up = np.minimum(q + rng.integers(0, 4, k), den)
    v = rng.integers(0, 8, k) / 8.0  # ties on purpose
    return v, lo / den, up / den


def test_omax_listings_agree_with_lp_exactly():
    rng = np.random.default_rng(7)
    for trial in range(400):
        k = int(rng.integers(1, 6))
        v, lo, up = _rand_column(rng, k)
        V = [Fr(x) for x in v]
        L = [Fr(x) for x in lo]
        U = [Fr(x) for x in up]
        for pess in (True, False):
            order = sorted(range(k), key=lambda i: (V[i] if pess else -V[i], i))
            p1 = omax_sequential(order, L, U)
            p2 = omax_prefix(order, L, U)
            assert p1 == p2
            assert sum(p1) == 1 and all(L[i] <= p1[i] <= U[i] for i in range(k))
            lp = lp_vertex_opt(V, L, U, minimize=pess)
            assert sum(a * b for a, b in zip(V, p1)) == lp


def test_oracle_omax_column_is_lp_optimum():
    rng = np.random.default_rng(11)
    for trial in range(400):
        k = int(rng.integers(1, 7))
        v, lo, up = _rand_column(rng, k)
        for pess in (True, False):
            q, p = oracle.omax_column(v, lo, up, pessimistic=pess)
            lp = lp_vertex_opt([Fr(x) for x in v], [Fr(x) for x in lo], [Fr(x) for x in up], minimize=pess)
            assert abs(q - float(lp)) < 1e-15
            assert abs(p.sum() - 1.0) < 1e-15
            assert np.all(p >= lo - 1e-16) and np.all(p <= up + 1e-16)


def test_omax_degenerate_columns():
    # a single entry with lower = upper = 1 (absorbing): q = v
    q, p = oracle.omax_column(np.array([0.3]), np.array([1.0]), np.array([1.0]))
    assert q == pytest.approx(0.3) and p[0] == 1.0
    # lower == upper: no freedom
    v = np.array([0.1, 0.9, 0.5])
    lo = np.array([0.25, 0.25, 0.5])
    q, p = oracle.omax_column(v, lo, lo)
    assert q == pytest.approx(0.1 * 0.25 + 0.9 * 0.25 + 0.5 * 0.5)
    # all values equal: any feasible p gives the same value
    q, _ = oracle.omax_column(np.full(4, 0.7), np.zeros(4), np.ones(4))
    assert q == pytest.approx(0.7)
    # empty intervals below, all freedom: pessimistic puts all mass on the minimum
    q, _ = oracle.omax_column(np.array([0.4, 0.1, 0.8]), np.zeros(3), np.ones(3), pessimistic=True)
    assert q == pytest.approx(0.1)
    q, _ = oracle.omax_column(np.array([0.4, 0.1, 0.8]), np.zeros(3), np.ones(3), pessimistic=False)
    assert q == pytest.approx(0.8)


# --------------------------------------------------------------------------- brute force on tiny IMDPs

@pytest.mark.parametrize("seed", range(6))
def test_tiny_random_imdp_vs_exact(seed):
    m = random_imdp(5, max_actions=3, density=0.7, seed=seed, exact_grid=32)
    assert oracle.validate(_om(m)) == "ok"
    cols = columns_from_csc(m.colptr, m.rowval, m.lower, m.upper)
    K = 5
    for pess, maxi in MODES:
        hist, argsets = exact_value_iteration(m.n_states, cols, m.stateptr, m.goal, K, pess, maxi)
        st, V, k, res, pol = oracle.value_iteration(
            _om(m), oracle.OracleSpec(horizon=K, reach=m.goal, pessimistic=pess, maximize=maxi), policy=True)
        np.testing.assert_allclose(V, [float(x) for x in hist[K]], atol=1e-14)
        for t in range(K):
            for s in range(m.n_states):
                if argsets[K - t - 1][s]:
                    assert pol[t][s] in argsets[K - t - 1][s]


@pytest.mark.parametrize("seed", range(3))
def test_tiny_reach_avoid_and_reward_vs_exact(seed):
    m = random_imdp(5, max_actions=2, density=0.8, seed=100 + seed, exact_grid=16)
    cols = columns_from_csc(m.colptr, m.rowval, m.lower, m.upper)
    K = 4
    hist, _ = exact_value_iteration(m.n_states, cols, m.stateptr, [4], K, True, True, avoid=[0])
    st, V, k, _, _ = oracle.value_iteration(
        _om(m), oracle.OracleSpec(property=oracle.REACH_AVOID, horizon=K, reach=[4], avoid=[0]))
    assert st == "ok"
    np.testing.assert_allclose(V, [float(x) for x in hist[K]], atol=1e-14)
    r = [Fr(1, 2), Fr(1), Fr(3, 2), Fr(2), Fr(-1, 4)]
    hist, _ = exact_value_iteration(m.n_states, cols, m.stateptr, [], K, False, True, reward=r,
                                    discount=Fr(3, 4))
    st, V, k, _, _ = oracle.value_iteration(
        _om(m), oracle.OracleSpec(property=oracle.REWARD, horizon=K, reward=np.array([float(x) for x in r]),
                                  discount=0.75, pessimistic=False))
    assert st == "ok"
    np.testing.assert_allclose(V, [float(x) for x in hist[K]], atol=1e-13)


# --------------------------------------------------------------------------- textbook reductions

def _dense_actions(m):
    """lower == upper: one transition matrix per local action index (padding with
    the first action where a state has fewer actions)."""
    n = m.n_states
    amax = int(np.max(np.diff(m.stateptr)))
    P = np.zeros((amax, n, n))
    for s in range(n):
        na = m.stateptr[s + 1] - m.stateptr[s]
        for a in range(amax):
            j = m.stateptr[s] + min(a, na - 1)
            for i in range(m.colptr[j], m.colptr[j + 1]):
                P[a, s, m.rowval[i]] = m.lower[i]
    return P


@pytest.mark.parametrize("maxi", [True, False])
def test_lower_equals_upper_is_an_mdp(maxi):
    m = random_imdp(30, max_actions=3, density=0.3, seed=3, lower_equals_upper=True)
    P = _dense_actions(m)
    G = np.zeros(m.n_states, bool)
    G[m.goal] = True
    V = G.astype(float)
    K = 40
    for _ in range(K):
        Q = P @ V  # (actions, states)
        V = np.where(G, 1.0, Q.max(0) if maxi else Q.min(0))
    for pess in (True, False):  # the adversary has no freedom
        st, Vo, k, _, _ = oracle.value_iteration(
            _om(m), oracle.OracleSpec(horizon=K, reach=m.goal, pessimistic=pess, maximize=maxi))
        np.testing.assert_allclose(Vo, V, atol=1e-13)


def _gamblers_ruin(N, p):
    """Birth-death chain on {0..N}: up with p, down with 1-p; 0 and N absorbing."""
    stateptr = np.arange(N + 2, dtype=np.int32)
    colptr, rowval, prob = [0], [], []
    for s in range(N + 1):
        if s in (0, N):
            rowval += [s]; prob += [1.0]
        else:
            rowval += [s - 1, s + 1]; prob += [1 - p, p]
        colptr.append(len(rowval))
    return oracle.OracleIMDP(N + 1, stateptr, np.array(colptr), np.array(rowval), np.array(prob),
                             np.array(prob))


@pytest.mark.parametrize("p", [0.4, 0.5, 0.6])
def test_infinite_horizon_gamblers_ruin_closed_form(p):
    N = 12
    m = _gamblers_ruin(N, p)
    st, V, k, res, pol = oracle.value_iteration(
        m, oracle.OracleSpec(infinite_time=True, eps=1e-13, horizon=10**6, reach=[N]), policy=True)
    assert st == "ok"
    i = np.arange(N + 1)
    if p == 0.5:
        exact = i / N
    else:
        r = (1 - p) / p
        exact = (1 - r ** i) / (1 - r ** N)
    np.testing.assert_allclose(V, exact, atol=1e-10)
    assert np.max(np.abs(res)) < 1e-13
    assert pol[0][N] == -1 and np.all(pol[0][:N] == 0)


def test_reward_closed_forms():
    # absorbing self-loop with reward r: V_K = r * sum_{i=0..K} gamma^i
    m = oracle.OracleIMDP(1, np.array([0, 1]), np.array([0, 1]), np.array([0]), np.array([1.0]), np.array([1.0]))
    for K, g in [(0, 0.9), (1, 0.9), (25, 0.95), (100, 0.5)]:
        st, V, k, _, _ = oracle.value_iteration(
            m, oracle.OracleSpec(property=oracle.REWARD, horizon=K, reward=np.array([2.0]), discount=g))
        assert st == "ok" and k == K
        assert V[0] == pytest.approx(2.0 * (1 - g ** (K + 1)) / (1 - g), rel=1e-14)
    # infinite horizon: r / (1 - gamma)
    st, V, k, _, _ = oracle.value_iteration(
        m, oracle.OracleSpec(property=oracle.REWARD, infinite_time=True, eps=1e-12, horizon=10**6,
                             reward=np.array([2.0]), discount=0.9))
    assert st == "ok" and V[0] == pytest.approx(20.0, abs=1e-10)


def test_reward_markov_chain_matrix_recursion():
    m = random_imdp(20, max_actions=1, density=0.4, seed=9, lower_equals_upper=True)
    P = _dense_actions(m)[0]
    r = np.linspace(-1, 2, m.n_states)
    V = r.copy()
    for _ in range(30):
        V = r + 0.9 * P @ V
    st, Vo, k, _, _ = oracle.value_iteration(
        _om(m), oracle.OracleSpec(property=oracle.REWARD, horizon=30, reward=r, discount=0.9))
    np.testing.assert_allclose(Vo, V, atol=1e-12)


def test_reach_avoid_markov_chain():
    m = random_imdp(25, max_actions=1, density=0.3, seed=12, lower_equals_upper=True)
    P = _dense_actions(m)[0]
    G = np.zeros(m.n_states, bool); G[[24, 3]] = True
    A = np.zeros(m.n_states, bool); A[[0, 7]] = True
    V = G.astype(float)
    for _ in range(15):
        V = np.where(G, 1.0, np.where(A, 0.0, P @ V))
    st, Vo, _, _, _ = oracle.value_iteration(
        _om(m), oracle.OracleSpec(property=oracle.REACH_AVOID, horizon=15, reach=[24, 3], avoid=[0, 7]))
    np.testing.assert_allclose(Vo, V, atol=1e-13)


# --------------------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def banded():
    return banded_imdp(300, 2, 300 * 2 * 20 + 300 * 2 + 1, eps=0.1, seed=21)


def _vi(m, **kw):
    sp = oracle.OracleSpec(reach=m.goal, **kw)
    st, V, k, res, pol = oracle.value_iteration(_om(m), sp, policy=True)
    assert st == "ok"
    return V, res, pol


def test_invariants_bounds_monotone_order(banded):
    m = banded
    Vpm, res, _ = _vi(m, horizon=30)
    assert np.all(Vpm >= 0) and np.all(Vpm <= 1)
    assert np.all(res >= -1e-15)  # V_k nondecreasing for reachability from 1_G
    Vom, _, _ = _vi(m, horizon=30, pessimistic=False)
    Vpn, _, _ = _vi(m, horizon=30, maximize=False)
    assert np.all(Vom >= Vpm - 1e-15) and np.all(Vpm >= Vpn - 1e-15)
    V20, _, _ = _vi(m, horizon=20)
    assert np.all(Vpm >= V20 - 1e-15)


def test_invariant_widening_intervals(banded):
    m = banded
    import copy
    w = copy.copy(m)
    w.lower = m.lower * 0.9
    w.upper = np.minimum(1.0, m.upper * 1.1)
    Vp, _, _ = _vi(m, horizon=25)
    Vpw, _, _ = _vi(w, horizon=25)
    Vo, _, _ = _vi(m, horizon=25, pessimistic=False)
    Vow, _, _ = _vi(w, horizon=25, pessimistic=False)
    assert np.all(Vpw <= Vp + 1e-15) and np.all(Vow >= Vo - 1e-15)


def test_invariant_state_permutation(banded):
    m = banded
    rng = np.random.default_rng(0)
    n = m.n_states
    perm = rng.permutation(n)  # new label of old state s is perm[s]
    inv = np.argsort(perm)
    stateptr = [0]; colptr = [0]; rows = []; lo = []; up = []
    for t in range(n):
        s = inv[t]
        for j in range(m.stateptr[s], m.stateptr[s + 1]):
            a, b = m.colptr[j], m.colptr[j + 1]
            r = perm[m.rowval[a:b]]
            o = np.argsort(r)
            rows += list(r[o]); lo += list(m.lower[a:b][o]); up += list(m.upper[a:b][o])
            colptr.append(len(rows))
        stateptr.append(len(colptr) - 1)
    pm = oracle.OracleIMDP(n, np.array(stateptr), np.array(colptr), np.array(rows), np.array(lo), np.array(up))
    st, Vp, _, _, _ = oracle.value_iteration(pm, oracle.OracleSpec(horizon=20, reach=perm[m.goal]))
    V, _, _ = _vi(m, horizon=20)
    np.testing.assert_allclose(Vp[perm], V, atol=1e-14)


def test_invariant_nonexpansive(banded):
    # one Bellman step T applied to arbitrary W via the reward recursion with
    # gamma = 1 and K = 1: V_1 = W + T(W)  =>  T(W) = V_1 - W.
    m = banded
    rng = np.random.default_rng(5)
    def T(W):
        st, V, _, _, _ = oracle.value_iteration(
            _om(m), oracle.OracleSpec(property=oracle.REWARD, horizon=1, reward=W, discount=1.0))
        return V - W
    for _ in range(5):
        A = rng.random(m.n_states)
        B = np.clip(A + rng.normal(0, 0.05, m.n_states), 0, 1)
        assert np.max(np.abs(T(A) - T(B))) <= np.max(np.abs(A - B)) + 1e-14


def test_infinite_horizon_stopping_rule(banded):
    m = banded
    eps = 1e-6
    st, V, k, res, pol = oracle.value_iteration(
        _om(m), oracle.OracleSpec(infinite_time=True, eps=eps, horizon=100000, reach=m.goal), policy=True)
    assert st == "ok" and np.max(np.abs(res)) < eps
    # the previous iteration had not yet converged
    Vf, resf, _ = _vi(m, horizon=k - 1)
    assert np.max(np.abs(resf)) >= eps
    Vk, _, _ = _vi(m, horizon=k)
    np.testing.assert_array_equal(Vk, V)


def test_policy_time_indexing(banded):
    m = banded
    _, _, pol30 = _vi(m, horizon=30)
    for t in (0, 5, 29):
        _, _, pol_short = _vi(m, horizon=30 - t)
        np.testing.assert_array_equal(pol30[t], pol_short[0])


def test_dense_and_sparse_storage_agree():
    # storing structural zeros explicitly must not change anything
    m = random_imdp(8, max_actions=2, density=0.5, seed=4)
    n = m.n_states
    colptr = [0]; rows = []; lo = []; up = []
    for j in range(m.n_cols):
        d = dict(zip(m.rowval[m.colptr[j]:m.colptr[j + 1]],
                     zip(m.lower[m.colptr[j]:m.colptr[j + 1]], m.upper[m.colptr[j]:m.colptr[j + 1]])))
        for s in range(n):
            l, u = d.get(s, (0.0, 0.0))
            rows.append(s); lo.append(l); up.append(u)
        colptr.append(len(rows))
    dm = oracle.OracleIMDP(n, m.stateptr, np.array(colptr), np.array(rows), np.array(lo), np.array(up))
    for pess, maxi in MODES:
        sp = oracle.OracleSpec(horizon=10, reach=m.goal, pessimistic=pess, maximize=maxi)
        np.testing.assert_allclose(oracle.value_iteration(dm, sp)[1], oracle.value_iteration(_om(m), sp)[1],
                                   atol=1e-15)


# --------------------------------------------------------------------------- validation

def test_validation_rejects_bad_models():
    base = dict(n_states=2, stateptr=np.array([0, 1, 2]), colptr=np.array([0, 2, 3]), rowval=np.array([0, 1, 1]),
                lower=np.array([0.2, 0.3, 1.0]), upper=np.array([0.6, 0.7, 1.0]))
    assert oracle.validate(oracle.OracleIMDP(**base)) == "ok"
    def v(**kw):
        d = dict(base); d.update(kw)
        return oracle.validate(oracle.OracleIMDP(**d))
    assert v(lower=np.array([0.6, 0.5, 1.0])) == "einfeasible"        # sum lower > 1
    assert v(upper=np.array([0.3, 0.4, 1.0])) == "einfeasible"        # sum upper < 1
    assert v(lower=np.array([0.7, 0.3, 1.0])) == "einfeasible"        # lower > upper
    assert v(lower=np.array([-0.1, 0.3, 1.0])) == "einfeasible"       # negative
    assert v(rowval=np.array([1, 0, 1])) == "einval"                   # unsorted destinations
    assert v(rowval=np.array([0, 2, 1])) == "einval"                   # out of range
    assert v(stateptr=np.array([0, 2, 2])) == "einval"                 # state without an action
    assert v(colptr=np.array([0, 3, 2])) == "einval"                   # decreasing colptr


def test_invalid_spec():
    m = _gamblers_ruin(4, 0.5)
    assert oracle.value_iteration(m, oracle.OracleSpec(reach=[7]))[0] == "einval"
    assert oracle.value_iteration(m, oracle.OracleSpec(property=oracle.REACH_AVOID, reach=[4], avoid=[4]))[0] == "einval"
    assert oracle.value_iteration(m, oracle.OracleSpec(infinite_time=True, eps=0.0, reach=[4]))[0] == "einval"
    assert oracle.value_iteration(m, oracle.OracleSpec(property=oracle.REWARD, reward=np.ones(5), discount=1.5))[0] == "einval"
    # non-convergence within the iteration cap is reported
    assert oracle.value_iteration(m, oracle.OracleSpec(infinite_time=True, eps=1e-300, horizon=5, reach=[4]))[0] == "enoconv"


# --------------------------------------------------------------------------- threaded sweep

@pytest.mark.parametrize("kind", ["finite", "infinite", "reward", "reach_avoid"])
def test_threaded_sweep_gives_the_same_words(kind):
    # The OpenMP sweep splits the states of one Bellman iteration over threads
    # (Sec. 4: the per-state problems are independent within an iteration) and
    # combines only the residual, by a max. Every state is computed by the same
    # sequential code whatever thread runs it, so 1, 2 and 8 threads must give
    # the same binary64 words, the same k and the same policy.
    if not oracle.has_openmp():
        pytest.skip("oracle built without OpenMP")
    m = banded_imdp(700, 3, 700 * 3 * 25 + 1, eps=0.1, seed=77)
    kw = dict(reach=m.goal)
    if kind == "finite":
        sp = oracle.OracleSpec(horizon=40, pessimistic=True, maximize=True, **kw)
    elif kind == "infinite":
        sp = oracle.OracleSpec(infinite_time=True, eps=1e-9, horizon=100000, pessimistic=False, maximize=True, **kw)
    elif kind == "reward":
        r = np.random.default_rng(3).random(m.n_states)
        sp = oracle.OracleSpec(property=oracle.REWARD, horizon=30, reward=r, discount=0.9, pessimistic=True,
                               maximize=False)
    else:
        avoid = np.setdiff1d(np.arange(0, m.n_states, 37), m.goal)
        sp = oracle.OracleSpec(property=oracle.REACH_AVOID, horizon=30, avoid=avoid, pessimistic=True,
                               maximize=True, **kw)
    ref = oracle.value_iteration(_om(m), sp, policy=True, threads=1)
    assert ref[0] == "ok"
    for t in (2, 8):
        got = oracle.value_iteration(_om(m), sp, policy=True, threads=t)
        assert got[0] == ref[0] and got[2] == ref[2]
        assert np.array_equal(got[1].view(np.uint64), ref[1].view(np.uint64))
        assert np.array_equal(got[3].view(np.uint64), ref[3].view(np.uint64))
        assert np.array_equal(got[4], ref[4])
