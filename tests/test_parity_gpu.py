"""CUDA path vs the CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2401_04068_gb300 as g
from gpu_helpers import TOL_F64, check_policy_row, om, q_values, run_oracle
from workloads import banded_batch, banded_imdp, concat_block_diagonal, make_config, random_imdp

pytestmark = pytest.mark.gpu

MODES = [(True, True), (True, False), (False, True), (False, False)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    g.load()


def _model(m):
    return g.create_model(m)


def _compare(m, model, tol=TOL_F64, policy=False, **kw):
    st, V, k, res, pol = g.value_iteration(model, m.n_states, policy=policy, **kw)
    ost, oV, ok, ores, opol = run_oracle(m, policy=policy, **kw)
    assert st == ost, (st, ost)
    assert k == ok
    np.testing.assert_allclose(V, oV, rtol=0, atol=tol)
    np.testing.assert_allclose(res, ores, rtol=0, atol=tol)
    return V, k, res, pol, oV


# --------------------------------------------------------------------------- the paper's worked example

@pytest.mark.parametrize("pess,maxi", MODES)
def test_worked_example(worked_example, pess, maxi):
    ex = worked_example
    class M: pass
    m = M()
    for key in ("n_states", "stateptr", "colptr", "rowval", "lower", "upper"):
        setattr(m, key, ex[key])
    m.n_cols = len(ex["colptr"]) - 1
    model = _model(m)
    for K in (0, 1, 2, 7, ex["horizon"]):
        _compare(m, model, horizon=K, reach=ex["goal"], pessimistic=pess, maximize=maxi)
    st, V, k, res, pol = g.value_iteration(model, 3, policy=True, horizon=1, reach=ex["goal"])
    np.testing.assert_allclose(V, [0.2, 0.4, 1.0], atol=1e-15)
    assert list(pol[0]) == [0, 1, -1]


# --------------------------------------------------------------------------- small random models, all modes

@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("pess,maxi", MODES)
def test_random_models(seed, pess, maxi):
    m = random_imdp(40, max_actions=3, density=0.3 + 0.05 * seed, seed=seed)
    model = _model(m)
    V, k, res, pol, _ = _compare(m, model, policy=True, horizon=12, reach=m.goal, pessimistic=pess, maximize=maxi)
    # policy at time 0 is the argmax of the last iteration: check it by Q-values
    Vprev = V - res
    check_policy_row(m, Vprev, pol[0], set(m.goal.tolist()), pess, maxi)


@pytest.mark.parametrize("seed", range(3))
def test_ties_and_exact_grids(seed):
    # bounds on a dyadic grid and many equal values: threshold ties everywhere
    m = random_imdp(30, max_actions=2, density=0.5, seed=50 + seed, exact_grid=16)
    model = _model(m)
    for pess, maxi in MODES:
        _compare(m, model, horizon=9, reach=m.goal, pessimistic=pess, maximize=maxi)


def test_lower_equals_upper_and_rem_zero():
    m = random_imdp(50, max_actions=2, density=0.2, seed=3, lower_equals_upper=True)
    model = _model(m)
    for pess, maxi in MODES:
        _compare(m, model, horizon=20, reach=m.goal, pessimistic=pess, maximize=maxi)


# --------------------------------------------------------------------------- column-size classes and ragged tails

@pytest.mark.parametrize("k_mean", [3, 20, 45, 100, 200, 400, 700, 1100, 2600])
def test_banded_column_classes(k_mean):
    # short columns (many per tile), long ones (a few per tile), and columns of
    # 1024 entries or more (their states run block-wide), with ragged lengths
    n_dom = max(3 * k_mean, 60) if k_mean < 1000 else k_mean + 200  # oracle-sized
    m = banded_imdp(n_dom, 2, n_dom * 2 * (k_mean + 1) + 1, eps=0.08, seed=k_mean)
    model = _model(m)
    for pess, maxi in [(True, True), (False, False)]:
        _compare(m, model, horizon=15, reach=m.goal, pessimistic=pess, maximize=maxi)


def test_wide_and_tiled_states_mixed():
    # one model whose states alternate between short columns (tiles) and columns
    # of >= 1024 entries or several long actions (wide states), batched with a
    # small model; results against the oracle, batch against alone to the bit
    rng = np.random.default_rng(77)
    n = 1400
    sp, cp, rv, lo, up = [0], [0], [], [], []
    for s in range(n):
        acts = 1 + (s % 3)
        for a in range(acts):
            k = int(rng.integers(1290, 1390)) if (s % 7 == 0 and a == 0) else int(rng.integers(3, 60))
            dest = np.sort(rng.choice(n, size=k, replace=False))
            p = rng.random(k) + 0.01
            p /= p.sum()
            l = p * (1 - 0.1 * rng.random(k))
            u = np.minimum(1.0, p * (1 + 0.1 * rng.random(k)))
            rv.extend(dest.tolist()), lo.extend(l.tolist()), up.extend(u.tolist())
            cp.append(len(rv))
        sp.append(len(cp) - 1)
    from workloads import IMDPInput
    goal = np.arange(100, 160, dtype=np.int32)
    m = IMDPInput(n, np.array(sp, np.int32), np.array(cp, np.int32), np.array(rv, np.int32), np.array(lo),
                  np.array(up), goal)
    model = _model(m)
    n_tiles, n_wide, wide_entries = g.imdp_model_plan(model)
    assert n_wide == 200 and n_tiles > 0
    k = np.diff(m.colptr)
    assert wide_entries == sum(int(k[m.stateptr[s]:m.stateptr[s + 1]].sum()) for s in range(0, n, 7))
    for pess, maxi in MODES:
        _compare(m, model, horizon=12, reach=m.goal, pessimistic=pess, maximize=maxi)
    small = random_imdp(30, max_actions=3, seed=78)
    sm = _model(small)
    specs = [g.make_spec(horizon=20, reach=m.goal), g.make_spec(horizon=20, reach=small.goal, pessimistic=False)]
    outs = [np.zeros(m.n_states), np.zeros(small.n_states)]
    ks = np.zeros(2, np.int32)
    g.imdp_value_iteration_batch([model, sm], specs, outs, ks)
    for mdl, spec, out, n_s in [(model, specs[0], outs[0], m.n_states), (sm, specs[1], outs[1], small.n_states)]:
        alone = np.zeros(n_s)
        g.imdp_value_iteration(mdl, spec, alone)
        np.testing.assert_array_equal(out, alone)


def _wide_model(seed, n=700, actions=2):
    # every state has one column of >= 1280 entries (a wide state) next to short ones
    rng = np.random.default_rng(seed)
    sp, cp, rv, lo, up = [0], [0], [], [], []
    for s in range(n):
        for a in range(actions):
            k = int(rng.integers(1290, 1400)) if a == 0 else int(rng.integers(5, 40))
            k = min(k, n)
            dest = np.sort(rng.choice(n, size=k, replace=False))
            p = rng.random(k) + 0.01
            p /= p.sum()
            rv.extend(dest.tolist()), lo.extend((p * (1 - 0.1 * rng.random(k))).tolist())
            up.extend(np.minimum(1.0, p * (1 + 0.1 * rng.random(k))).tolist())
            cp.append(len(rv))
        sp.append(len(cp) - 1)
    from workloads import IMDPInput
    return IMDPInput(n, np.array(sp, np.int32), np.array(cp, np.int32), np.array(rv, np.int32), np.array(lo),
                     np.array(up), np.arange(300, 340, dtype=np.int32))


def test_wide_states_rewards_infinite_horizon_and_policy():
    m = _wide_model(79, n=1400)
    model = _model(m)
    n_tiles, n_wide, _ = g.imdp_model_plan(model)
    assert n_wide == m.n_states and n_tiles == 0
    r = np.linspace(-0.5, 1.5, m.n_states)
    for pess, maxi in [(True, True), (False, False)]:
        _compare(m, model, property=oracle.REWARD, horizon=20, reward=r, discount=0.9, pessimistic=pess,
                 maximize=maxi)
    _compare(m, model, property=oracle.REWARD, infinite_time=True, eps=1e-9, horizon=100000, reward=r,
             discount=0.8)
    _compare(m, model, infinite_time=True, eps=1e-9, horizon=100000, reach=m.goal, pessimistic=False)
    avoid = np.arange(0, 30, dtype=np.int32)
    _compare(m, model, property=oracle.REACH_AVOID, horizon=15, reach=m.goal, avoid=avoid)
    # time-dependent policy rows from the block-wide argmax
    K = 4
    st, V, k, res, pol = g.value_iteration(model, m.n_states, policy=True, horizon=K, reach=m.goal)
    for t in range(K):
        _, Vp, _, _, _ = run_oracle(m, horizon=K - t - 1, reach=m.goal)
        check_policy_row(m, Vp, pol[t], set(m.goal.tolist()), True, True)


def test_reach_avoid():
    m = banded_imdp(400, 3, 400 * 3 * 13 + 1, eps=0.1, seed=8)
    model = _model(m)
    avoid = np.concatenate([m.sink, np.arange(0, 20)])
    for pess, maxi in MODES:
        _compare(m, model, property=oracle.REACH_AVOID, horizon=30, reach=m.goal, avoid=avoid,
                 pessimistic=pess, maximize=maxi)


@pytest.mark.parametrize("pess", [True, False])
def test_infinite_horizon(pess):
    m = banded_imdp(300, 2, 300 * 2 * 16 + 1, eps=0.05, seed=9)
    model = _model(m)
    V, k, res, pol, oV = _compare(m, model, policy=True, infinite_time=True, eps=1e-7, horizon=100000,
                                  reach=m.goal, pessimistic=pess)
    assert np.max(np.abs(res)) < 1e-7
    check_policy_row(m, V - res, pol[0], set(m.goal.tolist()), pess, True)


def test_infinite_horizon_cap_reports_noconv():
    m = banded_imdp(200, 1, 200 * 10 + 1, seed=10)
    model = _model(m)
    st, V, k, res, _ = g.value_iteration(model, m.n_states, infinite_time=True, eps=1e-300, horizon=7, reach=m.goal)
    assert st == "enoconv" and k == 7
    ost, oV, ok, _, _ = run_oracle(m, infinite_time=True, eps=1e-300, horizon=7, reach=m.goal)
    np.testing.assert_allclose(V, oV, atol=TOL_F64)


def test_time_dependent_policy_all_rows():
    m = random_imdp(25, max_actions=3, density=0.4, seed=77)
    model = _model(m)
    K = 6
    st, V, k, res, pol = g.value_iteration(model, m.n_states, policy=True, horizon=K, reach=m.goal)
    for t in range(K):
        # row t is the decision of iteration K - t, made from V_{K-t-1}
        _, Vp, _, _, _ = run_oracle(m, horizon=K - t - 1, reach=m.goal)
        check_policy_row(m, Vp, pol[t], set(m.goal.tolist()), True, True)


# --------------------------------------------------------------------------- batch vs alone, device buffers

def test_batch_equals_alone_bitwise():
    import torch
    ms = [banded_imdp(120, 2, 120 * 2 * 9 + 1, seed=s) for s in range(3)] + [random_imdp(30, seed=4)]
    models = [_model(m) for m in ms]
    specs = [g.make_spec(horizon=10 + 5 * i, reach=m.goal, pessimistic=(i % 2 == 0), maximize=(i < 2))
             for i, m in enumerate(ms)]
    outs = [np.zeros(m.n_states) for m in ms]
    ks = [0] * len(ms)
    g.imdp_value_iteration_batch(models, specs, outs, ks)
    for i, m in enumerate(ms):
        alone = np.zeros(m.n_states)
        kk = [0]
        g.imdp_value_iteration(models[i], specs[i], alone, kk)
        assert kk[0] == ks[i] == 10 + 5 * i
        np.testing.assert_array_equal(outs[i], alone)
        _, oV, _, _, _ = run_oracle(m, horizon=10 + 5 * i, reach=m.goal, pessimistic=(i % 2 == 0), maximize=(i < 2))
        np.testing.assert_allclose(alone, oV, atol=TOL_F64)
    # device output buffers give the same numbers
    dev = torch.zeros(ms[0].n_states, dtype=torch.float64, device="cuda")
    g.imdp_value_iteration(models[0], specs[0], dev)
    np.testing.assert_array_equal(dev.cpu().numpy(), outs[0])


def test_cta_shapes_agree_to_the_bit():
    # tiles of many short columns run in 24-warp CTAs, others (and every launch
    # with wide states) in 16-warp CTAs; a column's words do not depend on which
    m = banded_imdp(3000, 1, 3000 * 24 + 1, seed=91)
    model = _model(m)
    n_tiles, n_wide, _ = g.imdp_model_plan(model)
    assert n_wide == 0 and len(m.colptr) - 1 >= 16 * n_tiles  # the 24-warp shape alone
    spec = g.make_spec(horizon=25, reach=m.goal)
    alone = np.zeros(m.n_states)
    g.imdp_value_iteration(model, spec, alone)
    _, oV, _, _, _ = run_oracle(m, horizon=25, reach=m.goal)
    np.testing.assert_allclose(alone, oV, rtol=0, atol=TOL_F64)
    w = _wide_model(92, n=1300, actions=1)
    wm = _model(w)
    assert g.imdp_model_plan(wm)[1] > 0  # a batch with wide states: the 16-warp shape
    outs = [np.zeros(m.n_states), np.zeros(w.n_states)]
    g.imdp_value_iteration_batch([model, wm], [spec, g.make_spec(horizon=25, reach=w.goal)], outs, [0, 0])
    np.testing.assert_array_equal(outs[0], alone)
    wa = np.zeros(w.n_states)
    g.imdp_value_iteration(wm, g.make_spec(horizon=25, reach=w.goal), wa)
    np.testing.assert_array_equal(outs[1], wa)


def test_models_read_from_files(tmp_path):
    # the Sec. 3.1 model as PRISM explicit files (with its Sec. 3.2 query) and a
    # bmdp-tool round trip of a random model, run through the CUDA path
    import os
    f = g.imdp_read_prism(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_example"))
    model = _model(f)
    st, V, k, res, _ = g.value_iteration(model, f.n_states, **f.spec)
    _, oV, ok, _, _ = run_oracle(f, **f.spec)
    assert st == "ok" and k == ok == 100
    np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64)
    m = random_imdp(300, max_actions=3, seed=93)
    g.imdp_write_bmdp_tool(tmp_path / "m.bmdp", m, m.goal)
    fb = g.imdp_read_bmdp_tool(tmp_path / "m.bmdp")
    spec = dict(fb.spec, horizon=30)
    _compare(fb, _model(fb), **spec)


def test_checkpoint_and_resume():
    # stop a run after k1 iterations, restore (V_k1, k1) into a fresh session and
    # finish there: the same V as the uninterrupted run (hints start empty after
    # a restore, so within rounding rather than bitwise) and the oracle's V
    import torch
    m = banded_imdp(400, 2, 400 * 2 * 30 + 1, seed=94)
    model = _model(m)
    for spec_kw, k1 in [(dict(horizon=40, reach=m.goal), 15),
                        (dict(horizon=35, reach=m.goal, pessimistic=False, maximize=False), 35),
                        (dict(infinite_time=True, eps=1e-9, horizon=100000, reach=m.goal), 20)]:
        spec = g.make_spec(**spec_kw)
        full = g.imdp_session_create([model], [spec])
        g.imdp_session_run(full)
        V_full, k_full = np.zeros(m.n_states), [0]
        g.imdp_session_read(full, 0, V_full, k_full)

        first = g.imdp_session_create([model], [spec])
        g.imdp_session_step(first, k1)
        raw, k = g.imdp_session_checkpoint(first, 0)
        assert k == k1
        dev = torch.zeros(m.n_states, dtype=torch.int64, device="cuda")
        _, kd = g.imdp_session_checkpoint(first, 0, dev)  # device buffer: the same words
        assert kd == k1 and np.array_equal(dev.cpu().numpy().view(np.uint64), raw)

        second = g.imdp_session_create([model], [spec])
        g.imdp_session_restore(second, 0, raw, k)
        g.imdp_session_run(second)
        V, kk = np.zeros(m.n_states), [0]
        g.imdp_session_read(second, 0, V, kk)
        if spec_kw.get("infinite_time"):
            assert abs(kk[0] - k_full[0]) <= 1
        else:
            assert kk[0] == k_full[0] == spec_kw["horizon"]
        np.testing.assert_allclose(V, V_full, rtol=0, atol=1e-13)
        _, oV, _, _, _ = run_oracle(m, **spec_kw)
        np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64 if not spec_kw.get("infinite_time") else 1e-8)
    # bad arguments
    s = g.imdp_session_create([model], [g.make_spec(horizon=10, reach=m.goal)])
    raw = np.zeros(m.n_states, np.uint64)
    for idx, kk in [(1, 0), (0, 11), (0, -1)]:
        with pytest.raises(g.ImdpError):
            g.imdp_session_restore(s, idx, raw, kk)


def test_restore_into_a_session_that_already_ran():
    # A restore may target a session that has stepped or run before: the next
    # run must still carry the restored problem from k to its horizon (Eq. 2
    # iterations k + 1 .. K), not stop at the session's earlier launch count.
    m = banded_imdp(300, 2, 300 * 2 * 20 + 1, seed=96)
    model = _model(m)
    spec = g.make_spec(horizon=30, reach=m.goal)
    s = g.imdp_session_create([model], [spec])
    g.imdp_session_step(s, 10)
    raw, k = g.imdp_session_checkpoint(s, 0)
    assert k == 10
    g.imdp_session_run(s)  # to the horizon
    g.imdp_session_restore(s, 0, raw, k)
    g.imdp_session_run(s)
    V, kk = np.zeros(m.n_states), [0]
    assert g.imdp_session_read(s, 0, V, kk) == g.IMDP_OK and kk[0] == 30
    _, oV, _, _, _ = run_oracle(m, horizon=30, reach=m.goal)
    np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64)
    s.close()


def test_device_inputs():
    import torch
    m = banded_imdp(200, 2, 200 * 2 * 12 + 1, seed=12)
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(m, k))).cuda()
         for k in ("stateptr", "colptr", "rowval", "lower", "upper")}
    model = g.imdp_create_csc(m.n_states, m.n_cols, m.nnz, t["stateptr"], t["colptr"], t["rowval"], t["lower"],
                              t["upper"])
    host_model = _model(m)
    a = g.value_iteration(model, m.n_states, horizon=10, reach=m.goal)[1]
    b = g.value_iteration(host_model, m.n_states, horizon=10, reach=m.goal)[1]
    np.testing.assert_array_equal(a, b)


def test_dense_create_matches_csc(worked_example):
    ex = worked_example
    n = ex["n_states"]
    m_cols = len(ex["colptr"]) - 1
    lo = np.zeros((m_cols, n)); up = np.zeros((m_cols, n))
    for j in range(m_cols):
        for i in range(ex["colptr"][j], ex["colptr"][j + 1]):
            lo[j, ex["rowval"][i]] = ex["lower"][i]; up[j, ex["rowval"][i]] = ex["upper"][i]
    acts = np.diff(ex["stateptr"]).astype(np.int32)
    dm = g.imdp_create_dense(n, acts, np.ascontiguousarray(lo.reshape(-1)), np.ascontiguousarray(up.reshape(-1)))
    class M: pass
    m = M()
    for key in ("n_states", "stateptr", "colptr", "rowval", "lower", "upper"):
        setattr(m, key, ex[key])
    cm = _model(m)
    for K in (1, 5, 30):
        a = g.value_iteration(dm, n, horizon=K, reach=ex["goal"])[1]
        b = g.value_iteration(cm, n, horizon=K, reach=ex["goal"])[1]
        np.testing.assert_array_equal(a, b)


def test_dense_large_model_runs_wide():
    # a dense model (every column lists all 1500 states, the layout of Sec. 3.1's
    # dense matrices): every state is wide; against the oracle on the CSC form
    rng = np.random.default_rng(91)
    n, acts = 1500, 2
    P = rng.random((n * acts, n)) ** 6 + 1e-6
    P /= P.sum(axis=1, keepdims=True)
    lo = P * (1 - 0.2 * rng.random(P.shape))
    up = np.minimum(1.0, P * (1 + 0.2 * rng.random(P.shape)))
    dm = g.imdp_create_dense(n, np.full(n, acts, np.int32), np.ascontiguousarray(lo.reshape(-1)),
                             np.ascontiguousarray(up.reshape(-1)))
    assert g.imdp_model_plan(dm)[1] == n
    from workloads import IMDPInput
    m = IMDPInput(n, (np.arange(n + 1) * acts).astype(np.int32), (np.arange(n * acts + 1) * n).astype(np.int32),
                  np.tile(np.arange(n, dtype=np.int32), n * acts), lo.reshape(-1), up.reshape(-1),
                  np.arange(700, 760, dtype=np.int32))
    for pess, maxi in [(True, True), (False, True)]:
        _compare(m, dm, horizon=12, reach=m.goal, pessimistic=pess, maximize=maxi)


# --------------------------------------------------------------------------- errors

def test_rejects_infeasible_and_malformed():
    m = random_imdp(6, seed=1)
    bad = m.lower.copy(); bad[0] = m.upper[0] + 0.1
    with pytest.raises(g.ImdpError) as e:
        g.imdp_create_csc(m.n_states, m.n_cols, m.nnz, m.stateptr, m.colptr, m.rowval, bad, m.upper)
    assert e.value.status == g.IMDP_EINFEASIBLE
    rows = m.rowval.copy(); rows[0] = 99
    with pytest.raises(g.ImdpError) as e:
        g.imdp_create_csc(m.n_states, m.n_cols, m.nnz, m.stateptr, m.colptr, rows, m.lower, m.upper)
    assert e.value.status == g.IMDP_EINVAL
    model = _model(m)
    with pytest.raises(g.ImdpError):
        g.value_iteration(model, m.n_states, horizon=3, reach=[100])
    with pytest.raises(g.ImdpError):
        g.value_iteration(model, m.n_states, property=g.IMDP_REACH_AVOID, horizon=3, reach=[1], avoid=[1])


# --------------------------------------------------------------------------- full-size shapes, sampled outputs

@pytest.mark.parametrize("name", ["cartpole3840", "pimdp2"])
def test_full_size_sampled_one_step(name):
    """At the benchmark's full sizes: the last Bellman step of a K = 200 run,
    recomputed by the oracle state by state from the GPU's V_{K-1}."""
    m = make_config(name)
    model = _model(m)
    K = 200
    st, V, k, res, pol = g.value_iteration(model, m.n_states, policy=True, horizon=K, reach=m.goal)
    assert st == "ok" and k == K
    assert np.all(V >= 0) and np.all(V <= 1) and np.all(res >= 0)
    Vprev = V - res
    rng = np.random.default_rng(0)
    goal = set(m.goal.tolist())
    for s in rng.choice(m.n_states, 64, replace=False):
        if s in goal:
            assert V[s] == 1.0 and pol[0][s] == -1
            continue
        qs = []
        for j in range(m.stateptr[s], m.stateptr[s + 1]):
            a, b = m.colptr[j], m.colptr[j + 1]
            qs.append(oracle.omax_column(Vprev[m.rowval[a:b]], m.lower[a:b], m.upper[a:b], True)[0])
        assert abs(V[s] - max(qs)) <= 1e-12, (s, V[s], qs)
        assert abs(qs[pol[0][s]] - max(qs)) <= 1e-12


# --------------------------------------------------------------------------- discounted reward (Sec. 3.2)

def _reward_tol(oV):
    return TOL_F64 * max(1.0, float(np.max(np.abs(oV))))


@pytest.mark.parametrize("pess,maxi", MODES)
@pytest.mark.parametrize("gamma,K", [(0.9, 30), (0.95, 100), (1.0, 12)])
def test_finite_reward(pess, maxi, gamma, K):
    m = banded_imdp(300, 2, 300 * 2 * 14 + 1, eps=0.1, seed=40)
    r = np.random.default_rng(1).uniform(-1.0, 3.0, m.n_states)
    model = _model(m)
    st, V, k, res, pol = g.value_iteration(model, m.n_states, policy=True, property=g.IMDP_REWARD, horizon=K,
                                           reward=r, discount=gamma, pessimistic=pess, maximize=maxi)
    ost, oV, ok, ores, _ = run_oracle(m, property=oracle.REWARD, horizon=K, reward=r, discount=gamma,
                                      pessimistic=pess, maximize=maxi)
    assert st == ost == "ok" and k == ok == K
    tol = _reward_tol(oV)
    np.testing.assert_allclose(V, oV, rtol=0, atol=tol)
    np.testing.assert_allclose(res, ores, rtol=0, atol=tol)
    # policy: the chosen action attains the optimum of r + gamma * q
    q = q_values(m, V - res, pess)
    for s in range(0, m.n_states, 7):
        js = range(m.stateptr[s], m.stateptr[s + 1])
        qs = np.array([q[j] for j in js])
        best = qs.max() if maxi else qs.min()
        assert abs(qs[pol[0][s]] - best) * gamma <= tol


def test_infinite_reward_and_closed_form():
    m = banded_imdp(200, 2, 200 * 2 * 10 + 1, eps=0.05, seed=41)
    r = np.random.default_rng(2).uniform(0.0, 2.0, m.n_states)
    model = _model(m)
    st, V, k, res, _ = g.value_iteration(model, m.n_states, property=g.IMDP_REWARD, infinite_time=True, eps=1e-9,
                                         horizon=100000, reward=r, discount=0.9)
    ost, oV, ok, _, _ = run_oracle(m, property=oracle.REWARD, infinite_time=True, eps=1e-9, horizon=100000,
                                   reward=r, discount=0.9)
    assert st == ost == "ok"
    assert abs(k - ok) <= 1  # the stopping iteration may differ by one at the eps boundary
    np.testing.assert_allclose(V, oV, rtol=0, atol=1e-7)
    # the sink is absorbing with reward r_sink: V = r / (1 - gamma)
    s = int(m.sink[0])
    assert V[s] == pytest.approx(r[s] / 0.1, rel=1e-7)


def test_reward_batch_mixed_with_reachability():
    m = banded_imdp(150, 2, 150 * 2 * 8 + 1, seed=42)
    r = np.linspace(-2.0, 2.0, m.n_states)
    model = _model(m)
    specs = [g.make_spec(property=g.IMDP_REWARD, horizon=20, reward=r, discount=0.8),
             g.make_spec(horizon=25, reach=m.goal)]
    outs = [np.zeros(m.n_states), np.zeros(m.n_states)]
    ks = [0, 0]
    g.imdp_value_iteration_batch([model, model], specs, outs, ks)
    assert ks == [20, 25]
    _, oV, _, _, _ = run_oracle(m, property=oracle.REWARD, horizon=20, reward=r, discount=0.8)
    np.testing.assert_allclose(outs[0], oV, rtol=0, atol=_reward_tol(oV))
    _, oV2, _, _, _ = run_oracle(m, horizon=25, reach=m.goal)
    np.testing.assert_allclose(outs[1], oV2, rtol=0, atol=TOL_F64)


# --------------------------------------------------------------------------- wide intervals, resets

@pytest.mark.parametrize("k_mean,n_dom", [(40, 200), (300, 900), (3500, 3600)])
def test_wide_intervals_sum_of_upper_far_above_one(k_mean, n_dom):
    # upper = 1 on every entry: a column's upper bounds add up to k (gap sums
    # far beyond 2 in fixed point); the last case has columns longer than a
    # shared-memory tile, which run as wide states in the block-wide kernel
    m = banded_imdp(n_dom, 1, n_dom * (k_mean + 1) + 1, eps=0.1, seed=k_mean)
    m.upper = np.ones_like(m.upper)
    m.lower = m.lower * 0.5
    model = _model(m)
    for pess, maxi in MODES:
        _compare(m, model, horizon=6, reach=m.goal, pessimistic=pess, maximize=maxi)


def test_session_reset_restarts_from_v0():
    m = banded_imdp(300, 2, 300 * 2 * 20 + 1, seed=13)
    model = _model(m)
    spec = g.make_spec(horizon=40, reach=m.goal)
    sess = g.imdp_session_create([model], [spec])
    V1 = np.zeros(m.n_states)
    V2 = np.zeros(m.n_states)
    g.imdp_session_run(sess)
    g.imdp_session_read(sess, 0, V1)
    g.imdp_session_reset(sess)
    g.imdp_session_step(sess, 17)
    g.imdp_session_reset(sess)
    g.imdp_session_run(sess)
    k = [0]
    g.imdp_session_read(sess, 0, V2, k)
    assert k[0] == 40
    np.testing.assert_array_equal(V1, V2)
    _, oV, _, _, _ = run_oracle(m, horizon=40, reach=m.goal)
    np.testing.assert_allclose(V2, oV, atol=TOL_F64)


# --------------------------------------------------------------------------- 32-bit storage

@pytest.mark.parametrize("pess,maxi", MODES)
def test_f32_storage_within_a_priori_bound(pess, maxi):
    m = banded_imdp(400, 3, 400 * 3 * 40 + 1, eps=0.1, seed=70)
    model = g.create_model(m, dtype=g.IMDP_F32)
    d = model.error_bound()
    assert 0.0 < d < 1e-8
    K = 60
    st, V, k, res, _ = g.value_iteration(model, m.n_states, horizon=K, reach=m.goal, pessimistic=pess, maximize=maxi)
    _, oV, _, _, _ = run_oracle(m, horizon=K, reach=m.goal, pessimistic=pess, maximize=maxi)
    err = float(np.max(np.abs(V - oV)))
    assert err <= K * d + 1e-10, (err, K * d)


@pytest.mark.parametrize("name", ["pendulum240_x4096", "pimdp2"])
def test_f32_storage_benchmark_shapes_1e6(name):
    # the benchmark query (K = 200) on the 32-bit path stays within 1e-6 of the
    # binary64 oracle (checked on the oracle-sized part of each workload)
    if name == "pendulum240_x4096":
        m = make_config(name, n_models=16)
    else:
        m = make_config(name)
    model = g.create_model(m, dtype=g.IMDP_F32)
    K = 200
    st, V, k, res, _ = g.value_iteration(model, m.n_states, horizon=K, reach=m.goal)
    assert k == K and model.error_bound() * K < 1e-5
    if name == "pimdp2":
        # full-size: the last step recomputed by the oracle from the GPU's V_{K-1}
        # on the stored (rounded) bounds is within rounding; against binary64 bounds
        # the per-iteration bound applies
        Vprev = V - res
        rng = np.random.default_rng(1)
        for s in rng.choice(m.n_states, 48, replace=False):
            if s in set(m.goal.tolist()):
                continue
            qs = []
            for j in range(m.stateptr[s], m.stateptr[s + 1]):
                a, b = m.colptr[j], m.colptr[j + 1]
                qs.append(oracle.omax_column(Vprev[m.rowval[a:b]], m.lower[a:b], m.upper[a:b], True)[0])
            assert abs(V[s] - max(qs)) <= model.error_bound() + 1e-12
    else:
        _, oV, _, _, _ = run_oracle(m, horizon=K, reach=m.goal)
        assert float(np.max(np.abs(V - oV))) <= 1e-6


def test_f32_batch_with_f64_models():
    ms = [banded_imdp(200, 2, 200 * 2 * 15 + 1, seed=71), banded_imdp(100, 1, 100 * 30 + 1, seed=72)]
    models = [g.create_model(ms[0], dtype=g.IMDP_F32), g.create_model(ms[1])]
    specs = [g.make_spec(horizon=30, reach=ms[0].goal), g.make_spec(horizon=20, reach=ms[1].goal)]
    outs = [np.zeros(ms[0].n_states), np.zeros(ms[1].n_states)]
    g.imdp_value_iteration_batch(models, specs, outs)
    _, o0, _, _, _ = run_oracle(ms[0], horizon=30, reach=ms[0].goal)
    _, o1, _, _, _ = run_oracle(ms[1], horizon=20, reach=ms[1].goal)
    assert np.max(np.abs(outs[0] - o0)) <= 30 * models[0].error_bound() + 1e-10
    np.testing.assert_allclose(outs[1], o1, atol=TOL_F64)
