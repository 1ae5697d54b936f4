"""Launch configurations of the Bellman step and the autotuner, through the C ABI.

Every configuration (ring, direct or slice kernel, warps per CTA, CTAs per SM,
tile size, wide-state threshold) must compute the same words: each column's
value is the same multiset of exact integer terms whichever kernel runs it,
and every kernel takes the same path (warm start, neighbour check or search)
for a column given the same hint. Checked bitwise between configurations and
against the oracle within TOL_F64."""
import json
import os

import numpy as np
import pytest

import paper_2401_04068_gb300 as g
from gpu_helpers import TOL_F64, run_oracle
from workloads import banded_batch, banded_imdp, random_imdp

pytestmark = pytest.mark.gpu

CONFIGS = [
    dict(kernel=g.KERNEL_RING, cta_warps=16),
    dict(kernel=g.KERNEL_RING, cta_warps=24),
    dict(kernel=g.KERNEL_DIRECT, ctas_per_sm=4),
    dict(kernel=g.KERNEL_DIRECT, ctas_per_sm=3),
    dict(kernel=g.KERNEL_DIRECT, ctas_per_sm=4, tile_entries=300),
    dict(kernel=g.KERNEL_RING, cta_warps=16, tile_entries=700, wide_col=200),
    dict(kernel=g.KERNEL_DIRECT, ctas_per_sm=4, wide_col=1 << 30),
    dict(kernel=g.KERNEL_DIRECT, ctas_per_sm=3, wide_col=150),
    dict(kernel=g.KERNEL_SLICE, ctas_per_sm=4),
    dict(kernel=g.KERNEL_SLICE, ctas_per_sm=3),
]


def _run(model, m, spec, cfg, steps):
    sess = g.imdp_session_create([model], [spec])
    g.imdp_session_set_launch(sess, **cfg)
    g.imdp_session_step(sess, steps)
    raw, k = g.imdp_session_checkpoint(sess, 0)
    V = np.zeros(m.n_states)
    g.imdp_session_read(sess, 0, V, check=False)
    resolved = g.imdp_session_get_launch(sess)
    sess.close()
    return raw, k, V, resolved


@pytest.mark.parametrize("case", ["reach", "reach_avoid_opt", "reward", "infinite", "f32", "f32_pure", "mixed_wide"])
def test_every_launch_config_gives_the_same_words(case):
    if case == "mixed_wide":
        # short, medium and long columns in one model: tiles and wide states
        m = banded_imdp(900, 2, 900 * 2 * 180 + 900 * 2 + 1, eps=0.1, seed=61)
    else:
        m = banded_imdp(700, 3, 700 * 3 * 40 + 700 * 3 + 1, eps=0.1, seed=60)
    if case == "f32":  # a budget small enough to keep some columns exact
        model = g.create_model(m, dtype=g.IMDP_F32, budget=1.5e-9)
    elif case == "f32_pure":  # no correction column: the ring kernel runs it too
        model = g.create_model(m, dtype=g.IMDP_F32, budget=1.0)
    else:
        model = g.create_model(m)
    K = 40
    okw = dict(horizon=K, reach=m.goal)
    if case == "reach_avoid_opt":
        avoid = np.setdiff1d(np.arange(0, m.n_states, 29), m.goal)
        okw.update(property=g.IMDP_REACH_AVOID, avoid=avoid, pessimistic=False, maximize=False)
    elif case == "reward":
        r = np.random.default_rng(2).uniform(-1, 2, m.n_states)
        okw = dict(property=g.IMDP_REWARD, horizon=K, reward=r, discount=0.9)
    elif case == "infinite":
        okw = dict(infinite_time=True, eps=1e-8, horizon=5000, reach=m.goal)
    spec = g.make_spec(**okw)
    steps = 5000 if case == "infinite" else K
    if case == "f32":
        assert g.imdp_model_exact_columns(model)[0] > 0  # correction columns in both kernels
    ref = None
    for cfg in CONFIGS:
        raw, k, V, resolved = _run(model, m, spec, cfg, steps)
        assert resolved["kernel"] == cfg["kernel"]
        if ref is None:
            ref = (raw, k, V)
            ost, oV, ok, _, _ = run_oracle(m, **okw)
            # the stopping test compares the residual in each side's arithmetic;
            # at the threshold the two may stop one iteration apart
            assert abs(k - ok) <= (1 if case == "infinite" else 0)
            tol = TOL_F64 * max(1.0, float(np.max(np.abs(oV))))
            if case.startswith("f32"):
                tol = K * model.error_bound() + TOL_F64
            if case == "infinite":
                tol = 1e-7
            assert float(np.max(np.abs(V - oV))) <= tol
        else:
            assert k == ref[1], cfg
            assert np.array_equal(raw, ref[0]), cfg
    model.close()


def test_heterogeneous_batch_direct_equals_ring():
    ms = [banded_imdp(150 + 40 * i, 1 + i % 3, (150 + 40 * i) * (1 + i % 3) * (8 + 7 * i) + 1, seed=80 + i)
          for i in range(6)]
    models = [g.create_model(x) for x in ms]
    specs = [g.make_spec(horizon=10 + 5 * i, reach=x.goal, pessimistic=i % 2 == 0) for i, x in enumerate(ms)]
    outs = {}
    for cfg in (dict(kernel=g.KERNEL_RING), dict(kernel=g.KERNEL_DIRECT, ctas_per_sm=4, tile_entries=256),
                dict(kernel=g.KERNEL_SLICE)):
        sess = g.imdp_session_create(models, specs)
        g.imdp_session_set_launch(sess, **cfg)
        g.imdp_session_run(sess)
        outs[cfg["kernel"]] = [g.imdp_session_checkpoint(sess, i) for i in range(len(ms))]
        sess.close()
    for other in (g.KERNEL_DIRECT, g.KERNEL_SLICE):
        for (ra, ka), (rb, kb) in zip(outs[g.KERNEL_RING], outs[other]):
            assert ka == kb and np.array_equal(ra, rb)


def test_autotune_picks_a_config_and_caches_it(tmp_path):
    m = banded_batch(64, 120, 1, 120 * 30 + 120 + 1, eps=0.05, seed=7)
    model = g.create_model(m)
    spec = g.make_spec(horizon=30, reach=m.goal)
    cache = str(tmp_path / "tuned.json")
    sess = g.imdp_session_create([model], [spec])
    cfg, ms = g.imdp_session_autotune(sess, 8, cache)
    assert ms > 0 and cfg["kernel"] in (g.KERNEL_RING, g.KERNEL_DIRECT, g.KERNEL_SLICE)
    data = json.load(open(cache))
    assert len(data) == 1
    entry = next(iter(data.values()))
    assert entry["kernel"] == cfg["kernel"] and entry["ms_per_iter"] > 0
    # the tuned session still answers the query exactly
    g.imdp_session_run(sess)
    V = np.zeros(m.n_states)
    g.imdp_session_read(sess, 0, V)
    _, oV, _, _, _ = run_oracle(m, horizon=30, reach=m.goal)
    np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64)
    sess.close()
    # a second session of the same shape takes the cached choice without timing
    sess2 = g.imdp_session_create([model], [spec])
    cfg2, ms2 = g.imdp_session_autotune(sess2, 8, cache)
    assert ms2 == 0.0 and cfg2 == cfg
    sess2.close()
    assert os.path.exists(cache)


@pytest.mark.parametrize("cfg", [dict(kernel=g.KERNEL_RING), dict(kernel=g.KERNEL_DIRECT, tile_entries=512),
                                 dict(kernel=g.KERNEL_SLICE)])
def test_finished_problems_leave_the_tile_walk(cfg):
    # Problems of different horizons (the longest not first) and one infinite
    # horizon in one session: launches walk only the running problems' tiles.
    # Every result equals the problem run alone, to the bit, and a restore into
    # the finished session brings a problem's tiles back.
    ms = [banded_imdp(200 + 30 * i, 1 + i % 2, (200 + 30 * i) * (1 + i % 2) * 12 + 1, seed=90 + i) for i in range(5)]
    models = [g.create_model(x) for x in ms]
    horizons = [7, 40, 3, 25, None]
    specs = [g.make_spec(horizon=h, reach=x.goal) if h else
             g.make_spec(infinite_time=True, eps=1e-9, horizon=100000, reach=x.goal) for x, h in zip(ms, horizons)]
    sess = g.imdp_session_create(models, specs)
    g.imdp_session_set_launch(sess, **cfg)
    g.imdp_session_run(sess)
    for i, (x, sp) in enumerate(zip(ms, specs)):
        raw, k = g.imdp_session_checkpoint(sess, i)
        alone = g.imdp_session_create([models[i]], [sp])
        g.imdp_session_set_launch(alone, **cfg)
        g.imdp_session_run(alone)
        raw1, k1 = g.imdp_session_checkpoint(alone, 0)
        alone.close()
        assert k == k1 and np.array_equal(raw, raw1), i
    # every problem is done: restore problem 1 to iteration 10 and run again
    raw_full, k_full = g.imdp_session_checkpoint(sess, 1)
    first = g.imdp_session_create([models[1]], [specs[1]])
    g.imdp_session_step(first, 10)
    raw10, k10 = g.imdp_session_checkpoint(first, 0)
    first.close()
    g.imdp_session_restore(sess, 1, raw10, k10)
    g.imdp_session_run(sess)
    V, kk = np.zeros(ms[1].n_states), [0]
    g.imdp_session_read(sess, 1, V, kk)
    assert kk[0] == 40
    _, oV, _, _, _ = run_oracle(ms[1], horizon=40, reach=ms[1].goal)
    np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64)
    sess.close()


@pytest.mark.parametrize("case", ["reach", "reach_avoid", "reward", "infinite", "policy", "f32"])
def test_single_cta_kernel_matches_tiled_kernels(case):
    # A session of one small problem runs all its iterations in one launch of
    # one CTA (the rule picks it); the tiled kernels give the same words.
    m = banded_imdp(120, 3, 120 * 3 * 8 + 120 * 3 + 1, eps=0.1, seed=70)
    # short columns round finely: a budget this small keeps some of them exact
    model = g.create_model(m, dtype=g.IMDP_F32, budget=7e-10) if case == "f32" else g.create_model(m)
    if case == "f32":
        assert g.imdp_model_exact_columns(model)[0] > 0
    K = 30
    okw = dict(horizon=K, reach=m.goal)
    if case == "reach_avoid":
        okw.update(property=g.IMDP_REACH_AVOID, avoid=np.setdiff1d(np.arange(0, m.n_states, 17), m.goal),
                   pessimistic=False)
    elif case == "reward":
        okw = dict(property=g.IMDP_REWARD, horizon=K, reward=np.linspace(-1.0, 2.0, m.n_states), discount=0.95,
                   maximize=False)
    elif case == "infinite":
        okw = dict(infinite_time=True, eps=1e-9, horizon=100000, reach=m.goal)
    spec = g.make_spec(**okw)
    outs = []
    for kernel in (g.KERNEL_RULE, g.KERNEL_RING, g.KERNEL_DIRECT):
        sess = g.imdp_session_create([model], [spec], want_policy=[1] if case == "policy" else None)
        g.imdp_session_set_launch(sess, kernel=kernel)
        want = g.KERNEL_TINY if kernel == g.KERNEL_RULE else kernel
        assert g.imdp_session_get_launch(sess)["kernel"] == want
        g.imdp_session_run(sess)
        raw, k = g.imdp_session_checkpoint(sess, 0)
        pol = None
        if case == "policy":
            pol = np.zeros((K, m.n_states), np.int32)
            g.imdp_session_read(sess, 0, None, None, None, pol)
        res = np.zeros(m.n_states)
        g.imdp_session_read(sess, 0, None, None, res, check=False)
        outs.append((raw, k, pol, res))
        sess.close()
    for raw, k, pol, res in outs[1:]:
        assert k == outs[0][1] and np.array_equal(raw, outs[0][0])
        assert np.array_equal(res, outs[0][3])
        if pol is not None:
            assert np.array_equal(pol, outs[0][2])
    V = np.zeros(m.n_states)
    st, oV, ok, _, _ = run_oracle(m, **okw)
    sess = g.imdp_session_create([model], [spec])
    g.imdp_session_run(sess)
    g.imdp_session_read(sess, 0, V)
    sess.close()
    tol = TOL_F64 * max(1.0, float(np.max(np.abs(oV))))
    if case == "f32":
        tol = K * model.error_bound() + TOL_F64
    if case == "infinite":
        tol = 1e-8
    assert float(np.max(np.abs(V - oV))) <= tol


def test_single_cta_kernel_stepwise_and_restore():
    # step calls of several sizes (one launch each) equal one long run; a
    # checkpoint taken mid-way resumes there
    m = random_imdp(40, max_actions=3, seed=71)
    model = g.create_model(m)
    spec = g.make_spec(horizon=50, reach=m.goal)
    a = g.imdp_session_create([model], [spec])
    g.imdp_session_run(a)
    ra, ka = g.imdp_session_checkpoint(a, 0)
    b = g.imdp_session_create([model], [spec])
    for n in (1, 7, 16, 3):
        g.imdp_session_step(b, n)
    raw, k = g.imdp_session_checkpoint(b, 0)
    assert k == 27
    c = g.imdp_session_create([model], [spec])
    g.imdp_session_restore(c, 0, raw, k)
    g.imdp_session_run(c)
    g.imdp_session_step(b, 100)  # past the horizon: nothing changes after 50
    rb, kb = g.imdp_session_checkpoint(b, 0)
    rc, kc = g.imdp_session_checkpoint(c, 0)
    assert ka == kb == kc == 50
    assert np.array_equal(ra, rb)
    np.testing.assert_allclose(rc.astype(np.float64), ra.astype(np.float64), rtol=0, atol=1e-13 * 2.0 ** 63)
    for s_ in (a, b, c):
        s_.close()


def _windows(stateptr, cap=256):
    # windows of the slice layout: whole states, at most `cap` columns, one state at least
    n, s, w = len(stateptr) - 1, 0, 0
    while s < n:
        cols = 0
        while s < n and (cols == 0 or cols + stateptr[s + 1] - stateptr[s] <= cap):
            cols += stateptr[s + 1] - stateptr[s]
            s += 1
        w += 1
    return w


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_slice_kernel_windows_switching_and_policy(dtype):
    # States of up to 600 actions (a state of more than 256 columns is a window
    # of its own, several slices, columns dealt by length) beside a model of
    # single-action states; the kernel switched between steps (hints and values
    # carry over); time-dependent policies and the slice layout's windows, all
    # equal to the ring kernel's, to the bit.
    ms = [random_imdp(30, max_actions=600, density=0.3, seed=72),
          banded_imdp(700, 1, 700 * 90 + 700 + 1, eps=0.1, seed=73)]
    budget = 1.5e-9 if dtype == "f32" else None
    models = [g.create_model(x, dtype=g.IMDP_F32 if dtype == "f32" else g.IMDP_F64, budget=budget) for x in ms]
    K = 24
    specs = [g.make_spec(horizon=K, reach=x.goal, pessimistic=i == 0) for i, x in enumerate(ms)]
    pol_ref = None
    runs = [[(K, dict(kernel=g.KERNEL_RING))],
            [(K, dict(kernel=g.KERNEL_SLICE))],
            [(5, dict(kernel=g.KERNEL_SLICE)), (6, dict(kernel=g.KERNEL_DIRECT, tile_entries=700)),
             (7, dict(kernel=g.KERNEL_SLICE, ctas_per_sm=3)), (6, dict(kernel=g.KERNEL_RING))]]
    ref = None
    for plan in runs:
        sess = g.imdp_session_create(models, specs, want_policy=[1, 1])
        for n, cfg in plan:
            g.imdp_session_set_launch(sess, **cfg)
            g.imdp_session_step(sess, n)
        words = [g.imdp_session_checkpoint(sess, i) for i in range(2)]
        pols = []
        for i, x in enumerate(ms):
            pol = np.zeros((K, x.n_states), np.int32)
            g.imdp_session_read(sess, i, None, None, None, pol)
            pols.append(pol)
        if plan[0][1]["kernel"] == g.KERNEL_SLICE and len(plan) == 1:
            nt, nw, _ = g.imdp_session_plan(sess)
            assert nw == 0 and nt == sum(_windows(x.stateptr) for x in ms)
        sess.close()
        if ref is None:
            ref = (words, pols)
            for i, x in enumerate(ms):
                _, oV, _, _, _ = run_oracle(x, horizon=K, reach=x.goal, pessimistic=i == 0)
                V = words[i][0].astype(np.float64) / 2.0 ** 63
                tol = K * models[i].error_bound() + TOL_F64 if dtype == "f32" else TOL_F64
                assert float(np.max(np.abs(V - oV))) <= tol
        else:
            for (ra, ka), (rb, kb) in zip(ref[0], words):
                assert ka == kb == K and np.array_equal(ra, rb)
            for pa, pb in zip(ref[1], pols):
                assert np.array_equal(pa, pb)
    for x in models:
        x.close()


def test_rule_follows_the_batch_shape():
    # By rule (no launch configuration) a session runs the kernel the
    # autotuner picks on GB300 for its shape: long columns the direct kernel
    # (3 CTAs per SM, 1024-entry tiles); short columns the ring kernel while a
    # model has no slice layout, the slice kernel once it has one. The words
    # are those of any other configuration.
    K = 25
    long_m = banded_imdp(300, 2, 300 * 2 * 300 + 300 * 2 + 1, eps=0.05, seed=81)
    short_m = banded_imdp(2000, 1, 2000 * 40 + 2000 + 1, eps=0.05, seed=82)
    assert long_m.nnz >= 256 * long_m.n_cols and short_m.nnz < 256 * short_m.n_cols

    def by_rule(model, m):
        sess = g.imdp_session_create([model], [g.make_spec(horizon=K, reach=m.goal)])
        got = g.imdp_session_get_launch(sess)
        g.imdp_session_step(sess, K)
        raw, k = g.imdp_session_checkpoint(sess, 0)
        sess.close()
        assert k == K
        return got, raw

    def explicit(model, m, cfg):
        sess = g.imdp_session_create([model], [g.make_spec(horizon=K, reach=m.goal)])
        g.imdp_session_set_launch(sess, **cfg)
        g.imdp_session_step(sess, K)
        raw, _ = g.imdp_session_checkpoint(sess, 0)
        sess.close()
        return raw

    mdl = g.create_model(long_m)
    got, raw = by_rule(mdl, long_m)
    assert (got["kernel"], got["ctas_per_sm"], got["tile_entries"]) == (g.KERNEL_DIRECT, 3, 1024)
    np.testing.assert_array_equal(raw, explicit(mdl, long_m, dict(kernel=g.KERNEL_RING, cta_warps=16)))
    mdl.close()

    mdl = g.create_model(short_m)
    got, raw = by_rule(mdl, short_m)
    assert got["kernel"] == g.KERNEL_RING
    # a session that selects the slice kernel builds the model's slice layout
    raw_slice = explicit(mdl, short_m, dict(kernel=g.KERNEL_SLICE))
    got2, raw2 = by_rule(mdl, short_m)
    assert (got2["kernel"], got2["ctas_per_sm"]) == (g.KERNEL_SLICE, 3)
    np.testing.assert_array_equal(raw, raw_slice)
    np.testing.assert_array_equal(raw, raw2)
    _, oV, _, _, _ = run_oracle(short_m, horizon=K, reach=short_m.goal)
    # the one-shot call runs by rule too (now the slice kernel)
    st, V, k, _, _ = g.value_iteration(mdl, short_m.n_states, horizon=K, reach=short_m.goal)
    assert st == "ok" and k == K
    np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64)
    mdl.close()
