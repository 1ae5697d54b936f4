"""The 32-bit fast path and its correction stage, through the C ABI.

IMDP_F32 stores bounds in 32 bits and keeps values at 32 bits; a column whose
rounding would move one Bellman step (Eq. 2, with the Sec. 4 inner problem)
by more than the per-iteration budget keeps its exact bounds. The model's
error bound is then guaranteed: K iterations stay within K * bound of exact
value iteration, which the oracle computes in binary64."""
import numpy as np
import pytest

import paper_2401_04068_gb300 as g
from gpu_helpers import TOL_F64, run_oracle
from workloads import banded_imdp, make_config

pytestmark = pytest.mark.gpu


def _f32(m, budget=None):
    return g.create_model(m, dtype=g.IMDP_F32, budget=budget)


def test_budget_orders_the_correction_columns():
    # boundary columns carry a large sink probability (coarse 32-bit scale):
    # they are the first to be kept exact as the budget shrinks
    m = banded_imdp(600, 2, 600 * 2 * 60 + 600 * 2 + 1, eps=0.1, seed=50)
    counts, bounds = [], []
    for budget in (1.0, 2e-8, 5e-9, 1e-9, 0.0):
        model = _f32(m, budget)
        n_exact, entries, b = g.imdp_model_exact_columns(model)
        assert b == budget
        counts.append(n_exact)
        bounds.append(model.error_bound())
        if budget >= 2.0 ** -32 + 1e-12:
            # the guarantee: every 32-bit column within the budget
            assert model.error_bound() <= budget + 1e-15
        model.close()
    assert counts[0] == 0 and counts[-1] == m.n_cols
    assert counts == sorted(counts)
    assert bounds == sorted(bounds, reverse=True)


@pytest.mark.parametrize("budget", [None, 1.0, 0.0])
@pytest.mark.parametrize("pess,maxi", [(True, True), (False, False)])
def test_f32_within_its_guaranteed_bound(budget, pess, maxi):
    m = banded_imdp(500, 3, 500 * 3 * 45 + 500 * 3 + 1, eps=0.1, seed=51)
    model = _f32(m, budget)
    K = 80
    st, V, k, res, _ = g.value_iteration(model, m.n_states, horizon=K, reach=m.goal, pessimistic=pess, maximize=maxi)
    _, oV, ok, _, _ = run_oracle(m, horizon=K, reach=m.goal, pessimistic=pess, maximize=maxi)
    assert st == "ok" and k == ok == K
    err = float(np.max(np.abs(V - oV)))
    assert err <= K * model.error_bound() + TOL_F64, (err, K * model.error_bound())
    if budget is None:  # the default budget: 1e-6 over K = 200
        assert K * model.error_bound() <= 200 * 5e-9 + 1e-12
    model.close()


def test_all_exact_columns_differ_from_64bit_only_by_value_rounding():
    m = banded_imdp(400, 2, 400 * 2 * 40 + 400 * 2 + 1, eps=0.05, seed=52)
    K = 60
    a = g.value_iteration(_f32(m, 0.0), m.n_states, horizon=K, reach=m.goal)[1]
    b = g.value_iteration(g.create_model(m), m.n_states, horizon=K, reach=m.goal)[1]
    assert 0.0 < float(np.max(np.abs(a - b))) <= K * 2.0 ** -32 + TOL_F64


def test_f32_reward_and_reach_avoid_with_correction_columns():
    m = banded_imdp(500, 2, 500 * 2 * 50 + 500 * 2 + 1, eps=0.1, seed=53)
    model = _f32(m, 3e-9)
    assert g.imdp_model_exact_columns(model)[0] > 0
    K = 40
    r = np.random.default_rng(4).uniform(0.0, 1.0, m.n_states)
    st, V, k, _, _ = g.value_iteration(model, m.n_states, property=g.IMDP_REWARD, horizon=K, reward=r, discount=0.95)
    _, oV, _, _, _ = run_oracle(m, property=g.IMDP_REWARD, horizon=K, reward=r, discount=0.95)
    span = float(np.max(np.abs(oV))) + 1.0
    assert float(np.max(np.abs(V - oV))) <= K * model.error_bound() * span * 2 + 1e-9
    avoid = np.setdiff1d(np.arange(0, m.n_states, 23), m.goal)
    st, V, k, _, _ = g.value_iteration(model, m.n_states, property=g.IMDP_REACH_AVOID, horizon=K, reach=m.goal,
                                       avoid=avoid)
    _, oV, _, _, _ = run_oracle(m, property=g.IMDP_REACH_AVOID, horizon=K, reach=m.goal, avoid=avoid)
    assert float(np.max(np.abs(V - oV))) <= K * model.error_bound() + TOL_F64


def test_f32_correction_columns_in_wide_states_and_batches():
    # long columns (wide states, block-wide kernel) with correction columns, in a
    # batch beside a 64-bit model: each problem as it is alone, to the bit
    ms = [banded_imdp(1600, 1, 1600 * 1500 + 1600 + 1, eps=0.1, seed=54),
          banded_imdp(300, 2, 300 * 2 * 30 + 300 * 2 + 1, eps=0.1, seed=55)]
    models = [_f32(ms[0]), g.create_model(ms[1])]
    assert g.imdp_model_exact_columns(models[0])[0] > 0
    specs = [g.make_spec(horizon=30, reach=x.goal) for x in ms]
    outs = [np.zeros(x.n_states) for x in ms]
    g.imdp_value_iteration_batch(models, specs, outs)
    alone = g.value_iteration(models[0], ms[0].n_states, horizon=30, reach=ms[0].goal)[1]
    np.testing.assert_array_equal(outs[0], alone)
    _, o0, _, _, _ = run_oracle(ms[0], horizon=30, reach=ms[0].goal)
    assert float(np.max(np.abs(outs[0] - o0))) <= 30 * models[0].error_bound() + TOL_F64
    _, o1, _, _, _ = run_oracle(ms[1], horizon=30, reach=ms[1].goal)
    np.testing.assert_allclose(outs[1], o1, rtol=0, atol=TOL_F64)


def test_f32_pendulum_batch_k200_within_1e6():
    # the 4096-model benchmark batch's shape, the oracle-sized part of it, at the
    # default budget: guaranteed and measured within 1e-6 of binary64
    m = make_config("pendulum240_x4096", n_models=24)
    model = _f32(m)
    K = 200
    st, V, k, _, _ = g.value_iteration(model, m.n_states, horizon=K, reach=m.goal)
    _, oV, _, _, _ = run_oracle(m, horizon=K, reach=m.goal, threads=8)
    err = float(np.max(np.abs(V - oV)))
    assert K * model.error_bound() <= 1e-6 + 1e-12
    assert err <= K * model.error_bound() + TOL_F64


@pytest.mark.parametrize("prop", ["reach", "reward", "reach_slice"])
def test_infinite_horizon_polished_in_64_bit(prop):
    # 32-bit storage to its fixed point, then 64-bit sweeps from there: the
    # result passes the 64-bit path's own stopping test, needs fewer 64-bit
    # sweeps than the 64-bit path alone, and sits within the stopping
    # tolerance of it and of the oracle (binary64)
    m = banded_imdp(800, 2, 800 * 2 * 40 + 800 * 2 + 1, eps=0.1, seed=56)
    m32, m64 = _f32(m), g.create_model(m)
    launch = dict(kernel=g.KERNEL_SLICE) if prop == "reach_slice" else None
    if prop.startswith("reach"):
        kw = dict(infinite_time=True, eps=1e-9, horizon=100000, reach=m.goal)
    else:
        kw = dict(property=g.IMDP_REWARD, infinite_time=True, eps=1e-9, horizon=100000,
                  reward=np.linspace(0.0, 1.0, m.n_states), discount=0.95)
    spec = g.make_spec(**kw)
    V, k, res = np.zeros(m.n_states), [0], np.zeros(m.n_states)
    st, k32 = g.imdp_value_iteration_polished(m32, m64, spec, V, k, res, launch32=launch, launch64=launch)
    assert st == g.IMDP_OK and 0 < k32 < k[0]
    _, V64, k64, res64, _ = g.value_iteration(m64, m.n_states, **kw)
    assert k[0] - k32 < k64  # fewer 64-bit sweeps than the 64-bit path alone
    assert float(np.max(res)) < 1e-9 * max(1.0, float(np.max(np.abs(V64))))  # the 64-bit stopping test held
    _, oV, _, _, _ = run_oracle(m, **kw)
    scale = max(1.0, float(np.max(np.abs(oV))))
    assert float(np.max(np.abs(V - V64))) <= 1e-6 * scale
    assert float(np.max(np.abs(V - oV))) <= 1e-6 * scale
    # wrong arguments: storage types swapped, a finite horizon
    with pytest.raises(g.ImdpError):
        g.imdp_value_iteration_polished(m64, m32, spec, V)
    with pytest.raises(g.ImdpError):
        g.imdp_value_iteration_polished(m32, m64, g.make_spec(horizon=10, reach=m.goal), V)
    m32.close()
    m64.close()
