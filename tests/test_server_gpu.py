"""Continuous-batching server: requests that arrive while others run are admitted
into the running batch; every result equals the same request run alone."""
import time

import numpy as np
import pytest

import oracle
import paper_2401_04068_gb300 as g
from gpu_helpers import TOL_F64, run_oracle
from workloads import banded_imdp, random_imdp

pytestmark = pytest.mark.gpu


def _wait(server, ticket, n):
    V = np.zeros(n)
    k = [0]
    lat = [0.0]
    st = g.imdp_server_wait(server, ticket, 60000.0, V, k, lat)
    return st, V, k[0], lat[0]


@pytest.mark.parametrize("launch", [None, dict(kernel=g.KERNEL_DIRECT, ctas_per_sm=4, tile_entries=1024),
                                    dict(kernel=g.KERNEL_RING, cta_warps=16, wide_col=300)])
def test_server_mixed_stream_matches_alone(launch):
    models_in = [banded_imdp(300, 2, 300 * 2 * 20 + 1, seed=60),
                 banded_imdp(150, 3, 150 * 3 * 12 + 1, seed=61),
                 random_imdp(40, max_actions=3, seed=62)]
    models = [g.create_model(m) for m in models_in]
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(24):
        j = int(rng.integers(len(models)))
        m = models_in[j]
        kind = i % 4
        if kind == 0:
            spec = g.make_spec(horizon=int(rng.integers(5, 80)), reach=m.goal, pessimistic=bool(i % 2))
        elif kind == 1:
            spec = g.make_spec(infinite_time=True, eps=1e-7, horizon=100000, reach=m.goal, maximize=False)
        elif kind == 2:
            spec = g.make_spec(property=g.IMDP_REACH_AVOID, horizon=30, reach=m.goal, avoid=[0, 1])
        else:
            spec = g.make_spec(property=g.IMDP_REWARD, horizon=25, reward=np.linspace(-1, 1, m.n_states),
                               discount=0.9, pessimistic=False)
        reqs.append((j, spec))
    server = g.imdp_server_create(256 << 20)
    if launch:  # every launch configuration computes the same words
        g.imdp_server_set_launch(server, **launch)
    tickets = []
    for i, (j, spec) in enumerate(reqs):
        tickets.append(g.imdp_server_submit(server, models[j], spec))
        if i % 6 == 5:
            time.sleep(0.002)  # later requests arrive while earlier ones are on the device
    for (j, spec), t in zip(reqs, tickets):
        m = models_in[j]
        st, V, k, lat = _wait(server, t, m.n_states)
        assert st in (g.IMDP_OK, g.IMDP_ENOCONV), g.STATUS_NAMES[st]
        assert lat > 0.0
        alone = np.zeros(m.n_states)
        ka = [0]
        g.imdp_value_iteration(models[j], spec, alone, ka)
        assert k == ka[0]
        np.testing.assert_array_equal(V, alone)
    st = g.imdp_server_stats(server)
    assert st["chunks"] > 0 and st["mean_requests"] >= 1.0
    assert 0.0 < st["device_ms"] <= 1.05 * st["wall_ms"] + 1.0  # the worker waits for its launches
    server.close()


def test_server_against_oracle_and_errors():
    m = banded_imdp(200, 2, 200 * 2 * 15 + 1, seed=63)
    model = g.create_model(m)
    server = g.imdp_server_create(64 << 20)
    spec = g.make_spec(horizon=40, reach=m.goal)
    t = g.imdp_server_submit(server, model, spec)
    st, V, k, _ = _wait(server, t, m.n_states)
    assert st == g.IMDP_OK and k == 40
    _, oV, _, _, _ = run_oracle(m, horizon=40, reach=m.goal)
    np.testing.assert_allclose(V, oV, atol=TOL_F64)
    # a finished ticket is released; unknown tickets are reported
    assert g.imdp_server_poll(server, t) == g.IMDP_ENOTFOUND
    # a request larger than the whole budget is refused at submit time
    small = g.imdp_server_create(1 << 20)
    big_m = banded_imdp(40000, 1, 40000 * 4 + 1, seed=64)
    with pytest.raises(g.ImdpError) as e:
        g.imdp_server_submit(small, g.create_model(big_m), g.make_spec(horizon=3, reach=big_m.goal))
    assert e.value.status == g.IMDP_ENOMEM
    small.close()
    server.close()


def test_server_admission_waits_for_budget():
    # budget for about two requests at a time: the rest queue and still finish
    m = banded_imdp(2000, 1, 2000 * 8 + 1, seed=65)
    model = g.create_model(m)
    per_req = 2 * 8 * m.n_states + m.n_states + 4 * m.n_cols + 8 * m.n_states
    server = g.imdp_server_create(max(1 << 20, int(2.5 * (per_req + 4096))))
    specs = [g.make_spec(horizon=30 + i, reach=m.goal) for i in range(8)]
    tickets = [g.imdp_server_submit(server, model, s) for s in specs]
    for s, t in zip(specs, tickets):
        st, V, k, _ = _wait(server, t, m.n_states)
        assert st == g.IMDP_OK and k == s.horizon
        alone = np.zeros(m.n_states)
        g.imdp_value_iteration(model, s, alone)
        np.testing.assert_array_equal(V, alone)
    server.close()
