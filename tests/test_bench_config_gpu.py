"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the whole 4096-model pendulum batch as one resident session stepped K =
200 times on a stream (graph-captured chunks), and a 200-problem uneven batch
with per-problem horizons. Sampled models (independent blocks) are recomputed
one by one by the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_04068_gb300 as g
from gpu_helpers import TOL_F64
from workloads import make_config
from workloads.imdp_synth import uneven_batch

pytestmark = pytest.mark.gpu


def _block(m, b):
    s0, s1 = int(m.model_state_offsets[b]), int(m.model_state_offsets[b + 1])
    c0, c1 = int(m.stateptr[s0]), int(m.stateptr[s1])
    e0, e1 = int(m.colptr[c0]), int(m.colptr[c1])
    om = oracle.OracleIMDP(s1 - s0, m.stateptr[s0:s1 + 1] - c0, m.colptr[c0:c1 + 1] - e0, m.rowval[e0:e1] - s0,
                           m.lower[e0:e1], m.upper[e0:e1])
    goal = m.goal[(m.goal >= s0) & (m.goal < s1)] - s0
    return om, goal, s0, s1


def test_full_pendulum_batch_as_benchmarked():
    m = make_config("pendulum240_x4096")
    st = torch.cuda.Stream()
    model = g.create_model(m, stream=st)
    sess = g.imdp_session_create([model], [g.make_spec(horizon=200, reach=m.goal)], stream=st)
    for _ in range(2):  # a reset between queries, as in the timed loop
        g.imdp_session_reset(sess, st)
        g.imdp_session_step(sess, 200, st)
    V = torch.empty(m.n_states, dtype=torch.float64, device="cuda")
    k = [0]
    assert g.imdp_session_read(sess, 0, V, k, stream=st) == g.IMDP_OK and k[0] == 200
    V = V.cpu().numpy()
    rng = np.random.default_rng(5)
    for b in sorted(rng.choice(4096, 8, replace=False).tolist()) + [0, 4095]:
        om, goal, s0, s1 = _block(m, b)
        _, oV, ok, _, _ = oracle.value_iteration(om, oracle.OracleSpec(horizon=200, reach=goal))
        assert ok == 200
        np.testing.assert_allclose(V[s0:s1], oV, rtol=0, atol=TOL_F64)
    sess.close()


def test_uneven_batch_per_problem_horizons():
    ms, Ks = uneven_batch(200, seed=17, threads=4)
    models = [g.create_model(x) for x in ms]
    specs = [g.make_spec(horizon=int(K), reach=x.goal) for x, K in zip(ms, Ks)]
    st = torch.cuda.Stream()
    sess = g.imdp_session_create(models, specs, stream=st)
    g.imdp_session_reset(sess, st)
    g.imdp_session_step(sess, int(Ks.max()), st)
    rng = np.random.default_rng(6)
    for i in sorted(rng.choice(200, 10, replace=False).tolist()):
        x = ms[i]
        V = np.zeros(x.n_states)
        k = [0]
        assert g.imdp_session_read(sess, i, V, k, stream=st) == g.IMDP_OK and k[0] == Ks[i]
        om = oracle.OracleIMDP(x.n_states, x.stateptr, x.colptr, x.rowval, x.lower, x.upper)
        _, oV, _, _, _ = oracle.value_iteration(om, oracle.OracleSpec(horizon=int(Ks[i]), reach=x.goal), threads=4)
        np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64)
    sess.close()
