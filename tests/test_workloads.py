"""The synthetic generators produce valid models with the paper's table shapes."""
import numpy as np

import oracle
from workloads import CONFIGS, banded_batch, banded_imdp, concat_block_diagonal, make_config, random_imdp


def _valid(m):
    return oracle.validate(oracle.OracleIMDP(m.n_states, m.stateptr, m.colptr, m.rowval, m.lower, m.upper))


def test_linear5_shape():
    m = make_config("linear5")
    assert (m.n_states, m.nnz) == (6, 31)  # linear_5_states_*_0.1_sigma row of the table
    assert _valid(m) == "ok"


def test_banded_shapes_and_feasibility():
    m = banded_imdp(240, 1, 26321, seed=1)
    assert (m.n_states, m.n_cols, m.nnz) == (241, 241, 26321)
    assert _valid(m) == "ok"
    m3 = banded_imdp(500, 3, 500 * 3 * 40, seed=2)
    assert m3.n_states == 501 and m3.n_cols == 1501 and m3.nnz == 60000
    assert _valid(m3) == "ok"


def test_batch_is_block_diagonal_and_deterministic():
    b = banded_batch(16, 60, 2, 60 * 2 * 10 + 60 * 2 + 1, seed=3, stress_frac=0.25)
    assert _valid(b) == "ok"
    off = b.model_state_offsets
    for j in range(b.n_cols):
        s = np.searchsorted(b.stateptr, j, side="right") - 1
        mdl = np.searchsorted(off, s, side="right") - 1
        r = b.rowval[b.colptr[j]:b.colptr[j + 1]]
        assert r.min() >= off[mdl] and r.max() < off[mdl + 1]
    b2 = banded_batch(16, 60, 2, 60 * 2 * 10 + 60 * 2 + 1, seed=3, stress_frac=0.25)
    np.testing.assert_array_equal(b.lower, b2.lower)


def test_concat():
    ms = [random_imdp(5, seed=s) for s in range(3)]
    c = concat_block_diagonal(ms)
    assert c.n_states == 15 and c.nnz == sum(m.nnz for m in ms)
    assert _valid(c) == "ok"


def test_config_table_covers_paper_rows():
    assert {"linear5", "pendulum240_x4096", "cartpole3840", "harrier", "pimdp2"} <= set(CONFIGS)
    assert CONFIGS["pimdp2"]["nnz"] == 48106480 and CONFIGS["harrier"]["nnz"] == 18574307


def test_uneven_batch_shapes_valid_and_thread_independent():
    from workloads.imdp_synth import uneven_batch
    a, Ka = uneven_batch(40, seed=3, threads=1)
    b, Kb = uneven_batch(40, seed=3, threads=4)
    assert np.array_equal(Ka, Kb) and Ka.min() >= 50 and Ka.max() <= 500
    for x, y in zip(a, b):
        for f in ("stateptr", "colptr", "rowval", "lower", "upper", "goal"):
            assert np.array_equal(getattr(x, f), getattr(y, f))
        assert 6 <= x.n_states <= 961
        acts = np.diff(x.stateptr)
        assert 1 <= acts[:-1].min() and acts.max() <= 4 and acts[-1] == 1
        assert x.colptr[-1] == x.nnz and x.rowval.min() >= 0 and x.rowval.max() < x.n_states
        assert x.goal.min() >= 0 and x.goal.max() < x.n_states - 1
        assert oracle.validate(oracle.OracleIMDP(x.n_states, x.stateptr, x.colptr, x.rowval, x.lower,
                                                 x.upper)) == "ok"


def test_served_stream_requests_refer_to_earlier_models():
    from workloads.imdp_synth import served_stream
    models, reqs = served_stream(60, seed=2)
    seen = -1
    for (mi, K, pess, goal) in reqs:
        assert mi <= seen + 1
        seen = max(seen, mi)
        assert 100 <= K <= 500
        n = models[mi].n_states
        assert 50 <= n <= 4000 and goal.min() >= 0 and goal.max() < n - 1
    assert seen + 1 == len(models)
