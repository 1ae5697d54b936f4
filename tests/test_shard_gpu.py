"""State-sharded iteration on one GPU: the slices of a model run in lockstep in
one process (each a session on its own slice), exchanging their owned values
after every step through device copies, as the ranks of a sharded run do
through an all-gather. The assembled result must equal the unsharded session
word for word, and the oracle within tolerance."""
import numpy as np
import pytest
import torch

import paper_2401_04068_gb300 as g
from paper_2401_04068_gb300.sharded import SliceRunner
from gpu_helpers import TOL_F64, run_oracle
from workloads import banded_imdp, random_imdp

pytestmark = pytest.mark.gpu


def _lockstep(m, parts, spec_kw, dtype=g.IMDP_F64, launch=None):
    b = g.imdp_partition_states(m.n_states, m.stateptr, m.colptr, parts)
    runners = [SliceRunner(m, b, r, spec_kw, dtype, launch=launch) for r in range(parts)]
    for r in runners:
        r.reset()
    for _ in range(runners[0].horizon):
        owns = [r.step().clone() for r in runners]
        for r in runners:
            r.put(owns)
        if runners[0].infinite:
            # the maximum of the slices' residuals decides, for every slice
            rmax = max(int(r.residual().item()) for r in runners)
            if rmax < runners[0].eps_raw:
                break
    out = []
    for r in runners:
        V = np.zeros(m.n_states)
        k = [0]
        r.read(V, k)
        out.append((V, k[0]))
        r.close()
    return b, out


def _whole(m, spec_kw, dtype=g.IMDP_F64):
    model = g.create_model(m, dtype=dtype)
    V = np.zeros(m.n_states)
    k = [0]
    g.imdp_value_iteration(model, g.make_spec(**spec_kw), V, k)
    return V, k[0]


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("pess,maxi", [(True, True), (False, False)])
@pytest.mark.parametrize("kernel", [g.KERNEL_RULE, g.KERNEL_SLICE])
def test_sharded_equals_whole_reach(parts, pess, maxi, kernel):
    # the slice kernel lays out the owned states of each slice only
    m = banded_imdp(600, 2, 600 * 2 * 25 + 1, seed=81)
    kw = dict(horizon=40, reach=m.goal, pessimistic=pess, maximize=maxi)
    Vw, kw_ = _whole(m, kw)
    b, outs = _lockstep(m, parts, kw, launch=dict(kernel=kernel) if kernel else None)
    for V, k in outs:
        assert k == kw_ == 40
        np.testing.assert_array_equal(V, Vw)  # every slice holds the whole iterate after the last exchange
    _, oV, _, _, _ = run_oracle(m, horizon=40, reach=m.goal, pessimistic=pess, maximize=maxi)
    np.testing.assert_allclose(outs[0][0], oV, atol=TOL_F64)


def test_sharded_reach_avoid_reward_and_f32():
    m = random_imdp(40, max_actions=3, seed=82)
    avoid = np.array([s for s in range(m.n_states) if s not in set(m.goal.tolist())][:3], np.int32)
    kw = dict(property=g.IMDP_REACH_AVOID, horizon=25, reach=m.goal, avoid=avoid)
    Vw, _ = _whole(m, kw)
    _, outs = _lockstep(m, 3, kw)
    np.testing.assert_array_equal(outs[1][0], Vw)
    r = np.linspace(-1.0, 2.0, m.n_states)
    kw = dict(property=g.IMDP_REWARD, horizon=30, reward=r, discount=0.95, pessimistic=False)
    Vw, _ = _whole(m, kw)
    _, outs = _lockstep(m, 2, kw)
    np.testing.assert_array_equal(outs[0][0], Vw)
    m2 = banded_imdp(400, 1, 400 * 30 + 1, seed=83)
    kw = dict(horizon=20, reach=m2.goal)
    Vw, _ = _whole(m2, kw, g.IMDP_F32)
    _, outs = _lockstep(m2, 2, kw, g.IMDP_F32)
    np.testing.assert_array_equal(outs[0][0], Vw)


@pytest.mark.parametrize("parts", [2, 3])
def test_sharded_infinite_horizon_equals_whole(parts):
    # the slices stop on the maximum residual over all of them: the same
    # iteration count and the same words as the unsharded infinite run
    m = banded_imdp(500, 2, 500 * 2 * 20 + 1, eps=0.05, seed=85)
    for kw in (dict(infinite_time=True, eps=1e-8, horizon=100000, reach=m.goal),
               dict(infinite_time=True, eps=1e-6, horizon=100000, reach=m.goal, pessimistic=False, maximize=False)):
        Vw, kw_ = _whole(m, kw)
        b, outs = _lockstep(m, parts, kw)
        for V, k in outs:
            assert k == kw_ > 10
            np.testing.assert_array_equal(V, Vw)
    r = np.linspace(0.0, 1.0, m.n_states)
    kw = dict(property=g.IMDP_REWARD, infinite_time=True, eps=1e-7, horizon=100000, reward=r, discount=0.9)
    Vw, kw_ = _whole(m, kw)
    _, outs = _lockstep(m, 2, kw)
    assert outs[0][1] == kw_
    np.testing.assert_array_equal(outs[0][0], Vw)


def test_slice_errors():
    m = banded_imdp(100, 1, 100 * 10 + 1, seed=84)
    sm = g.create_model_slice(m, 0, 50)
    # an infinite horizon on a slice stops on the residual of all slices: the
    # session may be stepped, but not run to convergence on its own states
    s_inf = g.imdp_session_create([sm], [g.make_spec(infinite_time=True, eps=1e-6, reach=m.goal)])
    with pytest.raises(g.ImdpError) as e:
        g.imdp_session_run(s_inf)
    assert e.value.status == g.IMDP_EINVAL
    with pytest.raises(g.ImdpError):
        g.value_iteration(sm, m.n_states, infinite_time=True, eps=1e-6, reach=m.goal)
    g.imdp_session_step(s_inf, 2)
    res = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.imdp_session_residual(s_inf, 0, 2, 0, 50, res)
    with pytest.raises(g.ImdpError):
        g.imdp_session_residual(s_inf, 0, 0, 0, 50, res)  # k >= 1
    s_inf.close()
    # slices run in sessions only
    srv = g.imdp_server_create(16 << 20)
    with pytest.raises(g.ImdpError):
        g.imdp_server_submit(srv, sm, g.make_spec(horizon=3, reach=m.goal))
    srv.close()
    s = g.imdp_session_create([sm], [g.make_spec(horizon=3, reach=m.goal)])
    buf = torch.zeros(60, dtype=torch.int64, device="cuda")
    with pytest.raises(g.ImdpError):
        g.imdp_session_values_get(s, 0, 0, 0, m.n_states + 1, buf)  # range past the states
    with pytest.raises(g.ImdpError):
        g.imdp_session_values_get(s, 0, 0, 0, 10, np.zeros(10, np.int64))  # host memory
    g.imdp_session_values_get(s, 0, 0, 0, 50, buf)  # V_0 after create: goal states 1 (2^63), others 0
    V0 = buf[:50].cpu().numpy().view(np.uint64)
    goal = set(m.goal.tolist())
    assert all((V0[i] == (1 << 63)) == (i in goal) for i in range(50))
    s.close()
    # a slice stateptr that does not end at n_cols is rejected
    sp, cp, rv, lo, up = g.slice_arrays(m, 0, 50)
    with pytest.raises(g.ImdpError):
        g.imdp_create_csc_slice(m.n_states, 0, 49, len(cp) - 1, len(rv), sp, cp, rv, lo, up)
    sm.close()


def test_run_sharded_through_nccl_on_a_side_stream():
    # The library's driver as a caller runs it: one rank of an NCCL group, the
    # slice's session on its own stream, the exchange ordered after each step
    # on the device (no host wait per step); finite and infinite horizons equal
    # the unsharded session word for word.
    import socket
    import torch.distributed as dist
    from paper_2401_04068_gb300.sharded import run_sharded
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        m = banded_imdp(700, 2, 700 * 2 * 30 + 1, seed=86)
        st = torch.cuda.Stream()
        for kw in (dict(horizon=60, reach=m.goal),
                   dict(infinite_time=True, eps=1e-8, horizon=100000, reach=m.goal)):
            Vw, kw_ = _whole(m, kw)
            V, k = run_sharded(m, kw, 0, 1, stream=st)
            assert k == kw_
            np.testing.assert_array_equal(V, Vw)
    finally:
        dist.destroy_process_group()
