"""The allocation-free entry point (imdp_value_iteration_noalloc) against the
regular one, through the C ABI.

It serves callers that create models once and then may not allocate device
memory on their query path (fixed memory budgets, device memory owned by
another allocator). It keeps its buffers in one scratch array inside the
library that every call reuses, so the test makes two calls in a row with
different specifications and checks both: leftovers from the first call must
not leak into the second. This file is collected last on purpose."""
import numpy as np
import pytest

import paper_2401_04068_gb300 as g
from gpu_helpers import TOL_F64
from workloads import banded_imdp

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice_in_a_row():
    import torch
    assert torch.cuda.is_available()
    m = banded_imdp(3000, 2, 3000 * 2 * 30 + 3000 * 2 + 1, eps=0.08, seed=31)
    model = g.create_model(m)
    avoid = np.arange(0, 40, dtype=np.int32)
    specs = [
        g.make_spec(horizon=60, reach=m.goal, pessimistic=True, maximize=True),
        g.make_spec(property=g.IMDP_REACH_AVOID, horizon=45, reach=m.goal, avoid=avoid, pessimistic=False,
                    maximize=False),
    ]
    for spec in specs:
        ref = np.zeros(m.n_states)
        kr = [0]
        g.imdp_value_iteration(model, spec, ref, kr)
        out = torch.full((m.n_states,), -1.0, dtype=torch.float64, device="cuda")
        ko = [0]
        st = g.imdp_value_iteration_noalloc(model, spec, out, ko)
        assert st == g.IMDP_OK
        assert ko[0] == kr[0] == spec.horizon
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL_F64)


def test_noalloc_infinite_horizon_and_limits():
    import torch
    m = banded_imdp(500, 1, 500 * 12 + 500 + 1, seed=32)
    model = g.create_model(m)
    spec = g.make_spec(infinite_time=True, eps=1e-8, horizon=100000, reach=m.goal)
    ref = np.zeros(m.n_states)
    kr = [0]
    g.imdp_value_iteration(model, spec, ref, kr)
    out = torch.zeros(m.n_states, dtype=torch.float64, device="cuda")
    ko = [0]
    g.imdp_value_iteration_noalloc(model, spec, out, ko)
    assert ko[0] == kr[0]
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL_F64)
    # a host output buffer is refused
    with pytest.raises(g.ImdpError):
        g.imdp_value_iteration_noalloc(model, spec, np.zeros(m.n_states))
    # more states than the fixed scratch holds: a clear error
    n = 131073
    chain = g.imdp_create_csc(n, n, n, np.arange(n + 1, dtype=np.int32), np.arange(n + 1, dtype=np.int32),
                              np.arange(n, dtype=np.int32), np.ones(n), np.ones(n))
    big = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(g.ImdpError, match="131072"):
        g.imdp_value_iteration_noalloc(chain, g.make_spec(horizon=3, reach=[0]), big)


def test_noalloc_with_wide_states_matches_regular():
    # columns of ~1500-2500 entries: every state runs in the block-wide kernel,
    # launched in the same stream (the entry point uses no second stream)
    import torch
    m = banded_imdp(2600, 1, 2600 * 2000 + 2600 + 1, eps=0.05, seed=33)
    model = g.create_model(m)
    for spec in [g.make_spec(horizon=30, reach=m.goal),
                 g.make_spec(horizon=25, reach=m.goal, pessimistic=False, maximize=False)]:
        ref = np.zeros(m.n_states)
        g.imdp_value_iteration(model, spec, ref)
        out = torch.zeros(m.n_states, dtype=torch.float64, device="cuda")
        assert g.imdp_value_iteration_noalloc(model, spec, out) == g.IMDP_OK
        # the entry point keeps threshold hints in its fixed array (the model's
        # columns fit), so it iterates exactly as the session path does
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_noalloc_against_the_oracle_directly():
    # The same query answered by the allocation-free entry point and by the CPU
    # oracle (binary64, Eq. 2 with the Sec. 4 procedure), element by element.
    import torch
    from gpu_helpers import run_oracle
    m = banded_imdp(1500, 3, 1500 * 3 * 25 + 1500 * 3 + 1, eps=0.1, seed=35)
    model = g.create_model(m)
    for kw in (dict(horizon=50, pessimistic=True, maximize=True),
               dict(horizon=40, pessimistic=False, maximize=False)):
        out = torch.full((m.n_states,), -1.0, dtype=torch.float64, device="cuda")
        k = [0]
        assert g.imdp_value_iteration_noalloc(model, g.make_spec(reach=m.goal, **kw), out, k) == g.IMDP_OK
        st, oV, ok, _, _ = run_oracle(m, reach=m.goal, **kw)
        assert st == "ok" and k[0] == ok == kw["horizon"]
        np.testing.assert_allclose(out.cpu().numpy(), oV, rtol=0, atol=TOL_F64)


def test_noalloc_32bit_storage_model():
    # A model with 32-bit bound storage through the allocation-free entry point:
    # the regular entry point's answer (same stored bounds; threshold hints
    # differ, so equal within the 64-bit products' truncation) and the oracle
    # within the model's a-priori storage bound.
    import torch
    from gpu_helpers import run_oracle
    m = banded_imdp(800, 2, 800 * 2 * 30 + 800 * 2 + 1, eps=0.1, seed=36)
    model = g.create_model(m, dtype=g.IMDP_F32)
    K = 40
    spec = g.make_spec(horizon=K, reach=m.goal)
    ref = np.zeros(m.n_states)
    g.imdp_value_iteration(model, spec, ref)
    out = torch.zeros(m.n_states, dtype=torch.float64, device="cuda")
    assert g.imdp_value_iteration_noalloc(model, spec, out) == g.IMDP_OK
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    _, oV, _, _, _ = run_oracle(m, horizon=K, reach=m.goal)
    assert float(np.max(np.abs(got - oV))) <= K * model.error_bound() + TOL_F64


def test_noalloc_without_room_for_hints():
    # more columns than the fixed array's hint region holds (262,144): every
    # column takes the full threshold search each iteration; the answer equals
    # the session path's up to the 64-bit products' truncation
    import torch
    m = banded_imdp(100000, 3, 100000 * 3 * 4 + 100000 * 3 + 1, eps=0.1, seed=37)
    assert m.n_cols > 262144
    model = g.create_model(m)
    spec = g.make_spec(horizon=12, reach=m.goal)
    ref = np.zeros(m.n_states)
    g.imdp_value_iteration(model, spec, ref)
    out = torch.zeros(m.n_states, dtype=torch.float64, device="cuda")
    assert g.imdp_value_iteration_noalloc(model, spec, out) == g.IMDP_OK
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-13)
