"""Failure detection on the GPU without a fault: with the test hook set, the ring
kernel's producer issues no copies, so every consumer wait runs into its bound
(about 2 s). The kernel records the error and returns; the host reads
IMDP_ETIMEOUT; the context stays usable and the next run is correct."""
import time

import numpy as np
import pytest

import paper_2401_04068_gb300 as g
from gpu_helpers import TOL_F64, run_oracle
from workloads import banded_imdp

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    m = banded_imdp(200, 1, 200 * 10 + 1, seed=95)
    model = g.create_model(m)
    sess = g.imdp_session_create([model], [g.make_spec(horizon=3, reach=m.goal)])
    # the hook starves the ring kernel's waits; a model this small would
    # otherwise run on the single-CTA kernel, which has none
    g.imdp_session_set_launch(sess, kernel=g.KERNEL_RING)
    V = np.zeros(m.n_states)
    g.imdp_debug_stall_producer(True)
    try:
        t = time.time()
        g.imdp_session_step(sess, 1)
        st = g.imdp_session_read(sess, 0, V, check=False)
        elapsed = time.time() - t
    finally:
        g.imdp_debug_stall_producer(False)
    assert st == g.IMDP_ETIMEOUT
    assert elapsed < 30.0  # bounded: the waits gave up on their own
    # the same session, reset, runs normally afterwards
    g.imdp_session_reset(sess)
    g.imdp_session_step(sess, 3)
    k = [0]
    assert g.imdp_session_read(sess, 0, V, k) == g.IMDP_OK and k[0] == 3
    _, oV, _, _, _ = run_oracle(m, horizon=3, reach=m.goal)
    np.testing.assert_allclose(V, oV, rtol=0, atol=TOL_F64)
    sess.close()
