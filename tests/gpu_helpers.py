"""Helpers for the GPU parity tests: run the CUDA path and the oracle on the
same seeded input and compare."""
import numpy as np

import oracle
import paper_2401_04068_gb300 as g

# Tolerance of the 64-bit path against the FP64 oracle: absolute, in V (values
# lie in [0, 1]). Both sides round once per product/sum; over K iterations of a
# non-expansive operator the difference stays below K * k_max * 2^-53
# (200 * 2300 * 1.1e-16 ~ 5e-11), so 1e-10 bounds it with margin.
TOL_F64 = 1e-10


def om(m):
    return oracle.OracleIMDP(m.n_states, m.stateptr, m.colptr, m.rowval, m.lower, m.upper)


def run_gpu(model, n_states, **kw):
    return g.value_iteration(model, n_states, **kw)


def run_oracle(m, policy=False, threads=1, **kw):
    prop = kw.pop("property", oracle.REACH)
    sp = oracle.OracleSpec(property=prop, **kw)
    return oracle.value_iteration(om(m), sp, policy=policy, threads=threads)


def q_values(m, V, pessimistic):
    """Oracle O-maximization value of every column for the given V."""
    q = np.zeros(m.n_cols)
    for j in range(m.n_cols):
        a, b = m.colptr[j], m.colptr[j + 1]
        q[j], _ = oracle.omax_column(V[m.rowval[a:b]], m.lower[a:b], m.upper[a:b], pessimistic)
    return q


def check_policy_row(m, V_prev, pol_row, fixed, pessimistic, maximize, tol=TOL_F64):
    """The chosen action's Q-value must equal the optimum (ties may pick any)."""
    q = q_values(m, V_prev, pessimistic)
    for s in range(m.n_states):
        if s in fixed:
            assert pol_row[s] == -1
            continue
        js = range(m.stateptr[s], m.stateptr[s + 1])
        qs = np.array([q[j] for j in js])
        best = qs.max() if maximize else qs.min()
        a = pol_row[s]
        assert 0 <= a < len(qs), (s, a)
        assert abs(qs[a] - best) <= tol, (s, a, qs, best)
