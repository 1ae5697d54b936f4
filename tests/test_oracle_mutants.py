"""Planted mistakes: each mutant of the oracle's C source must fail at least one
of the pins (exact-rational LP value iteration, worked example, MDP reduction,
policy time index, residual). Mutants are compiled on the CPU into a temporary
directory; the real oracle is untouched."""
import ctypes as C
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle as O
from exact_lp import columns_from_csc, exact_value_iteration
from workloads import random_imdp

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "imdp_oracle.c")

MUTANTS = {
    "ordering direction swapped": ("pessimistic ? cmp_ascending : cmp_descending",
                                   "pessimistic ? cmp_descending : cmp_ascending"),
    "remainder not reduced": ("      rem -= gap;\n", "\n"),
    "threshold takes its full gap": ("      p[o] += rem;\n      break;", "      p[o] += gap;\n      break;"),
    "goal not held at 1": ("fixed[s] = 1; fixed_val[s] = 1.0;", "fixed[s] = 1; fixed_val[s] = 0.0;"),
    "min instead of max over actions": ("(sp->maximize ? (q > opt) : (q < opt))", "(sp->maximize ? (q < opt) : (q > opt))"),
    "rem starts at 0": ("  double rem = 1.0;\n", "  double rem = 0.0;\n"),
    "policy time index reversed": ("int32_t t = K - k;", "int32_t t = k - 1;"),
    "residual sign flipped": ("Vold[s] - Vnew[s] : 0.0", "Vnew[s] - Vold[s] : 0.0"),
}


def _build_mutant(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, (name, old)
    path = os.path.join(tmp, "m.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp, "libm.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", so, path, "-lm"], check=True,
                   capture_output=True)
    lib = C.CDLL(so)
    lib.oracle_value_iteration.argtypes = [C.POINTER(O._CImdp), C.POINTER(O._CSpec), C.POINTER(C.c_double),
                                           C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                           C.c_int32]
    lib.oracle_value_iteration.restype = C.c_int
    return lib


def _run(lib, m, K, pess, maxi, reach):
    om = O.OracleIMDP(m.n_states, m.stateptr, m.colptr, m.rowval, m.lower, m.upper)
    r = np.ascontiguousarray(reach, dtype=np.int32)
    a = np.zeros(1, np.int32)
    cs = O._CSpec(0, 0, K, 0.0, int(pess), int(maxi), O._p(r, C.c_int32), r.size, O._p(a, C.c_int32), 0, None, 1.0)
    V = np.zeros(m.n_states)
    res = np.zeros(m.n_states)
    pol = np.zeros((max(K, 1), m.n_states), np.int32)
    k = C.c_int32(0)
    cm = om._c()
    lib.oracle_value_iteration(C.byref(cm), C.byref(cs), O._p(V, C.c_double), C.byref(k), O._p(res, C.c_double),
                               O._p(pol, C.c_int32), 1)
    return V, res, pol


def _pins_hold(lib):
    """True when the library passes every pin below."""
    for seed in range(3):
        m = random_imdp(5, max_actions=3, density=0.7, seed=seed, exact_grid=32)
        cols = columns_from_csc(m.colptr, m.rowval, m.lower, m.upper)
        K = 4
        for pess, maxi in [(True, True), (False, False), (True, False)]:
            hist, argsets = exact_value_iteration(m.n_states, cols, m.stateptr, m.goal, K, pess, maxi)
            V, res, pol = _run(lib, m, K, pess, maxi, m.goal)
            if np.max(np.abs(V - [float(x) for x in hist[K]])) > 1e-12:
                return False
            if np.max(np.abs(res - [float(a - b) for a, b in zip(hist[K], hist[K - 1])])) > 1e-12:
                return False
            for t in range(K):
                for s in range(m.n_states):
                    opts = argsets[K - t - 1][s]
                    if opts and pol[t][s] not in opts:
                        return False
    return True


def test_real_oracle_passes_the_mutant_harness(tmp_path):
    lib = C.CDLL(O.build_oracle())
    lib.oracle_value_iteration.argtypes = [C.POINTER(O._CImdp), C.POINTER(O._CSpec), C.POINTER(C.c_double),
                                           C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                           C.c_int32]
    assert _pins_hold(lib)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(str(tmp_path), name, old, new)
    assert not _pins_hold(lib), f"pins did not catch: {name}"
