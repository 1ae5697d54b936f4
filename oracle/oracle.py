"""ctypes wrapper around ``imdp_oracle.c`` (test infrastructure only).

The C file is compiled on first use (or by ``build_oracle()``) with gcc into
``oracle/_build/libimdp_oracle.so``.  Every function here only marshals
arguments; the arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "imdp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libimdp_oracle.so")

REACH, REACH_AVOID, REWARD = 0, 1, 2
STATUS = {0: "ok", 1: "einval", 2: "einfeasible", 3: "enomem", 4: "enoconv"}

_lock = threading.Lock()
_lib = None


class _CImdp(C.Structure):
    _fields_ = [
        ("n_states", C.c_int32),
        ("n_cols", C.c_int32),
        ("stateptr", C.POINTER(C.c_int32)),
        ("colptr", C.POINTER(C.c_int32)),
        ("rowval", C.POINTER(C.c_int32)),
        ("lower", C.POINTER(C.c_double)),
        ("upper", C.POINTER(C.c_double)),
    ]


class _CSpec(C.Structure):
    _fields_ = [
        ("property", C.c_int32),
        ("infinite_time", C.c_int32),
        ("horizon", C.c_int32),
        ("eps", C.c_double),
        ("pessimistic", C.c_int32),
        ("maximize", C.c_int32),
        ("reach", C.POINTER(C.c_int32)),
        ("n_reach", C.c_int32),
        ("avoid", C.POINTER(C.c_int32)),
        ("n_avoid", C.c_int32),
        ("reward", C.POINTER(C.c_double)),
        ("discount", C.c_double),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available). Returns the .so path."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.run(base[:4] + ["-fopenmp"] + base[4:] + ["-fopenmp"], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = C.CDLL(path)
        lib.oracle_validate.argtypes = [C.POINTER(_CImdp), C.c_double]
        lib.oracle_validate.restype = C.c_int
        lib.oracle_value_iteration.argtypes = [
            C.POINTER(_CImdp), C.POINTER(_CSpec), C.POINTER(C.c_double), C.POINTER(C.c_int32),
            C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_int32]
        lib.oracle_value_iteration.restype = C.c_int
        lib.oracle_omax_local.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double)]
        lib.oracle_omax_local.restype = C.c_double
        lib.oracle_has_openmp.restype = C.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


@dataclass
class OracleIMDP:
    """CSC IMDP: columns are (state, action) pairs, rows are destinations."""
    n_states: int
    stateptr: np.ndarray
    colptr: np.ndarray
    rowval: np.ndarray
    lower: np.ndarray
    upper: np.ndarray

    def __post_init__(self):
        self.stateptr = np.ascontiguousarray(self.stateptr, dtype=np.int32)
        self.colptr = np.ascontiguousarray(self.colptr, dtype=np.int32)
        self.rowval = np.ascontiguousarray(self.rowval, dtype=np.int32)
        self.lower = np.ascontiguousarray(self.lower, dtype=np.float64)
        self.upper = np.ascontiguousarray(self.upper, dtype=np.float64)

    @property
    def n_cols(self) -> int:
        return int(self.colptr.shape[0] - 1)

    def _c(self) -> _CImdp:
        return _CImdp(self.n_states, self.n_cols, _p(self.stateptr, C.c_int32), _p(self.colptr, C.c_int32),
                      _p(self.rowval, C.c_int32), _p(self.lower, C.c_double), _p(self.upper, C.c_double))


@dataclass
class OracleSpec:
    property: int = REACH
    infinite_time: bool = False
    horizon: int = 100
    eps: float = 1e-6
    pessimistic: bool = True
    maximize: bool = True
    reach: Sequence[int] = field(default_factory=list)
    avoid: Sequence[int] = field(default_factory=list)
    reward: Optional[np.ndarray] = None
    discount: float = 1.0


def validate(m: OracleIMDP, tol: float = 1e-12) -> str:
    lib = _load()
    cm = m._c()
    return STATUS[lib.oracle_validate(C.byref(cm), tol)]


def value_iteration(m: OracleIMDP, spec: OracleSpec, policy: bool = False, threads: int = 1):
    """Returns (status, V, k, residual, policy_or_None)."""
    lib = _load()
    n = m.n_states
    reach = np.ascontiguousarray(spec.reach, dtype=np.int32)
    avoid = np.ascontiguousarray(spec.avoid, dtype=np.int32)
    reward = (np.ascontiguousarray(spec.reward, dtype=np.float64) if spec.reward is not None
              else np.zeros(1, dtype=np.float64))
    cs = _CSpec(int(spec.property), int(bool(spec.infinite_time)), int(spec.horizon), float(spec.eps),
                int(bool(spec.pessimistic)), int(bool(spec.maximize)),
                _p(reach, C.c_int32), int(reach.size), _p(avoid, C.c_int32), int(avoid.size),
                _p(reward, C.c_double) if spec.reward is not None else None, float(spec.discount))
    V = np.zeros(n, dtype=np.float64)
    res = np.zeros(n, dtype=np.float64)
    k = C.c_int32(0)
    pol = None
    if policy:
        rows = 1 if spec.infinite_time else max(int(spec.horizon), 0)
        pol = np.full((max(rows, 1), n), -2, dtype=np.int32)[:rows]
        pol = np.ascontiguousarray(pol)
    cm = m._c()
    st = lib.oracle_value_iteration(C.byref(cm), C.byref(cs), _p(V, C.c_double), C.byref(k),
                                    _p(res, C.c_double), _p(pol, C.c_int32) if pol is not None else None,
                                    int(threads))
    return STATUS[st], V, int(k.value), res, pol


def omax_column(v_local: np.ndarray, lower: np.ndarray, upper: np.ndarray, pessimistic: bool = True):
    """O-maximization of one column with the destinations' values given locally.
    Returns (q, p)."""
    lib = _load()
    v = np.ascontiguousarray(v_local, dtype=np.float64)
    lo = np.ascontiguousarray(lower, dtype=np.float64)
    up = np.ascontiguousarray(upper, dtype=np.float64)
    p = np.zeros(v.size, dtype=np.float64)
    q = lib.oracle_omax_local(int(v.size), _p(v, C.c_double), _p(lo, C.c_double), _p(up, C.c_double),
                              int(bool(pessimistic)), _p(p, C.c_double))
    return float(q), p


def has_openmp() -> bool:
    return bool(_load().oracle_has_openmp())
