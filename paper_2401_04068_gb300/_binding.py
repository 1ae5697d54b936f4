"""ctypes binding of include/imdp.h: the same entry points, argument marshalling only.

Buffers may be numpy arrays (host) or CUDA torch tensors (device); pointers are
passed through unchanged and every computation runs in the CUDA library.  The
library is loaded from the package's ``_build`` directory; a missing library is
an error (there is no CPU fallback)."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

IMDP_OK, IMDP_EINVAL, IMDP_EINFEASIBLE, IMDP_ENOMEM, IMDP_EDEVICE = 0, 1, 2, 3, 4
IMDP_ETIMEOUT, IMDP_EBUSY, IMDP_ENOCONV, IMDP_ENOTFOUND, IMDP_EPENDING, IMDP_EIO = 5, 6, 7, 8, 9, 10
IMDP_F64, IMDP_F32 = 0, 1
IMDP_REACH, IMDP_REACH_AVOID, IMDP_REWARD = 0, 1, 2

STATUS_NAMES = {0: "ok", 1: "einval", 2: "einfeasible", 3: "enomem", 4: "edevice", 5: "etimeout", 6: "ebusy",
                7: "enoconv", 8: "enotfound", 9: "epending", 10: "eio"}

# Every symbol include/imdp.h declares (checked by the tests).
EXPORTED = [
    "imdp_status_string", "imdp_last_error", "imdp_version", "imdp_create_csc", "imdp_create_dense",
    "imdp_model_destroy", "imdp_model_info", "imdp_value_iteration", "imdp_value_iteration_batch",
    "imdp_session_create", "imdp_session_reset", "imdp_session_step", "imdp_session_run", "imdp_session_read",
    "imdp_session_launches", "imdp_session_destroy", "imdp_value_iteration_noalloc",
    "imdp_server_create", "imdp_server_submit", "imdp_server_poll", "imdp_server_wait", "imdp_server_destroy",
    "imdp_model_error_bound", "imdp_partition_states", "imdp_create_csc_slice", "imdp_session_values_get",
    "imdp_session_values_put", "imdp_model_plan", "imdp_debug_stall_producer",
    "imdp_read_bmdp_tool", "imdp_write_bmdp_tool", "imdp_read_prism", "imdp_write_prism", "imdp_file_free",
    "imdp_session_checkpoint", "imdp_session_restore",
    "imdp_session_set_launch", "imdp_session_get_launch", "imdp_session_autotune", "imdp_session_plan",
    "imdp_create_csc_f32", "imdp_model_exact_columns", "imdp_session_residual", "imdp_session_stop_threshold",
    "imdp_server_set_launch", "imdp_server_stats", "imdp_value_iteration_polished",
]


class imdp_launch_config(C.Structure):
    _fields_ = [
        ("kernel", C.c_int32),
        ("cta_warps", C.c_int32),
        ("ctas_per_sm", C.c_int32),
        ("tile_entries", C.c_int32),
        ("wide_col", C.c_int32),
    ]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


KERNEL_RULE, KERNEL_RING, KERNEL_DIRECT, KERNEL_TINY, KERNEL_SLICE = 0, 1, 2, 3, 4


class ImdpError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({detail})")
        self.status = status


class imdp_spec(C.Structure):
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


class imdp_file(C.Structure):
    _fields_ = [
        ("n_states", C.c_int32),
        ("n_cols", C.c_int32),
        ("nnz", C.c_int64),
        ("stateptr", C.POINTER(C.c_int32)),
        ("colptr", C.POINTER(C.c_int32)),
        ("rowval", C.POINTER(C.c_int32)),
        ("lower", C.POINTER(C.c_double)),
        ("upper", C.POINTER(C.c_double)),
        ("action", C.POINTER(C.c_int32)),
        ("spec", imdp_spec),
    ]


_lib = None
_LIB_PATH = _build.LIB


def library_path() -> str:
    return _LIB_PATH


def load(path: Optional[str] = None):
    """Load the CUDA library (it must have been built; see ``build.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CUDA library not built: {p} (run python -m paper_2401_04068_gb300.build)")
    lib = C.CDLL(p)
    vp = C.c_void_p
    lib.imdp_status_string.argtypes = [C.c_int]
    lib.imdp_status_string.restype = C.c_char_p
    lib.imdp_last_error.restype = C.c_char_p
    lib.imdp_version.restype = C.c_char_p
    lib.imdp_create_csc.argtypes = [C.c_int32, C.c_int32, C.c_int64, vp, vp, vp, vp, vp, C.c_int, vp,
                                    C.POINTER(vp)]
    lib.imdp_create_dense.argtypes = [C.c_int32, vp, vp, vp, C.c_int, vp, C.POINTER(vp)]
    lib.imdp_create_csc_f32.argtypes = [C.c_int32, C.c_int32, C.c_int64, vp, vp, vp, vp, vp, C.c_double, vp,
                                        C.POINTER(vp)]
    lib.imdp_model_exact_columns.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)]
    lib.imdp_model_destroy.argtypes = [vp]
    lib.imdp_model_destroy.restype = None
    lib.imdp_model_info.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_size_t), C.POINTER(C.c_int32)]
    lib.imdp_value_iteration.argtypes = [vp, C.POINTER(imdp_spec), vp, C.POINTER(C.c_int32), vp, vp, vp]
    lib.imdp_value_iteration_polished.argtypes = [vp, vp, C.POINTER(imdp_spec), C.POINTER(imdp_launch_config),
                                                  C.POINTER(imdp_launch_config), vp, C.POINTER(C.c_int32),
                                                  C.POINTER(C.c_int32), vp, vp, vp]
    lib.imdp_value_iteration_batch.argtypes = [C.POINTER(vp), C.POINTER(imdp_spec), C.c_int32, C.POINTER(vp),
                                               C.POINTER(C.c_int32), vp]
    lib.imdp_session_create.argtypes = [C.POINTER(vp), C.POINTER(imdp_spec), C.c_int32, vp, vp, C.POINTER(vp)]
    lib.imdp_session_set_launch.argtypes = [vp, C.POINTER(imdp_launch_config), vp]
    lib.imdp_session_get_launch.argtypes = [vp, C.POINTER(imdp_launch_config)]
    lib.imdp_session_plan.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    lib.imdp_server_set_launch.argtypes = [vp, C.POINTER(imdp_launch_config)]
    lib.imdp_server_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_double)]
    lib.imdp_session_residual.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, vp]
    lib.imdp_session_stop_threshold.argtypes = [vp, C.c_int32, C.POINTER(C.c_uint64)]
    lib.imdp_session_autotune.argtypes = [vp, C.c_int32, C.c_char_p, vp, C.POINTER(imdp_launch_config),
                                          C.POINTER(C.c_double)]
    lib.imdp_session_reset.argtypes = [vp, vp]
    lib.imdp_session_step.argtypes = [vp, C.c_int32, vp]
    lib.imdp_session_run.argtypes = [vp, C.c_int32, vp]
    lib.imdp_session_read.argtypes = [vp, C.c_int32, vp, C.POINTER(C.c_int32), vp, vp, vp]
    lib.imdp_session_launches.argtypes = [vp]
    lib.imdp_session_launches.restype = C.c_int64
    lib.imdp_session_destroy.argtypes = [vp]
    lib.imdp_session_destroy.restype = None
    lib.imdp_value_iteration_noalloc.argtypes = [vp, C.POINTER(imdp_spec), vp, C.POINTER(C.c_int32), vp]
    lib.imdp_value_iteration_noalloc.restype = C.c_int
    lib.imdp_server_create.argtypes = [C.c_size_t, C.POINTER(vp)]
    lib.imdp_server_create.restype = C.c_int
    lib.imdp_server_submit.argtypes = [vp, vp, C.POINTER(imdp_spec), C.POINTER(C.c_uint64)]
    lib.imdp_server_submit.restype = C.c_int
    lib.imdp_server_poll.argtypes = [vp, C.c_uint64, vp, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.imdp_server_poll.restype = C.c_int
    lib.imdp_server_wait.argtypes = [vp, C.c_uint64, C.c_double, vp, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.imdp_server_wait.restype = C.c_int
    lib.imdp_model_error_bound.argtypes = [vp, C.POINTER(C.c_double)]
    lib.imdp_model_error_bound.restype = C.c_int
    lib.imdp_server_destroy.argtypes = [vp]
    lib.imdp_server_destroy.restype = None
    lib.imdp_debug_stall_producer.argtypes = [C.c_int32]
    lib.imdp_debug_stall_producer.restype = None
    lib.imdp_model_plan.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    lib.imdp_model_plan.restype = C.c_int
    lib.imdp_partition_states.argtypes = [C.c_int32, vp, vp, C.c_int32, vp]
    lib.imdp_partition_states.restype = C.c_int
    lib.imdp_create_csc_slice.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64, vp, vp, vp, vp, vp,
                                          C.c_int, vp, C.POINTER(vp)]
    lib.imdp_create_csc_slice.restype = C.c_int
    lib.imdp_read_bmdp_tool.argtypes = [C.c_char_p, C.POINTER(C.POINTER(imdp_file))]
    lib.imdp_read_prism.argtypes = [C.c_char_p, C.POINTER(C.POINTER(imdp_file))]
    lib.imdp_write_bmdp_tool.argtypes = [C.c_char_p, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp, C.c_int32]
    lib.imdp_write_prism.argtypes = [C.c_char_p, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, C.POINTER(imdp_spec)]
    for f in ("imdp_read_bmdp_tool", "imdp_read_prism", "imdp_write_bmdp_tool", "imdp_write_prism"):
        getattr(lib, f).restype = C.c_int
    lib.imdp_session_checkpoint.argtypes = [vp, C.c_int32, vp, C.POINTER(C.c_int32), vp]
    lib.imdp_session_checkpoint.restype = C.c_int
    lib.imdp_session_restore.argtypes = [vp, C.c_int32, vp, C.c_int32, vp]
    lib.imdp_session_restore.restype = C.c_int
    lib.imdp_file_free.argtypes = [C.POINTER(imdp_file)]
    lib.imdp_file_free.restype = None
    for f in ("imdp_session_values_get", "imdp_session_values_put"):
        getattr(lib, f).argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, vp]
        getattr(lib, f).restype = C.c_int
    for f in ("imdp_create_csc", "imdp_create_dense", "imdp_model_info", "imdp_value_iteration",
              "imdp_value_iteration_batch", "imdp_session_create", "imdp_session_reset", "imdp_session_step",
              "imdp_session_run", "imdp_session_read"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _ptr(x) -> Optional[int]:
    """Raw address of a numpy array or a torch tensor (None stays None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _check(status: int, where: str):
    if status != IMDP_OK:
        raise ImdpError(status, where, load().imdp_last_error().decode(errors="replace"))


def imdp_status_string(status: int) -> str:
    return load().imdp_status_string(int(status)).decode()


def imdp_last_error() -> str:
    return load().imdp_last_error().decode(errors="replace")


def imdp_version() -> str:
    return load().imdp_version().decode()


class Model:
    """Owns an ``imdp_model*``; frees it on ``close()`` / garbage collection."""

    def __init__(self, handle: int):
        self.handle = handle

    def close(self):
        if self.handle:
            load().imdp_model_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error_bound(self) -> float:
        d = C.c_double(0.0)
        _check(load().imdp_model_error_bound(C.c_void_p(self.handle), C.byref(d)), "imdp_model_error_bound")
        return d.value

    def info(self):
        ns, nc, nz, mc = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32()
        by = C.c_size_t()
        _check(load().imdp_model_info(C.c_void_p(self.handle), C.byref(ns), C.byref(nc), C.byref(nz), C.byref(by),
                                      C.byref(mc)), "imdp_model_info")
        return dict(n_states=ns.value, n_cols=nc.value, nnz=nz.value, device_bytes=by.value, max_col_nnz=mc.value)


def imdp_create_csc(n_states, n_cols, nnz, stateptr, colptr, rowval, lower, upper, dtype=IMDP_F64,
                    stream=None) -> Model:
    out = C.c_void_p()
    st = load().imdp_create_csc(int(n_states), int(n_cols), int(nnz), _ptr(stateptr), _ptr(colptr), _ptr(rowval),
                                _ptr(lower), _ptr(upper), int(dtype), _stream(stream), C.byref(out))
    _check(st, "imdp_create_csc")
    return Model(out.value)


def imdp_create_csc_f32(n_states, n_cols, nnz, stateptr, colptr, rowval, lower, upper, budget_per_iteration,
                        stream=None) -> Model:
    """32-bit storage with correction columns chosen by a per-iteration error budget."""
    out = C.c_void_p()
    st = load().imdp_create_csc_f32(int(n_states), int(n_cols), int(nnz), _ptr(stateptr), _ptr(colptr),
                                    _ptr(rowval), _ptr(lower), _ptr(upper), float(budget_per_iteration),
                                    _stream(stream), C.byref(out))
    _check(st, "imdp_create_csc_f32")
    return Model(out.value)


def imdp_model_exact_columns(model: Model):
    """(correction columns, their transitions, the budget they were chosen by) of an IMDP_F32 model."""
    n, e, b = C.c_int32(0), C.c_int64(0), C.c_double(0.0)
    _check(load().imdp_model_exact_columns(C.c_void_p(model.handle), C.byref(n), C.byref(e), C.byref(b)),
           "imdp_model_exact_columns")
    return n.value, e.value, b.value


def imdp_create_dense(n_states, n_actions, lower, upper, dtype=IMDP_F64, stream=None) -> Model:
    out = C.c_void_p()
    st = load().imdp_create_dense(int(n_states), _ptr(n_actions), _ptr(lower), _ptr(upper), int(dtype),
                                  _stream(stream), C.byref(out))
    _check(st, "imdp_create_dense")
    return Model(out.value)


def imdp_model_destroy(model: Model):
    model.close()


def make_spec(property=IMDP_REACH, infinite_time=False, horizon=100, eps=1e-6, pessimistic=True, maximize=True,
              reach=(), avoid=(), reward=None, discount=1.0):
    """Build an ``imdp_spec`` plus the arrays it points to (keep both alive)."""
    keep = []
    r = np.ascontiguousarray(reach, dtype=np.int32)
    a = np.ascontiguousarray(avoid, dtype=np.int32)
    keep += [r, a]
    rw = None
    if reward is not None:
        rw = np.ascontiguousarray(reward, dtype=np.float64)
        keep.append(rw)
    s = imdp_spec(int(property), int(bool(infinite_time)), int(horizon), float(eps), int(bool(pessimistic)),
                  int(bool(maximize)), r.ctypes.data_as(C.POINTER(C.c_int32)), int(r.size),
                  a.ctypes.data_as(C.POINTER(C.c_int32)), int(a.size),
                  rw.ctypes.data_as(C.POINTER(C.c_double)) if rw is not None else None, float(discount))
    s._keep = keep
    return s


def imdp_value_iteration(model: Model, spec, V_out, k_out=None, residual_out=None, policy_out=None, stream=None,
                         check=True) -> int:
    """Raw call: V_out / residual_out / policy_out are caller buffers (host numpy
    or device torch). Returns the status; k is written to ``k_out[0]`` when given."""
    k = C.c_int32(0)
    st = load().imdp_value_iteration(C.c_void_p(model.handle), C.byref(spec), _ptr(V_out), C.byref(k),
                                     _ptr(residual_out), _ptr(policy_out), _stream(stream))
    if k_out is not None:
        k_out[0] = k.value
    if check and st not in (IMDP_OK, IMDP_ENOCONV):
        _check(st, "imdp_value_iteration")
    return st


def imdp_value_iteration_polished(model32: Model, model64: Model, spec, V_out, k_out=None, residual_out=None,
                                  policy_out=None, stream=None, check=True, launch32: Optional[dict] = None,
                                  launch64: Optional[dict] = None):
    """Raw call: the infinite-horizon query on 32-bit storage, then polished on the
    64-bit model (``launch32`` / ``launch64``: launch configuration fields of the
    two phases, None: by rule). Returns (status, iterations on 32-bit storage); all
    iterations go to ``k_out[0]`` when given."""
    def cfg(d):
        if d is None:
            return None
        c = imdp_launch_config()
        for f, _ in imdp_launch_config._fields_:
            setattr(c, f, int(d.get(f, 0)))
        return C.byref(c)
    k32, k = C.c_int32(0), C.c_int32(0)
    st = load().imdp_value_iteration_polished(C.c_void_p(model32.handle), C.c_void_p(model64.handle), C.byref(spec),
                                              cfg(launch32), cfg(launch64), _ptr(V_out), C.byref(k32), C.byref(k),
                                              _ptr(residual_out), _ptr(policy_out), _stream(stream))
    if k_out is not None:
        k_out[0] = k.value
    if check and st not in (IMDP_OK, IMDP_ENOCONV):
        _check(st, "imdp_value_iteration_polished")
    return st, k32.value


def imdp_value_iteration_batch(models: Sequence[Model], specs: Sequence, V_out: Sequence, k_out=None, stream=None,
                               check=True) -> int:
    n = len(models)
    hs = (C.c_void_p * n)(*[m.handle for m in models])
    sp = (imdp_spec * n)(*specs)
    vo = (C.c_void_p * n)(*[_ptr(v) for v in V_out])
    ks = (C.c_int32 * n)()
    st = load().imdp_value_iteration_batch(hs, sp, n, vo, ks, _stream(stream))
    if k_out is not None:
        for i in range(n):
            k_out[i] = ks[i]
    if check and st not in (IMDP_OK, IMDP_ENOCONV):
        _check(st, "imdp_value_iteration_batch")
    return st


class Session:
    """Owns an ``imdp_session*`` (resident value-iteration state for a batch)."""

    def __init__(self, handle: int, models):
        self.handle = handle
        self._models = list(models)  # keep the models alive

    def close(self):
        if self.handle:
            load().imdp_session_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def imdp_session_create(models: Sequence[Model], specs: Sequence, want_policy=None, stream=None) -> Session:
    n = len(models)
    hs = (C.c_void_p * n)(*[m.handle for m in models])
    sp = (imdp_spec * n)(*specs)
    wp = None
    if want_policy is not None:
        wp = np.ascontiguousarray(want_policy, dtype=np.int32)
    out = C.c_void_p()
    st = load().imdp_session_create(hs, sp, n, _ptr(wp), _stream(stream), C.byref(out))
    _check(st, "imdp_session_create")
    return Session(out.value, models)


def imdp_session_reset(s: Session, stream=None):
    _check(load().imdp_session_reset(C.c_void_p(s.handle), _stream(stream)), "imdp_session_reset")


def imdp_session_step(s: Session, n_iters: int, stream=None):
    _check(load().imdp_session_step(C.c_void_p(s.handle), int(n_iters), _stream(stream)), "imdp_session_step")


def imdp_session_run(s: Session, check_every: int = 32, stream=None):
    _check(load().imdp_session_run(C.c_void_p(s.handle), int(check_every), _stream(stream)), "imdp_session_run")


def imdp_session_read(s: Session, index: int, V_out=None, k_out=None, residual_out=None, policy_out=None,
                      stream=None, check=True) -> int:
    k = C.c_int32(0)
    st = load().imdp_session_read(C.c_void_p(s.handle), int(index), _ptr(V_out), C.byref(k), _ptr(residual_out),
                                  _ptr(policy_out), _stream(stream))
    if k_out is not None:
        k_out[0] = k.value
    if check and st not in (IMDP_OK, IMDP_ENOCONV):
        _check(st, "imdp_session_read")
    return st


def imdp_session_launches(s: Session) -> int:
    return int(load().imdp_session_launches(C.c_void_p(s.handle)))


def imdp_session_destroy(s: Session):
    s.close()


def imdp_session_set_launch(s: Session, kernel: int = 0, cta_warps: int = 0, ctas_per_sm: int = 0,
                            tile_entries: int = 0, wide_col: int = 0, stream=None):
    """Launch configuration of the session's Bellman step (0 fields: by rule)."""
    cfg = imdp_launch_config(kernel, cta_warps, ctas_per_sm, tile_entries, wide_col)
    _check(load().imdp_session_set_launch(C.c_void_p(s.handle), C.byref(cfg), _stream(stream)),
           "imdp_session_set_launch")


def imdp_session_get_launch(s: Session) -> dict:
    """The resolved launch configuration of the session."""
    cfg = imdp_launch_config()
    _check(load().imdp_session_get_launch(C.c_void_p(s.handle), C.byref(cfg)), "imdp_session_get_launch")
    return cfg.as_dict()


def imdp_session_residual(s: Session, index: int, k: int, s0: int, s1: int, dst, stream=None):
    """max |V_k - V_{k-1}| over states [s0, s1) (raw word) into one device word ``dst``."""
    _check(load().imdp_session_residual(C.c_void_p(s.handle), int(index), int(k), int(s0), int(s1), _ptr(dst),
                                        _stream(stream)), "imdp_session_residual")


def imdp_session_stop_threshold(s: Session, index: int) -> int:
    """Raw threshold of the infinite-horizon stopping test of problem ``index``."""
    e = C.c_uint64(0)
    _check(load().imdp_session_stop_threshold(C.c_void_p(s.handle), int(index), C.byref(e)),
           "imdp_session_stop_threshold")
    return int(e.value)


def imdp_session_plan(s: Session):
    """(tiles, wide states, transitions of wide states) of the session's current tile plan."""
    t, w, e = C.c_int32(0), C.c_int32(0), C.c_int64(0)
    _check(load().imdp_session_plan(C.c_void_p(s.handle), C.byref(t), C.byref(w), C.byref(e)), "imdp_session_plan")
    return t.value, w.value, e.value


def imdp_session_autotune(s: Session, iters: int, cache_path: Optional[str] = None, stream=None):
    """Time the candidate launch configurations (or take the cached choice) and
    keep the fastest. Returns (configuration dict, ms per iteration; 0 when cached)."""
    cfg = imdp_launch_config()
    ms = C.c_double(0.0)
    _check(load().imdp_session_autotune(C.c_void_p(s.handle), int(iters),
                                        cache_path.encode() if cache_path else None, _stream(stream),
                                        C.byref(cfg), C.byref(ms)), "imdp_session_autotune")
    return cfg.as_dict(), float(ms.value)


def imdp_value_iteration_noalloc(model: Model, spec, V_out, k_out=None, stream=None, check=True) -> int:
    """Value iteration using only the library's fixed scratch array (no device
    allocation during the call). ``V_out`` must be a device buffer."""
    k = C.c_int32(0)
    st = load().imdp_value_iteration_noalloc(C.c_void_p(model.handle), C.byref(spec), _ptr(V_out), C.byref(k),
                                             _stream(stream))
    if k_out is not None:
        k_out[0] = k.value
    if check and st not in (IMDP_OK, IMDP_ENOCONV):
        _check(st, "imdp_value_iteration_noalloc")
    return st


class Server:
    """Owns an ``imdp_server*`` (continuous-batching request server)."""

    def __init__(self, handle: int):
        self.handle = handle
        self._keep = {}  # ticket -> (model, spec) kept alive until the result is taken

    def close(self):
        if self.handle:
            load().imdp_server_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def imdp_server_create(hbm_budget: int) -> Server:
    out = C.c_void_p()
    _check(load().imdp_server_create(int(hbm_budget), C.byref(out)), "imdp_server_create")
    return Server(out.value)


def imdp_server_set_launch(server: Server, kernel: int = 0, cta_warps: int = 0, ctas_per_sm: int = 0,
                           tile_entries: int = 0, wide_col: int = 0):
    """Launch configuration of the server's Bellman launches (0 fields: by rule)."""
    cfg = imdp_launch_config(kernel, cta_warps, ctas_per_sm, tile_entries, wide_col)
    _check(load().imdp_server_set_launch(C.c_void_p(server.handle), C.byref(cfg)), "imdp_server_set_launch")


def imdp_server_stats(server: Server) -> dict:
    """Device time, worker wall time, chunks and mean requests per chunk of a server."""
    d, w, c, r = C.c_double(0), C.c_double(0), C.c_int64(0), C.c_double(0)
    _check(load().imdp_server_stats(C.c_void_p(server.handle), C.byref(d), C.byref(w), C.byref(c), C.byref(r)),
           "imdp_server_stats")
    return dict(device_ms=d.value, wall_ms=w.value, chunks=c.value, mean_requests=r.value)


def imdp_server_submit(server: Server, model: Model, spec) -> int:
    t = C.c_uint64(0)
    _check(load().imdp_server_submit(C.c_void_p(server.handle), C.c_void_p(model.handle), C.byref(spec),
                                     C.byref(t)), "imdp_server_submit")
    server._keep[t.value] = (model, spec)
    return t.value


def imdp_server_poll(server: Server, ticket: int, V_out=None, k_out=None, latency_out=None) -> int:
    """Returns the status: IMDP_EPENDING while the request runs."""
    k = C.c_int32(0)
    lat = C.c_double(0.0)
    st = load().imdp_server_poll(C.c_void_p(server.handle), C.c_uint64(ticket), _ptr(V_out), C.byref(k), C.byref(lat))
    if st != IMDP_EPENDING:
        server._keep.pop(ticket, None)
        if k_out is not None:
            k_out[0] = k.value
        if latency_out is not None:
            latency_out[0] = lat.value
    return st


def imdp_server_wait(server: Server, ticket: int, timeout_ms: float, V_out=None, k_out=None, latency_out=None) -> int:
    k = C.c_int32(0)
    lat = C.c_double(0.0)
    st = load().imdp_server_wait(C.c_void_p(server.handle), C.c_uint64(ticket), float(timeout_ms), _ptr(V_out),
                                 C.byref(k), C.byref(lat))
    if st not in (IMDP_ETIMEOUT,):
        server._keep.pop(ticket, None)
        if k_out is not None:
            k_out[0] = k.value
        if latency_out is not None:
            latency_out[0] = lat.value
    return st


def imdp_server_destroy(server: Server):
    server.close()


# ---------------------------------------------------------------- convenience wrappers (host numpy in/out)

def create_model(m, dtype=IMDP_F64, stream=None, budget=None) -> Model:
    """Model from any object with n_states/stateptr/colptr/rowval/lower/upper.
    ``budget``: per-iteration error budget of 32-bit storage (IMDP_F32 only)."""
    arrs = (np.ascontiguousarray(m.stateptr, np.int32), np.ascontiguousarray(m.colptr, np.int32),
            np.ascontiguousarray(m.rowval, np.int32), np.ascontiguousarray(m.lower, np.float64),
            np.ascontiguousarray(m.upper, np.float64))
    if budget is not None:
        if dtype != IMDP_F32:
            raise ValueError("a budget applies to IMDP_F32 storage only")
        return imdp_create_csc_f32(m.n_states, len(m.colptr) - 1, len(m.rowval), *arrs, budget, stream)
    return imdp_create_csc(m.n_states, len(m.colptr) - 1, len(m.rowval), *arrs, dtype, stream)


def value_iteration(model: Model, n_states: int, policy: bool = False, stream=None, **spec_kw):
    """Returns (status, V, k, residual, policy_or_None) as host numpy arrays."""
    spec = make_spec(**spec_kw)
    V = np.zeros(n_states, np.float64)
    res = np.zeros(n_states, np.float64)
    pol = None
    if policy:
        rows = 1 if spec_kw.get("infinite_time") else int(spec_kw.get("horizon", 100))
        pol = np.zeros((rows, n_states), np.int32)
    k = [0]
    st = imdp_value_iteration(model, spec, V, k, res, pol, stream)
    return STATUS_NAMES[st], V, k[0], res, pol


# ---------------------------------------------------------------- state sharding

def imdp_partition_states(n_states: int, stateptr, colptr, n_parts: int) -> np.ndarray:
    """Contiguous state ranges of about equal work: int32[n_parts + 1] bounds (host-only call)."""
    sp = np.ascontiguousarray(stateptr, dtype=np.int32)
    cp = np.ascontiguousarray(colptr, dtype=np.int32)
    out = np.zeros(int(n_parts) + 1, np.int32)
    _check(load().imdp_partition_states(int(n_states), _ptr(sp), _ptr(cp), int(n_parts), _ptr(out)),
           "imdp_partition_states")
    return out


def imdp_create_csc_slice(n_states: int, s0: int, s1: int, n_cols: int, nnz: int, stateptr, colptr, rowval, lower,
                          upper, dtype=IMDP_F64, stream=None) -> Model:
    out = C.c_void_p()
    st = load().imdp_create_csc_slice(int(n_states), int(s0), int(s1), int(n_cols), int(nnz), _ptr(stateptr),
                                      _ptr(colptr), _ptr(rowval), _ptr(lower), _ptr(upper), int(dtype),
                                      _stream(stream), C.byref(out))
    _check(st, "imdp_create_csc_slice")
    return Model(out.value)


def imdp_session_checkpoint(s: Session, index: int, raw_out=None, stream=None):
    """(raw iterate, k) of problem ``index``; ``raw_out`` may be a host array or a
    CUDA tensor of n_states uint64 words (allocated on the host when None)."""
    if raw_out is None:
        raw_out = np.zeros(s._models[index].info()["n_states"], np.uint64)
    k = C.c_int32(0)
    _check(load().imdp_session_checkpoint(C.c_void_p(s.handle), int(index), _ptr(raw_out), C.byref(k),
                                          _stream(stream)), "imdp_session_checkpoint")
    return raw_out, k.value


def imdp_session_restore(s: Session, index: int, raw, k: int, stream=None):
    """Write a checkpoint (raw iterate, k) into problem ``index``."""
    _check(load().imdp_session_restore(C.c_void_p(s.handle), int(index), _ptr(raw), int(k), _stream(stream)),
           "imdp_session_restore")


def imdp_session_values_get(s: Session, index: int, k: int, s0: int, s1: int, dst, stream=None):
    _check(load().imdp_session_values_get(C.c_void_p(s.handle), int(index), int(k), int(s0), int(s1), _ptr(dst),
                                          _stream(stream)), "imdp_session_values_get")


def imdp_session_values_put(s: Session, index: int, k: int, s0: int, s1: int, src, stream=None):
    _check(load().imdp_session_values_put(C.c_void_p(s.handle), int(index), int(k), int(s0), int(s1), _ptr(src),
                                          _stream(stream)), "imdp_session_values_put")


def slice_arrays(m, s0: int, s1: int):
    """Host CSC arrays of the columns of states [s0, s1) of a model (rowval keeps
    whole-model state indices): (stateptr, colptr, rowval, lower, upper)."""
    c0, c1 = int(m.stateptr[s0]), int(m.stateptr[s1])
    e0, e1 = int(m.colptr[c0]), int(m.colptr[c1])
    return (np.ascontiguousarray(m.stateptr[s0:s1 + 1] - c0, dtype=np.int32),
            np.ascontiguousarray(m.colptr[c0:c1 + 1] - e0, dtype=np.int32),
            np.ascontiguousarray(m.rowval[e0:e1], dtype=np.int32),
            np.ascontiguousarray(m.lower[e0:e1], dtype=np.float64),
            np.ascontiguousarray(m.upper[e0:e1], dtype=np.float64))


def create_model_slice(m, s0: int, s1: int, dtype=IMDP_F64, stream=None) -> Model:
    sp, cp, rv, lo, up = slice_arrays(m, s0, s1)
    return imdp_create_csc_slice(m.n_states, s0, s1, len(cp) - 1, len(rv), sp, cp, rv, lo, up, dtype, stream)


def imdp_model_plan(model: Model):
    """(tiles, wide states, entries in wide states) of a model's launch plan."""
    t, w, e = C.c_int32(0), C.c_int32(0), C.c_int64(0)
    _check(load().imdp_model_plan(C.c_void_p(model.handle), C.byref(t), C.byref(w), C.byref(e)), "imdp_model_plan")
    return t.value, w.value, e.value


def imdp_debug_stall_producer(on: bool):
    """Test hook: step launches leave every consumer wait unsatisfied (see include/imdp.h)."""
    load().imdp_debug_stall_producer(1 if on else 0)


# ---------------------------------------------------------------- model files (Sec. 3.1)

class FileModel:
    """A model read from a file: the CSC arrays ``create_model`` takes, the file's
    action (choice) index of every column (-1 for an added absorbing self-loop),
    and ``spec``: keyword arguments for ``make_spec`` / ``value_iteration``."""

    def __init__(self, n_states, stateptr, colptr, rowval, lower, upper, action, spec):
        self.n_states = n_states
        self.stateptr, self.colptr, self.rowval = stateptr, colptr, rowval
        self.lower, self.upper, self.action = lower, upper, action
        self.spec = spec


def _path(p) -> bytes:
    return os.fsencode(os.fspath(p))


def _take_file(fp) -> FileModel:
    """Copy a library-owned imdp_file into numpy arrays and free it."""
    def arr(ptr, count, dtype):
        return np.ctypeslib.as_array(ptr, shape=(count,)).astype(dtype, copy=True) if count else np.zeros(0, dtype)

    try:
        f = fp.contents
        n, m, nnz = f.n_states, f.n_cols, f.nnz
        sp = f.spec
        spec = dict(property=sp.property, infinite_time=bool(sp.infinite_time), horizon=sp.horizon, eps=sp.eps,
                    pessimistic=bool(sp.pessimistic), maximize=bool(sp.maximize),
                    reach=arr(sp.reach, sp.n_reach, np.int32), avoid=arr(sp.avoid, sp.n_avoid, np.int32))
        return FileModel(n, arr(f.stateptr, n + 1, np.int32), arr(f.colptr, m + 1, np.int32),
                         arr(f.rowval, nnz, np.int32), arr(f.lower, nnz, np.float64), arr(f.upper, nnz, np.float64),
                         arr(f.action, m, np.int32), spec)
    finally:
        load().imdp_file_free(fp)


def imdp_read_bmdp_tool(path) -> FileModel:
    """Read a bmdp-tool file (see include/imdp.h for the layout)."""
    fp = C.POINTER(imdp_file)()
    _check(load().imdp_read_bmdp_tool(_path(path), C.byref(fp)), "imdp_read_bmdp_tool")
    return _take_file(fp)


def imdp_read_prism(path_stem) -> FileModel:
    """Read PRISM explicit files path_stem.{sta,lab,tra,pctl}."""
    fp = C.POINTER(imdp_file)()
    _check(load().imdp_read_prism(_path(path_stem), C.byref(fp)), "imdp_read_prism")
    return _take_file(fp)


def _csc_args(m):
    arrs = [np.ascontiguousarray(m.stateptr, np.int32), np.ascontiguousarray(m.colptr, np.int32),
            np.ascontiguousarray(m.rowval, np.int32), np.ascontiguousarray(m.lower, np.float64),
            np.ascontiguousarray(m.upper, np.float64)]
    return arrs, [a.ctypes.data for a in arrs]


def imdp_write_bmdp_tool(path, m, terminal):
    """Write model ``m`` (CSC arrays) and its terminal states as a bmdp-tool file."""
    arrs, ptrs = _csc_args(m)
    t = np.ascontiguousarray(terminal, np.int32)
    _check(load().imdp_write_bmdp_tool(_path(path), int(m.n_states), len(arrs[1]) - 1, *ptrs,
                                       t.ctypes.data if t.size else None, int(t.size)), "imdp_write_bmdp_tool")


def imdp_write_prism(path_stem, m, **spec_kw):
    """Write model ``m`` and a reachability / reach-avoid query (``make_spec``
    keywords) as PRISM explicit files path_stem.{sta,lab,tra,pctl}."""
    arrs, ptrs = _csc_args(m)
    spec = make_spec(**spec_kw)
    _check(load().imdp_write_prism(_path(path_stem), int(m.n_states), len(arrs[1]) - 1, *ptrs, C.byref(spec)),
           "imdp_write_prism")
