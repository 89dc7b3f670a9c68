"""Thin Python binding of libveloxq (the C ABI in include/veloxq.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Functions keep the C names. Host-pointer entry points take numpy arrays; the
``*_dev`` entry points take CUDA tensors (PyTorch supplies device memory and
the stream; the call is enqueued on ``torch.cuda.current_stream()``).

If the compiled library is missing this module raises ImportError: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libveloxq.so")

VELOXQ_OK, VELOXQ_EINVAL, VELOXQ_ENOMEM, VELOXQ_ECUDA, VELOXQ_ETIMEDOUT, VELOXQ_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
VELOXQ_I8, VELOXQ_I32, VELOXQ_F32, VELOXQ_F64 = 0, 1, 2, 3
VELOXQ_PREC_FP32, VELOXQ_PREC_BF16, VELOXQ_PREC_FP8, VELOXQ_PREC_FP8_ONE_TERM = 0, 1, 2, 3
VELOXQ_PATH_AUTO, VELOXQ_PATH_RESIDENT, VELOXQ_PATH_STREAM, VELOXQ_PATH_DENSE = 0, 1, 2, 3
VELOXQ_METHOD_BSB, VELOXQ_METHOD_ASB, VELOXQ_METHOD_PA = 0, 1, 2

_VT = {np.dtype(np.int8): VELOXQ_I8, np.dtype(np.int32): VELOXQ_I32,
       np.dtype(np.float32): VELOXQ_F32, np.dtype(np.float64): VELOXQ_F64}

EXPORTED = [
    "veloxq_schedule_default", "veloxq_create_dense", "veloxq_create_csr", "veloxq_create_ising_dense",
    "veloxq_create_ising_csr", "veloxq_destroy", "veloxq_last_error", "veloxq_get_info", "veloxq_set_stream",
    "veloxq_solve", "veloxq_solve_batch", "veloxq_energy", "veloxq_energy_dev", "veloxq_init_state_dev",
    "veloxq_field_dev", "veloxq_steps_dev", "veloxq_spectral_radius", "veloxq_grad", "veloxq_last_timing",
    "veloxq_batch_state_dev", "veloxq_energy_dev_noalloc", "veloxq_hubo3_reduce", "veloxq_hubo3_reduce_local",
    "veloxq_selftest_timeout",
]


class Schedule(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_float), ("a0", ctypes.c_float), ("kappa", ctypes.c_float),
                ("c0", ctypes.c_float), ("sigma0", ctypes.c_float), ("n_knots", ctypes.c_int32),
                ("a_knots", ctypes.POINTER(ctypes.c_float)), ("readout_every", ctypes.c_int32),
                ("prec", ctypes.c_int), ("path", ctypes.c_int), ("method", ctypes.c_int),
                ("momentum", ctypes.c_float)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz_field", ctypes.c_int64), ("is_dense", ctypes.c_int32),
                ("is_integer", ctypes.c_int32), ("rho", ctypes.c_double), ("K0", ctypes.c_double),
                ("ising_offset", ctypes.c_double)]


class Timing(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_main", ctypes.c_double), ("launches", ctypes.c_int64),
                ("path", ctypes.c_int32), ("main_launches", ctypes.c_int32),
                ("stream_gather", ctypes.c_int32), ("stream_chunk", ctypes.c_int32),
                ("batch_stages", ctypes.c_int32), ("batch_group", ctypes.c_int32)]


class VeloxqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"veloxq status {status}: {message}")
        self.status = status
        self.message = message


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libveloxq is not built ({LIB_PATH} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    S = ctypes.POINTER(Schedule)
    sig = {
        "veloxq_schedule_default": (None, [S]),
        "veloxq_create_dense": (I, [P, I64, I, P, P, P]),
        "veloxq_create_csr": (I, [P, I64, P, P, I, P, P, P]),
        "veloxq_create_ising_dense": (I, [P, I64, I, P, P, P]),
        "veloxq_create_ising_csr": (I, [P, I64, P, P, I, P, P, P]),
        "veloxq_destroy": (None, [P]),
        "veloxq_last_error": (ctypes.c_char_p, []),
        "veloxq_get_info": (I, [P, ctypes.POINTER(Info)]),
        "veloxq_set_stream": (I, [P, P]),
        "veloxq_solve": (I, [P, I32, I32, S, U64, P, P, P, P]),
        "veloxq_solve_batch": (I, [P, I32, I32, I32, S, U64, P, P]),
        "veloxq_energy": (I, [P, I64, P, P, P]),
        "veloxq_energy_dev": (I, [P, I64, P, P, P]),
        "veloxq_init_state_dev": (I, [P, I32, U64, ctypes.c_float, P, P]),
        "veloxq_field_dev": (I, [P, I32, I, P, P]),
        "veloxq_steps_dev": (I, [P, I32, I32, I32, I32, S, P, P, P]),
        "veloxq_spectral_radius": (I, [P, ctypes.POINTER(D)]),
        "veloxq_grad": (I, [P, I32, I32, S, U64, I32, P, P, P, P]),
        "veloxq_last_timing": (I, [P, ctypes.POINTER(Timing)]),
        "veloxq_batch_state_dev": (I, [P, I32, P, P]),
        "veloxq_energy_dev_noalloc": (I, [P, I64, P, P, P]),
        "veloxq_hubo3_reduce": (I, [I64, P, I64, P, P, P, I64, P, P, P, P, P, P, P, P, P, P, P]),
        "veloxq_hubo3_reduce_local": (I, [I64, P, I64, P, P, P, I64, P, P, P, P, P, P, P, P, P, P, P, P]),
        "veloxq_selftest_timeout": (I, [I64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(status: int):
    if status != VELOXQ_OK:
        raise VeloxqError(status, _lib.veloxq_last_error().decode(errors="replace"))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(a.data_ptr())   # torch tensor


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype_name: str, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("device entry points take CUDA tensors")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError(f"expected a {dtype_name} tensor, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owner of a veloxq_ctx*; destroyed with the object (or by destroy())."""

    def __init__(self, handle: ctypes.c_void_p, keep=None):
        self.handle = handle
        self._keep = keep

    def destroy(self):
        if self.handle:
            _lib.veloxq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @property
    def info(self) -> Info:
        return veloxq_get_info(self)


def veloxq_schedule_default() -> Schedule:
    s = Schedule()
    _lib.veloxq_schedule_default(ctypes.byref(s))
    return s


def make_schedule(**kw) -> Schedule:
    """A Schedule with the library defaults, overridden by keyword (knots=list)."""
    s = veloxq_schedule_default()
    knots = kw.pop("knots", None)
    for k, v in kw.items():
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    if knots is not None:
        arr = (ctypes.c_float * len(knots))(*[float(v) for v in knots])
        s.n_knots = len(knots)
        s.a_knots = ctypes.cast(arr, ctypes.POINTER(ctypes.c_float))
        s._knots_keepalive = arr
    return s


def _vt(a: np.ndarray) -> int:
    if a.dtype not in _VT:
        raise TypeError(f"unsupported value dtype {a.dtype} (int8, int32, float32, float64)")
    return _VT[a.dtype]


def veloxq_create_dense(Q: np.ndarray, c: Optional[np.ndarray] = None, stream=None) -> Context:
    Q = np.ascontiguousarray(Q)
    if Q.ndim != 2 or Q.shape[0] != Q.shape[1]:
        raise ValueError("Q must be square")
    cc = None if c is None else _host(c, np.float64)
    h = ctypes.c_void_p()
    _check(_lib.veloxq_create_dense(ctypes.byref(h), Q.shape[0], _vt(Q), _ptr(Q), _ptr(cc), stream))
    return Context(h)


def veloxq_create_ising_dense(J: np.ndarray, h: Optional[np.ndarray] = None, stream=None) -> Context:
    J = np.ascontiguousarray(J)
    if J.ndim != 2 or J.shape[0] != J.shape[1]:
        raise ValueError("J must be square")
    hh = None if h is None else _host(h, np.float64)
    out = ctypes.c_void_p()
    _check(_lib.veloxq_create_ising_dense(ctypes.byref(out), J.shape[0], _vt(J), _ptr(J), _ptr(hh), stream))
    return Context(out)


def veloxq_create_csr(n: int, rowptr, col, val, c=None, stream=None) -> Context:
    rp = _host(rowptr, np.int64)
    cl = _host(col, np.int32)
    vl = np.ascontiguousarray(val)
    if rp.shape[0] != n + 1:
        raise ValueError("rowptr must hold n + 1 entries")
    cc = None if c is None else _host(c, np.float64)
    h = ctypes.c_void_p()
    _check(_lib.veloxq_create_csr(ctypes.byref(h), n, _ptr(rp), _ptr(cl), _vt(vl), _ptr(vl), _ptr(cc), stream))
    return Context(h)


def veloxq_create_ising_csr(n: int, rowptr, col, J, h=None, stream=None) -> Context:
    rp = _host(rowptr, np.int64)
    cl = _host(col, np.int32)
    jv = np.ascontiguousarray(J)
    if rp.shape[0] != n + 1:
        raise ValueError("rowptr must hold n + 1 entries")
    hh = None if h is None else _host(h, np.float64)
    out = ctypes.c_void_p()
    _check(_lib.veloxq_create_ising_csr(ctypes.byref(out), n, _ptr(rp), _ptr(cl), _vt(jv), _ptr(jv), _ptr(hh), stream))
    return Context(out)


def veloxq_hubo3_reduce(n: int, h=None, pairs=None, triples=None, local: bool = False) -> dict:
    """Third-order Ising cost function -> second order (one auxiliary spin
    per cubic term). pairs = (pi, pj, J), triples = (ti, tj, tk, K). Returns
    n (with the auxiliary spins), rowptr, col, val, lin and offset of the
    reduced Ising instance, ready for veloxq_create_ising_csr. local=True
    numbers the spins for locality (veloxq_hubo3_reduce_local) and adds
    "index", the reduced index of every original and auxiliary spin."""
    empty_i, empty_f = np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.float64)
    pi, pj, J2 = (empty_i, empty_i, empty_f) if pairs is None else pairs
    ti, tj, tk, K3 = (empty_i, empty_i, empty_i, empty_f) if triples is None else triples
    pi, pj, ti, tj, tk = (_host(a, np.int64) for a in (pi, pj, ti, tj, tk))
    J2, K3 = _host(J2, np.float64), _host(K3, np.float64)
    hh = None if h is None else _host(h, np.float64)
    n2, n3 = pi.shape[0], ti.shape[0]
    N = n + n3
    cap = max(1, 2 * (n2 + 6 * n3))
    rowptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(cap, dtype=np.int32)
    val = np.zeros(cap, dtype=np.float64)
    lin = np.zeros(N, dtype=np.float64)
    n_out, nnz_out, off = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    args = (n, _ptr(hh), n2, _ptr(pi), _ptr(pj), _ptr(J2), n3, _ptr(ti), _ptr(tj), _ptr(tk), _ptr(K3),
            ctypes.byref(n_out), ctypes.byref(nnz_out), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(lin),
            ctypes.byref(off))
    index = np.zeros(N, dtype=np.int64) if local else None
    if local:
        _check(_lib.veloxq_hubo3_reduce_local(*args, _ptr(index)))
    else:
        _check(_lib.veloxq_hubo3_reduce(*args))
    m = nnz_out.value
    out = {"n": n_out.value, "rowptr": rowptr, "col": col[:m].copy(), "val": val[:m].copy(), "lin": lin,
           "offset": off.value}
    if local:
        out["index"] = index
    return out


def veloxq_selftest_timeout(budget_cycles: int) -> None:
    """Run the bounded-wait self-test (raises VeloxqError: ETIMEDOUT is the
    expected outcome)."""
    _check(_lib.veloxq_selftest_timeout(int(budget_cycles)))


def veloxq_destroy(ctx: Context):
    ctx.destroy()


def veloxq_last_error() -> str:
    return _lib.veloxq_last_error().decode(errors="replace")


def veloxq_get_info(ctx: Context) -> Info:
    info = Info()
    _check(_lib.veloxq_get_info(ctx.handle, ctypes.byref(info)))
    return info


def veloxq_set_stream(ctx: Context, stream) -> None:
    _check(_lib.veloxq_set_stream(ctx.handle, stream))


def veloxq_last_timing(ctx: Context) -> Timing:
    t = Timing()
    _check(_lib.veloxq_last_timing(ctx.handle, ctypes.byref(t)))
    return t


def veloxq_spectral_radius(ctx: Context) -> float:
    r = ctypes.c_double()
    _check(_lib.veloxq_spectral_radius(ctx.handle, ctypes.byref(r)))
    return r.value


def veloxq_solve(ctx: Context, replicas: int, steps: int, sched: Optional[Schedule] = None, seed: int = 0,
                 want_x: bool = True, want_per_replica: bool = True) -> dict:
    """Returns dict(x, E, E_int (integer contexts), E_per_replica)."""
    n = ctx.info.n
    integer = bool(ctx.info.is_integer)
    x = np.zeros(n, dtype=np.uint8) if want_x else None
    E = ctypes.c_double()
    Ei = ctypes.c_int64()
    per = np.zeros(replicas, dtype=np.float64) if want_per_replica else None
    _check(_lib.veloxq_solve(ctx.handle, replicas, steps, ctypes.byref(sched) if sched is not None else None,
                             ctypes.c_uint64(seed), _ptr(x), ctypes.byref(E), ctypes.byref(Ei) if integer else None,
                             _ptr(per)))
    return {"x": x, "E": E.value, "E_int": Ei.value if integer else None, "E_per_replica": per}


def veloxq_solve_batch(ctxs: Sequence[Context], replicas: int, steps: int, sched: Optional[Schedule] = None,
                       seed: int = 0, want_x: bool = True) -> dict:
    m = len(ctxs)
    handles = (ctypes.c_void_p * m)(*[c.handle for c in ctxs])
    xs = [np.zeros(c.info.n, dtype=np.uint8) for c in ctxs] if want_x else None
    xp = (ctypes.c_void_p * m)(*[x.ctypes.data for x in xs]) if want_x else None
    E = np.zeros(m, dtype=np.float64)
    _check(_lib.veloxq_solve_batch(handles, m, replicas, steps, ctypes.byref(sched) if sched is not None else None,
                                   ctypes.c_uint64(seed), xp, _ptr(E)))
    return {"x": xs, "E": E}


def veloxq_energy(ctx: Context, X: np.ndarray) -> dict:
    X = _host(np.atleast_2d(X), np.uint8)
    B = X.shape[0]
    if X.shape[1] != ctx.info.n:
        raise ValueError("X must be [batch][n]")
    E = np.zeros(B, dtype=np.float64)
    integer = bool(ctx.info.is_integer)
    Ei = np.zeros(B, dtype=np.int64) if integer else None
    _check(_lib.veloxq_energy(ctx.handle, B, _ptr(X), _ptr(E), _ptr(Ei)))
    return {"E": E, "E_int": Ei}


def veloxq_energy_dev(ctx: Context, X, E, E_int=None) -> None:
    B = X.shape[0]
    veloxq_set_stream(ctx, _stream_ptr())
    _check(_lib.veloxq_energy_dev(ctx.handle, B, _dev(X, "uint8", (B, ctx.info.n)), _dev(E, "float64", (B,)),
                                  _dev(E_int, "int64", (B,)) if E_int is not None else None))


def veloxq_batch_state_dev(ctx: Context, R: int, S, Y) -> None:
    n = ctx.info.n
    veloxq_set_stream(ctx, _stream_ptr())
    _check(_lib.veloxq_batch_state_dev(ctx.handle, R, _dev(S, "float32", (R, n)), _dev(Y, "float32", (R, n))))


def veloxq_energy_dev_noalloc(ctx: Context, X, E, E_int=None) -> None:
    """veloxq_energy_dev without any device allocation (fixed scratch; see the header)."""
    B_ = X.shape[0]
    veloxq_set_stream(ctx, _stream_ptr())
    _check(_lib.veloxq_energy_dev_noalloc(ctx.handle, B_, _dev(X, "uint8", (B_, ctx.info.n)), _dev(E, "float64", (B_,)),
                                          _dev(E_int, "int64", (B_,)) if E_int is not None else None))


def veloxq_init_state_dev(ctx: Context, R: int, seed: int, sigma0: float, S, Y) -> None:
    n = ctx.info.n
    veloxq_set_stream(ctx, _stream_ptr())
    _check(_lib.veloxq_init_state_dev(ctx.handle, R, ctypes.c_uint64(seed), ctypes.c_float(sigma0),
                                      _dev(S, "float32", (R, n)), _dev(Y, "float32", (R, n))))


def veloxq_field_dev(ctx: Context, R: int, prec: int, S, F) -> None:
    n = ctx.info.n
    veloxq_set_stream(ctx, _stream_ptr())
    _check(_lib.veloxq_field_dev(ctx.handle, R, prec, _dev(S, "float32", (R, n)), _dev(F, "float32", (R, n))))


def veloxq_steps_dev(ctx: Context, R: int, k_begin: int, k_count: int, K: int, sched: Optional[Schedule],
                     S, Y, F_last=None) -> None:
    n = ctx.info.n
    veloxq_set_stream(ctx, _stream_ptr())
    _check(_lib.veloxq_steps_dev(ctx.handle, R, k_begin, k_count, K,
                                 ctypes.byref(sched) if sched is not None else None,
                                 _dev(S, "float32", (R, n)), _dev(Y, "float32", (R, n)),
                                 _dev(F_last, "float32", (R, n)) if F_last is not None else None))


def veloxq_grad(ctx: Context, replicas: int, steps: int, sched: Optional[Schedule] = None, seed: int = 0,
                ckpt_every: int = 20) -> dict:
    nk = sched.n_knots if (sched is not None and sched.n_knots > 0) else 2
    loss, d_dt, d_kappa = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    d_knots = np.zeros(nk, dtype=np.float64)
    _check(_lib.veloxq_grad(ctx.handle, replicas, steps, ctypes.byref(sched) if sched is not None else None,
                            ctypes.c_uint64(seed), ckpt_every, ctypes.byref(loss), ctypes.byref(d_dt),
                            ctypes.byref(d_kappa), _ptr(d_knots)))
    return {"loss": loss.value, "d_dt": d_dt.value, "d_kappa": d_kappa.value, "d_knots": d_knots}
