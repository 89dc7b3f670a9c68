"""FP64 oracle of the VeloxQ hot path (arXiv:2501.19221) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package. The CUDA library never calls it and it
shares no code with the library: ``oracle.c`` is compiled on its own with gcc.

Every function below is either a ctypes call into ``oracle.c`` (plain loops in
FP64, each citing the passage it follows) or a numpy/scipy library routine used
as one step (a dense eigen-solver for the spectral radius of App. B's
c0 = 1/lambda_max). The arithmetic each function performs is stated in its
docstring with the paper passage it restates.

Pins (``tests/test_oracle_pins.py``): exhaustive enumeration, the single-flip
energy identity, App. A conversions against brute force, the Wishart planted
energy, published Philox4x32-10 test vectors, closed-form uncoupled dynamics,
Z2 equivariance, replica permutation, finite differences of the gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, u64, f64, f32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_float
        sig = {
            "oracle_philox4x32_10": (None, [P, P, P]),
            "oracle_init_state": (None, [i64, i32, u64, f32, P, P]),
            "oracle_energy_batch_i64": (None, [i64, i64, P, P, P, P, i64, P, P]),
            "oracle_energy_batch_f64": (None, [i64, i64, P, P, P, P, i64, P, P]),
            "oracle_bruteforce_i64": (i64, [i64, i64, P, P, P, P, P, P]),
            "oracle_bruteforce_f64": (f64, [i64, i64, P, P, P, P, P]),
            "oracle_ising_energy": (f64, [i64, P, P, P]),
            "oracle_ising_to_qubo": (None, [i64, P, P, P, P]),
            "oracle_qubo_to_ising": (None, [i64, P, P, P, P]),
            "oracle_bias": (None, [i64, i64, P, P, P, P, P, P]),
            "oracle_field": (None, [i64, i64, P, P, P, i32, P, P]),
            "oracle_schedule": (None, [i32, i32, P, P]),
            "oracle_bsb_update": (None, [i64, i32, P, P, f64, f64, f64, f64, P, P]),
            "oracle_update": (None, [i32, i64, i32, P, P, f64, f64, f64, f64, f64, P, P]),
            "oracle_field_operand": (None, [i32, i64, P, P]),
            "oracle_run": (ctypes.c_int, [i32, f64, i64, i64, P, P, P, P, P, P, i32, i32, f64, f64, f64,
                                          i32, P, i32, P, P, i32, P, P, P, P, P, P, P, P, P]),
            "oracle_bsb_run": (ctypes.c_int, [i64, i64, P, P, P, P, P, P, i32, i32, f64, f64, f64,
                                              i32, P, i32, P, P, i32, P, P, P, P, P, P, P, P, P]),
            "oracle_relaxed_energy": (None, [i64, i64, P, P, P, P, i32, P, P]),
            "oracle_bsb_grad": (ctypes.c_int, [i64, i64, P, P, P, P, i32, i32, f64, f64, f64,
                                               i32, P, P, P, P, P, P, P]),
            "oracle_bsb_loss": (ctypes.c_int, [i64, i64, P, P, P, P, i32, i32, f64, f64, f64,
                                               i32, P, P, P, P]),
            "oracle_ising_pairs_to_qubo": (None, [i64, i64, P, P, P, P, P, P, P, P]),
            "oracle_hubo3_energy": (f64, [i64, P, i64, P, P, P, i64, P, P, P, P, P]),
            "oracle_hubo3_reduce": (None, [i64, P, i64, P, P, P, i64, P, P, P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Problem container: every stored entry of Q as a coordinate list
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    """A QUBO  E(x) = sum_{i,j} Q_ij x_i x_j + sum_i c_i x_i  (Sec. 2, eq.
    qubo_model, read as a sum over every stored entry) as coordinate lists.

    ``ev_i64``/``c_i64`` are present when Q and c are integer-valued, and then
    energies are exact int64.
    """

    n: int
    er: np.ndarray
    ec: np.ndarray
    ev: np.ndarray
    c: np.ndarray
    ev_i64: Optional[np.ndarray] = None
    c_i64: Optional[np.ndarray] = None

    @property
    def nnz(self) -> int:
        return int(self.er.shape[0])

    @property
    def integer(self) -> bool:
        return self.ev_i64 is not None

    def dense(self) -> np.ndarray:
        Q = np.zeros((self.n, self.n))
        np.add.at(Q, (self.er, self.ec), self.ev)
        return Q


def _finish(n, er, ec, vals, c) -> Problem:
    c = np.zeros(n) if c is None else np.asarray(c, dtype=np.float64)
    integer = np.issubdtype(vals.dtype, np.integer) and np.all(c == np.round(c))
    ev = vals.astype(np.float64)
    p = Problem(n, np.ascontiguousarray(er, dtype=np.int64), np.ascontiguousarray(ec, dtype=np.int64),
                np.ascontiguousarray(ev), np.ascontiguousarray(c))
    if integer:
        p.ev_i64 = np.ascontiguousarray(vals.astype(np.int64))
        p.c_i64 = np.ascontiguousarray(c.astype(np.int64))
    return p


def problem_from_dense(Q: np.ndarray, c=None) -> Problem:
    """Every entry of a dense Q (zeros included) becomes one coordinate."""
    Q = np.asarray(Q)
    n = Q.shape[0]
    er, ec = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return _finish(n, er.ravel(), ec.ravel(), Q.ravel(), c)


def problem_from_csr(n, rowptr, col, val, c=None) -> Problem:
    rowptr = np.asarray(rowptr, dtype=np.int64)
    er = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    return _finish(n, er, np.asarray(col, dtype=np.int64), np.asarray(val), c)


# ---------------------------------------------------------------------------
# Random numbers
# ---------------------------------------------------------------------------
def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def init_state(n: int, R: int, seed: int, sigma0: float):
    """Initial (s0, y0) ~ U(-sigma0, sigma0) as exact float32 [R][n] arrays."""
    lib = _load()
    S0 = np.zeros((R, n), dtype=np.float32)
    Y0 = np.zeros((R, n), dtype=np.float32)
    lib.oracle_init_state(n, R, ctypes.c_uint64(seed), ctypes.c_float(sigma0), _p(S0), _p(Y0))
    return S0, Y0


# ---------------------------------------------------------------------------
# Energies and exhaustive search
# ---------------------------------------------------------------------------
def energy(p: Problem, X: np.ndarray) -> np.ndarray:
    """E(x) for a batch X [B][n] of binary vectors (int64 if Q is integer)."""
    lib = _load()
    X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.uint8)
    B = X.shape[0]
    if p.integer:
        E = np.zeros(B, dtype=np.int64)
        lib.oracle_energy_batch_i64(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev_i64), _p(p.c_i64), B, _p(X), _p(E))
    else:
        E = np.zeros(B, dtype=np.float64)
        lib.oracle_energy_batch_f64(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), _p(p.c), B, _p(X), _p(E))
    return E


def bruteforce(p: Problem):
    """(E_min, x_min, count_min) over all 2^n assignments (n <= 26)."""
    if p.n > 26:
        raise ValueError("exhaustive search is limited to n <= 26")
    lib = _load()
    arg = ctypes.c_uint64(0)
    if p.integer:
        cnt = ctypes.c_int64(0)
        E = lib.oracle_bruteforce_i64(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev_i64), _p(p.c_i64),
                                      ctypes.byref(arg), ctypes.byref(cnt))
        count = cnt.value
    else:
        E = lib.oracle_bruteforce_f64(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), _p(p.c), ctypes.byref(arg))
        count = None
    x = np.array([(arg.value >> i) & 1 for i in range(p.n)], dtype=np.uint8)
    return E, x, count


def ising_energy(J: np.ndarray, h: np.ndarray, s: np.ndarray) -> float:
    """H(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i (Sec. 2, eq. ising_model)."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return lib.oracle_ising_energy(J.shape[0], _p(J), _p(h), _p(s))


def hubo3_energy(n: int, h, pairs, triples, S: np.ndarray) -> np.ndarray:
    """H(s) = sum h s + sum J s s + sum K s s s per row of S (spins +-1), the
    third-order cost function of Sec. "HUBO" (eqs. nn, mw3s). pairs = (pi, pj,
    J), triples = (ti, tj, tk, K); either may be None."""
    lib = _load()
    z_i, z_f = np.zeros(0, dtype=np.int64), np.zeros(0)
    pi, pj, J2 = (z_i, z_i, z_f) if pairs is None else pairs
    ti, tj, tk, K3 = (z_i, z_i, z_i, z_f) if triples is None else triples
    pi, pj, ti, tj, tk = (np.ascontiguousarray(a, dtype=np.int64) for a in (pi, pj, ti, tj, tk))
    J2 = np.ascontiguousarray(J2, dtype=np.float64)
    K3 = np.ascontiguousarray(K3, dtype=np.float64)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.int8)
    return np.array([lib.oracle_hubo3_energy(n, _p(hh), pi.shape[0], _p(pi), _p(pj), _p(J2), ti.shape[0], _p(ti),
                                             _p(tj), _p(tk), _p(K3), _p(np.ascontiguousarray(s))) for s in S])


def hubo3_reduce(n: int, h, pairs, triples):
    """Second-order form of a third-order cost function (Sec. "HUBO", eq.
    reduction): one auxiliary spin per cubic term. Returns (n + n3, (pi, pj,
    J) unmerged pairs, lin, offset)."""
    lib = _load()
    z_i, z_f = np.zeros(0, dtype=np.int64), np.zeros(0)
    pi, pj, J2 = (z_i, z_i, z_f) if pairs is None else pairs
    ti, tj, tk, K3 = (z_i, z_i, z_i, z_f) if triples is None else triples
    pi, pj, ti, tj, tk = (np.ascontiguousarray(a, dtype=np.int64) for a in (pi, pj, ti, tj, tk))
    J2 = np.ascontiguousarray(J2, dtype=np.float64)
    K3 = np.ascontiguousarray(K3, dtype=np.float64)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    n2, n3 = pi.shape[0], ti.shape[0]
    m = n2 + 6 * n3
    qi, qj, qv = np.zeros(m, dtype=np.int64), np.zeros(m, dtype=np.int64), np.zeros(m)
    lin = np.zeros(n + n3)
    off = ctypes.c_double()
    lib.oracle_hubo3_reduce(n, _p(hh), n2, _p(pi), _p(pj), _p(J2), n3, _p(ti), _p(tj), _p(tk), _p(K3),
                            _p(qi), _p(qj), _p(qv), _p(lin), ctypes.byref(off))
    return n + n3, (qi, qj, qv), lin, off.value


def ising_to_qubo(J: np.ndarray, h: np.ndarray):
    """App. A Ising -> QUBO: returns (Q, C) with H(s) = 2 Q(x) + C."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    n = J.shape[0]
    Q = np.zeros((n, n))
    C = ctypes.c_double(0.0)
    lib.oracle_ising_to_qubo(n, _p(J), _p(h), _p(Q), ctypes.byref(C))
    return Q, C.value


def ising_csr_to_qubo(n, rowptr, col, J, h=None):
    """App. A Ising -> QUBO for a sparse Ising model given in CSR; the pair
    (i < j) takes the value stored at its upper-triangle position. Returns
    (Problem, C) with H(s) = 2 E(x) + C. Integer J and h give an integer Problem."""
    lib = _load()
    rowptr = np.asarray(rowptr, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    col = np.asarray(col, dtype=np.int64)
    upper = col > rows                      # select the (i < j) entries: no arithmetic
    pi = np.ascontiguousarray(rows[upper])
    pj = np.ascontiguousarray(col[upper])
    Jv = np.asarray(J)
    pv = np.ascontiguousarray(Jv[upper], dtype=np.float64)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    m = pi.shape[0]
    er = np.zeros(2 * m + n, dtype=np.int64)
    ec = np.zeros(2 * m + n, dtype=np.int64)
    ev = np.zeros(2 * m + n, dtype=np.float64)
    C = ctypes.c_double(0.0)
    lib.oracle_ising_pairs_to_qubo(n, m, _p(pi), _p(pj), _p(pv), _p(hh), _p(er), _p(ec), _p(ev), ctypes.byref(C))
    integer = np.issubdtype(Jv.dtype, np.integer) and (hh is None or np.all(hh == np.round(hh)))
    p = Problem(n, er, ec, ev, np.zeros(n))
    if integer:
        p.ev_i64 = np.ascontiguousarray(np.round(ev).astype(np.int64))
        p.c_i64 = np.zeros(n, dtype=np.int64)
    return p, C.value


def ising_pairs_to_qubo(n, pi, pj, pv, h=None):
    """App. A Ising -> QUBO from a list of coupled pairs (i < j, J_ij): returns
    (Problem, C) with H(s) = 2 E(x) + C. A subset of pairs gives the exact
    off-diagonal entries of those pairs (for sampled rows of huge instances);
    the diagonal is then that of the subset."""
    lib = _load()
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    pj = np.ascontiguousarray(pj, dtype=np.int64)
    pv = np.ascontiguousarray(pv, dtype=np.float64)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    m = pi.shape[0]
    er = np.zeros(2 * m + n, dtype=np.int64)
    ec = np.zeros(2 * m + n, dtype=np.int64)
    ev = np.zeros(2 * m + n, dtype=np.float64)
    C = ctypes.c_double(0.0)
    lib.oracle_ising_pairs_to_qubo(n, m, _p(pi), _p(pj), _p(pv), _p(hh), _p(er), _p(ec), _p(ev), ctypes.byref(C))
    return Problem(n, er, ec, ev, np.zeros(n)), C.value


def qubo_to_ising(Q: np.ndarray):
    """App. A QUBO -> Ising for symmetric Q: (J, h, C) with Q(x) = H(s)/2 + C/2."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = Q.shape[0]
    J = np.zeros((n, n))
    h = np.zeros(n)
    C = ctypes.c_double(0.0)
    lib.oracle_qubo_to_ising(n, _p(Q), _p(J), _p(h), ctypes.byref(C))
    return J, h, C.value


# ---------------------------------------------------------------------------
# Normalisation, field, schedule, update
# ---------------------------------------------------------------------------
def bias(p: Problem):
    """(b, K0) with b = Qs 1 + c and K0 such that E = s^T Qoff s/4 + b^T s/2 + K0."""
    lib = _load()
    b = np.zeros(p.n)
    K0 = ctypes.c_double(0.0)
    lib.oracle_bias(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), _p(p.c), _p(b), ctypes.byref(K0))
    return b, K0.value


def field(p: Problem, S: np.ndarray) -> np.ndarray:
    """F = Qoff S for S [R][n] (Qoff = off-diagonal part of (Q + Q^T)/2)."""
    lib = _load()
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64)
    F = np.zeros_like(S)
    lib.oracle_field(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), S.shape[0], _p(S), _p(F))
    return F


def field_dense_rows(Q: np.ndarray, S: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """F[:, rows] = Qoff[rows, :] S^T for a dense Q given as is (Qoff = the
    off-diagonal part of (Q + Q^T)/2), in FP64 with a library matmul as the
    product; for sampled rows of large instances. Returns [R][len(rows)]."""
    Q = np.asarray(Q)
    rows = np.asarray(rows)
    Qs = 0.5 * (Q[rows, :].astype(np.float64) + Q[:, rows].T.astype(np.float64))
    Qs[np.arange(rows.shape[0]), rows] = 0.0
    return np.asarray(S, dtype=np.float64) @ Qs.T


def bias_dense_rows(Q: np.ndarray, c, rows: np.ndarray) -> np.ndarray:
    """b[rows] with b = Qs 1 + c, Qs = (Q + Q^T)/2 (the linear term of the
    spin form under x = (1 + s)/2, Sec. 2 eq. qubo_model), for a dense Q given
    as is, summed in FP64 by a library routine; for sampled rows of large
    instances."""
    Q = np.asarray(Q)
    rows = np.asarray(rows)
    Qs = 0.5 * (Q[rows, :].astype(np.float64) + Q[:, rows].T.astype(np.float64))
    b = Qs.sum(axis=1)
    if c is not None:
        b = b + np.asarray(c, dtype=np.float64)[rows]
    return b


def abs_field_dense_rows(Q: np.ndarray, S: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """|Qoff|[rows, :] |S|^T, the scale of the rounding bound for field_dense_rows."""
    Q = np.asarray(Q)
    rows = np.asarray(rows)
    Qs = 0.5 * np.abs(Q[rows, :].astype(np.float64) + Q[:, rows].T.astype(np.float64))
    Qs[np.arange(rows.shape[0]), rows] = 0.0
    return np.abs(np.asarray(S, dtype=np.float64)) @ Qs.T


def abs_field(p: Problem, S: np.ndarray) -> np.ndarray:
    """|Qoff| |S|: the scale of the rounding error bound of F (same loop on |.|)."""
    q = Problem(p.n, p.er, p.ec, np.abs(p.ev), p.c)
    return field(q, np.abs(S))


def schedule(K: int, knots: Sequence[float]) -> np.ndarray:
    """a_k, k = 0..K-1, piecewise linear through evenly spread knots (App. B a(t))."""
    lib = _load()
    kn = np.ascontiguousarray(knots, dtype=np.float64)
    a = np.zeros(max(K, 1))
    lib.oracle_schedule(K, kn.shape[0], _p(kn), _p(a))
    return a[:K]


def bsb_update(F, b, a_k, dt, a0, c0, S, Y):
    """One ballistic-SB update given the field F (in place on float64 copies)."""
    lib = _load()
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64).copy()
    Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64).copy()
    F = np.ascontiguousarray(F, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    R, n = S.shape
    lib.oracle_bsb_update(n, R, _p(F), _p(b), a_k, dt, a0, c0, _p(S), _p(Y))
    return S, Y


def bsb_step(p: Problem, S, Y, a_k, dt, a0, c0):
    """Field then update: one full step (App. B, ballistic form). Returns (S, Y, F)."""
    b, _ = bias(p)
    F = field(p, S)
    S1, Y1 = bsb_update(F, b, a_k, dt, a0, c0, S, Y)
    return S1, Y1, F


METHODS = {"bsb": 0, "asb": 1, "pa": 2}


def field_operand(method: str, S) -> np.ndarray:
    """The state the field multiplies: S itself (SB forms) or the binarised
    spins, +1 where x > 0 and -1 elsewhere (PA)."""
    lib = _load()
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64)
    out = np.zeros_like(S)
    lib.oracle_field_operand(METHODS[method], S.size, _p(S), _p(out))
    return out


def update(method: str, F, b, a_k, dt, a0, c0, S, Y, alpha: float = 0.9):
    """One update of `method` ("bsb", "asb" or "pa") given the field F of the
    method's operand (returns new float64 copies)."""
    lib = _load()
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64).copy()
    Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64).copy()
    F = np.ascontiguousarray(F, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    R, n = S.shape
    lib.oracle_update(METHODS[method], n, R, _p(F), _p(b), a_k, dt, a0, c0, alpha, _p(S), _p(Y))
    return S, Y


def step(method: str, p: Problem, S, Y, a_k, dt, a0, c0, alpha: float = 0.9):
    """Field of the method's operand, then the update. Returns (S, Y, F)."""
    b, _ = bias(p)
    F = field(p, field_operand(method, S))
    S1, Y1 = update(method, F, b, a_k, dt, a0, c0, S, Y, alpha)
    return S1, Y1, F


def bsb_run(p: Problem, R: int, K: int, dt: float, a0: float, c0: float,
            knots: Sequence[float], readout_every: int, S0: np.ndarray, Y0: np.ndarray,
            n_snap: int = 0, method: str = "bsb", alpha: float = 0.9) -> dict:
    """K steps of `method` (ballistic SB by default; "asb" adiabatic SB, "pa"
    Parallel Annealing with momentum alpha) with readouts, exact energies and
    best-so-far.

    Returns per-replica best energies/vectors/steps, the final state, and the
    first ``n_snap`` fields and states if asked for.
    """
    lib = _load()
    n = p.n
    kn = np.ascontiguousarray(knots, dtype=np.float64)
    S0 = np.ascontiguousarray(S0, dtype=np.float32)
    Y0 = np.ascontiguousarray(Y0, dtype=np.float32)
    F_snap = np.zeros((n_snap, R, n)) if n_snap else None
    S_snap = np.zeros((n_snap, R, n)) if n_snap else None
    Y_snap = np.zeros((n_snap, R, n)) if n_snap else None
    S_fin = np.zeros((R, n))
    Y_fin = np.zeros((R, n))
    best_E = np.zeros(R)
    best_E_i64 = np.zeros(R, dtype=np.int64) if p.integer else None
    best_x = np.zeros((R, n), dtype=np.uint8)
    best_step = np.zeros(R, dtype=np.int32)
    rc = lib.oracle_run(METHODS[method], alpha, n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), _p(p.c),
                        _p(p.ev_i64), _p(p.c_i64), R, K, dt, a0, c0, kn.shape[0], _p(kn), readout_every,
                        _p(S0), _p(Y0), n_snap, _p(F_snap), _p(S_snap), _p(Y_snap), _p(S_fin), _p(Y_fin),
                        _p(best_E), _p(best_E_i64), _p(best_x), _p(best_step))
    if rc != 0:
        raise MemoryError("oracle_bsb_run failed to allocate")
    r_best = int(np.argmin(best_E_i64 if p.integer else best_E))   # lowest replica index on ties
    return {
        "best_E": best_E, "best_E_i64": best_E_i64, "best_x": best_x, "best_step": best_step,
        "S": S_fin, "Y": Y_fin, "F_snap": F_snap, "S_snap": S_snap, "Y_snap": Y_snap,
        "argmin": r_best, "E_min": (best_E_i64 if p.integer else best_E)[r_best],
    }


def relaxed_energy(p: Problem, S: np.ndarray) -> np.ndarray:
    """E_relax(s) = s^T Qoff s/4 + b^T s/2 + K0 per replica (continuous s)."""
    lib = _load()
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64)
    E = np.zeros(S.shape[0])
    lib.oracle_relaxed_energy(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), _p(p.c), S.shape[0], _p(S), _p(E))
    return E


def bsb_grad(p: Problem, R, K, dt, a0, c0, knots, S0, Y0) -> dict:
    """Reverse-mode gradient of L = mean_r E_relax(s_K) w.r.t. dt, c0, knots."""
    lib = _load()
    kn = np.ascontiguousarray(knots, dtype=np.float64)
    S0 = np.ascontiguousarray(S0, dtype=np.float32)
    Y0 = np.ascontiguousarray(Y0, dtype=np.float32)
    loss, d_dt, d_c0 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    d_kn = np.zeros(kn.shape[0])
    rc = lib.oracle_bsb_grad(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), _p(p.c), R, K, dt, a0, c0,
                             kn.shape[0], _p(kn), _p(S0), _p(Y0), ctypes.byref(loss), ctypes.byref(d_dt),
                             ctypes.byref(d_c0), _p(d_kn))
    if rc != 0:
        raise MemoryError("oracle_bsb_grad failed to allocate")
    return {"loss": loss.value, "d_dt": d_dt.value, "d_c0": d_c0.value, "d_knots": d_kn}


def bsb_loss(p: Problem, R, K, dt, a0, c0, knots, S0, Y0) -> float:
    """L = mean_r E_relax(s_K) after K steps (used for finite differences)."""
    lib = _load()
    kn = np.ascontiguousarray(knots, dtype=np.float64)
    S0 = np.ascontiguousarray(S0, dtype=np.float32)
    Y0 = np.ascontiguousarray(Y0, dtype=np.float32)
    loss = ctypes.c_double()
    rc = lib.oracle_bsb_loss(p.n, p.nnz, _p(p.er), _p(p.ec), _p(p.ev), _p(p.c), R, K, dt, a0, c0,
                             kn.shape[0], _p(kn), _p(S0), _p(Y0), ctypes.byref(loss))
    if rc != 0:
        raise MemoryError("oracle_bsb_loss failed to allocate")
    return loss.value


# ---------------------------------------------------------------------------
# Library routines used as one step
# ---------------------------------------------------------------------------
def spectral_radius(p: Problem) -> float:
    """rho(Qoff) = max |eigenvalue| of the off-diagonal symmetric part.

    App. B sets c0 = 1/lambda_max(J); the Ising coupling of the dynamics is
    J = -Qoff/2, so rho(J) = rho(Qoff)/2. Dense symmetric eigen-solver for
    n <= 6000, Lanczos (scipy eigsh) above.
    """
    if p.n <= 6000:
        Qs = p.dense()
        Qs = 0.5 * (Qs + Qs.T)
        np.fill_diagonal(Qs, 0.0)
        w = np.linalg.eigvalsh(Qs)
        return float(np.max(np.abs(w)))
    import scipy.sparse as sp
    from scipy.sparse.linalg import eigsh
    off = p.er != p.ec
    A = sp.coo_matrix((p.ev[off], (p.er[off], p.ec[off])), shape=(p.n, p.n)).tocsr()
    A = 0.5 * (A + A.T)
    w = eigsh(A, k=1, which="LM", return_eigenvectors=False, tol=1e-10)
    return float(np.max(np.abs(w)))
