"""Seeded synthetic problem instances shaped like the benchmark families of the
VeloxQ benchmark paper (arXiv:2501.19221).

This module only draws random numbers and lays out graphs. It holds none of the
solver's arithmetic: no energy, no QUBO/Ising conversion (App. A), no dynamics,
no normalisation. Both the CUDA library and the FP64 oracle consume what it
returns, so a mistake here cannot hide a disagreement between the two.

Families (each cites the passage whose shape it imitates):

* ``dense_int_qubo``  -- small dense QUBO with integer couplings; the dense
  all-to-all instances of Sec. "Brute force" use couplings uniform in [-1, 1].
* ``sk_qubo``         -- dense Sherrington-Kirkpatrick-type QUBO with Gaussian
  couplings scaled by 1/sqrt(n) (dense instances of the B&B comparison).
* ``chimera_ising``   -- Chimera C_{m,n} graph of K_{4,4} cells with +-J
  couplings (Sec. "Structure-exploiting solvers").
* ``wishart_ising``   -- Wishart planted ensemble (Sec. "Wishart ensemble").
* ``cubic_lattice_ising`` -- periodic 3-D +-J lattice (periodic-lattice
  planting family, very large sparse instances of Sec. "Zephyr").
* ``random_sparse_qubo`` -- ragged sparse QUBO (empty rows, uneven degree) used
  as an edge case by the tests.
* ``pegasus_edges`` / ``zephyr_csr`` and ``pegasus_qubo`` / ``zephyr_qubo`` --
  the D-Wave Pegasus P_m and Zephyr Z_{m,t} topologies (Sec. "Pegasus
  topology", Sec. "Zephyr topology") with random QUBO couplings on their
  edges.
* ``tile_planted_ising`` -- tile-planted periodic square lattice with a known
  ground state (Sec. "Tile planting").

Sparse instances are returned as symmetric CSR (both (i, j) and (j, i) are
stored, column indices strictly increasing within each row, no diagonal).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "SparseCoupling",
    "dense_int_qubo",
    "sk_qubo",
    "chimera_edges",
    "chimera_ising",
    "cubic_lattice_ising",
    "wishart_ising",
    "wishart_sizes",
    "random_sparse_qubo",
    "uniform_state",
    "random_binary",
    "pegasus_edges",
    "pegasus_qubo",
    "zephyr_csr",
    "zephyr_qubo",
    "tile_planted_ising",
]


@dataclass
class SparseCoupling:
    """A symmetric sparse coupling matrix in CSR form plus a linear term.

    ``rowptr`` is int64 (n+1), ``col`` int32 (nnz), ``val`` the coupling values
    (int8 / int32 / float32 / float64), ``lin`` the linear term (h for an Ising
    model, c for a QUBO) as float64 (n).
    """

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    lin: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self, dtype=np.float64) -> np.ndarray:
        out = np.zeros((self.n, self.n), dtype=dtype)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        out[rows, self.col] = self.val
        return out


def _csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray) -> tuple:
    """Symmetric CSR from an undirected edge list (u < v), sorted columns."""
    rows = np.concatenate([u, v]).astype(np.int64)
    cols = np.concatenate([v, u]).astype(np.int64)
    vals = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, cols.astype(np.int32), vals


def dense_int_qubo(n: int = 20, lo: int = -8, hi: int = 8, seed: int = 0):
    """Dense symmetric integer QUBO matrix (int32, n x n) and c = 0.

    The upper triangle including the diagonal is drawn uniformly from the
    integers [lo, hi] and mirrored into the lower triangle.
    """
    rng = np.random.default_rng(seed)
    upper = rng.integers(lo, hi + 1, size=(n, n), dtype=np.int64)
    Q = np.triu(upper) + np.triu(upper, 1).T
    return Q.astype(np.int32), np.zeros(n, dtype=np.float64)


def sk_qubo(n: int = 8192, seed: int = 0, dtype=np.float32):
    """Dense symmetric Gaussian QUBO: Q_ij ~ N(0, 1)/sqrt(n), Q_ii = 0, c = 0."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n), dtype=np.float32) if dtype == np.float32 else rng.standard_normal((n, n))
    Q = np.triu(g, 1)
    Q = Q + Q.T
    Q *= np.asarray(1.0 / np.sqrt(n), dtype=Q.dtype)
    return np.ascontiguousarray(Q.astype(dtype)), np.zeros(n, dtype=np.float64)


def chimera_edges(m: int = 16, n: int = 16, t: int = 4):
    """Edges (u < v) of the Chimera graph C_{m,n} with shore size t.

    Vertex (row, col, shore, k) has index ((row*n + col)*2 + shore)*t + k.
    Inside a cell the two shores form a complete bipartite graph K_{t,t};
    shore 0 couples to the same k in the cell below, shore 1 to the same k in
    the cell to the right.
    """
    def vid(r, c, s, k):
        return ((r * n + c) * 2 + s) * t + k

    us, vs = [], []
    for r in range(m):
        for c in range(n):
            for k1 in range(t):
                for k2 in range(t):
                    us.append(vid(r, c, 0, k1))
                    vs.append(vid(r, c, 1, k2))
            for k in range(t):
                if r + 1 < m:
                    us.append(vid(r, c, 0, k))
                    vs.append(vid(r + 1, c, 0, k))
                if c + 1 < n:
                    us.append(vid(r, c, 1, k))
                    vs.append(vid(r, c + 1, 1, k))
    u = np.asarray(us, dtype=np.int64)
    v = np.asarray(vs, dtype=np.int64)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    return lo, hi


def chimera_ising(m: int = 16, n: int = 16, t: int = 4, seed: int = 0) -> SparseCoupling:
    """Ising model on C_{m,n}: J uniform on {-1, +1} per edge (int8), h = 0."""
    u, v = chimera_edges(m, n, t)
    rng = np.random.default_rng(seed)
    w = (2 * rng.integers(0, 2, size=u.shape[0]) - 1).astype(np.int8)
    nv = 2 * t * m * n
    rowptr, col, val = _csr_from_edges(nv, u, v, w)
    return SparseCoupling(nv, rowptr, col, val, np.zeros(nv, dtype=np.float64))


def cubic_lattice_ising(L: int, seed: int = 0) -> SparseCoupling:
    """Periodic L x L x L +-J lattice (int8 couplings, h = 0), L >= 3.

    Site (x, y, z) has index (z*L + y)*L + x. Each site owns the three bonds
    to +x, +y, +z; every row therefore holds exactly six entries.
    """
    if L < 3:
        raise ValueError("L must be >= 3 so that the six neighbours are distinct")
    n = L * L * L
    rng = np.random.default_rng(seed)
    # one +-1 bond per site and direction (bond from i to i + e_d)
    bonds = (2 * rng.integers(0, 2, size=(3, n), dtype=np.int8) - 1).astype(np.int8)
    idx = np.arange(n, dtype=np.int64)
    x = idx % L
    y = (idx // L) % L
    z = idx // (L * L)
    strides = (1, L, L * L)
    coords = (x, y, z)
    cols = np.empty((6, n), dtype=np.int64)
    vals = np.empty((6, n), dtype=np.int8)
    for d in range(3):
        s = strides[d]
        c = coords[d]
        plus = idx + np.where(c == L - 1, -(L - 1) * s, s)
        minus = idx - np.where(c == 0, -(L - 1) * s, s)
        cols[2 * d] = plus
        vals[2 * d] = bonds[d]
        cols[2 * d + 1] = minus
        vals[2 * d + 1] = bonds[d][minus]
    del idx, x, y, z
    # sort the six columns of every row: odd-even transposition sort, 6 rounds
    pairs = [(0, 1), (2, 3), (4, 5), (1, 2), (3, 4)] * 3
    for a, b in pairs:
        swap = cols[a] > cols[b]
        ca, cb = cols[a].copy(), cols[b].copy()
        va, vb = vals[a].copy(), vals[b].copy()
        cols[a] = np.where(swap, cb, ca)
        cols[b] = np.where(swap, ca, cb)
        vals[a] = np.where(swap, vb, va)
        vals[b] = np.where(swap, va, vb)
    col = np.ascontiguousarray(cols.T).reshape(-1).astype(np.int32)
    val = np.ascontiguousarray(vals.T).reshape(-1)
    rowptr = np.arange(n + 1, dtype=np.int64) * 6
    return SparseCoupling(n, rowptr, col, val, np.zeros(n, dtype=np.float64))


def wishart_ising(N: int, alpha: float, seed: int = 0, dtype=np.float64) -> dict:
    """Wishart planted ensemble (Sec. "Wishart ensemble").

    Draws a planted +-1 vector t (gauge randomisation of the ferromagnetic
    state), M = max(1, round(alpha*N)) columns w ~ N(0, Sigma) with
    Sigma = N/(N-1) (I - t t^T / N), and returns

    * ``J``  -- the coupling matrix of H_WP = -1/2 sum_{i,j} J_ij s_i s_j,
      J = Jt - diag(Jt) with Jt = -W W^T / N (zero diagonal, symmetric);
    * ``Jt_diag`` -- diag(Jt), from which the planted energy follows;
    * ``t``  -- the planted state (int8);
    * ``W``  -- the N x M matrix.
    """
    rng = np.random.default_rng(seed)
    t = (2 * rng.integers(0, 2, size=N) - 1).astype(np.float64)
    M = max(1, int(round(alpha * N)))
    z = rng.standard_normal((N, M))
    proj = z - np.outer(t, t @ z) / N
    W = np.sqrt(N / (N - 1.0)) * proj
    Jt = -(W @ W.T) / N
    d = np.diag(Jt).copy()
    J = Jt - np.diag(d)
    return {"J": J.astype(dtype), "Jt_diag": d, "t": t.astype(np.int8), "W": W}


def wishart_sizes(count: int = 512, nmin: int = 100, nmax: int = 2000, seed: int = 0) -> np.ndarray:
    """Instance sizes n_i uniform on {nmin, ..., nmax} for a Wishart batch."""
    rng = np.random.default_rng(seed)
    return rng.integers(nmin, nmax + 1, size=count)


def random_sparse_qubo(n: int, mean_degree: float, seed: int = 0, vtype=np.int32,
                       lo: int = -5, hi: int = 5, empty_rows: int = 0,
                       with_diag: bool = True) -> SparseCoupling:
    """Ragged symmetric sparse QUBO for edge-case tests.

    Edges are drawn uniformly (duplicates removed); the first ``empty_rows``
    vertices get no edges at all. Values are integers in [lo, hi] \\ {0}
    (cast to ``vtype``). If ``with_diag`` the diagonal is stored too, so the
    CSR also carries linear terms the way a QUBO matrix does.
    """
    rng = np.random.default_rng(seed)
    m = int(mean_degree * n / 2)
    u = rng.integers(empty_rows, n, size=m)
    v = rng.integers(empty_rows, n, size=m)
    keep = u != v
    u, v = u[keep], v[keep]
    lo_, hi_ = np.minimum(u, v), np.maximum(u, v)
    key = np.unique(lo_ * n + hi_)
    lo_, hi_ = key // n, key % n
    w = rng.integers(lo, hi + 1, size=lo_.shape[0])
    w[w == 0] = 1
    if with_diag:
        diag_idx = np.arange(n, dtype=np.int64)
        dw = rng.integers(lo, hi + 1, size=n)
        rows = np.concatenate([lo_, hi_, diag_idx])
        cols = np.concatenate([hi_, lo_, diag_idx])
        vals = np.concatenate([w, w, dw])
        order = np.lexsort((cols, rows))
        rows, cols, vals = rows[order], cols[order], vals[order]
        counts = np.bincount(rows, minlength=n)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
        col = cols.astype(np.int32)
        val = vals
    else:
        rowptr, col, val = _csr_from_edges(n, lo_, hi_, w)
    return SparseCoupling(n, rowptr, col, np.asarray(val).astype(vtype), np.zeros(n, dtype=np.float64))


def uniform_state(R: int, n: int, lo: float = -1.0, hi: float = 1.0, seed: int = 0) -> np.ndarray:
    """A float32 replica-major state block [R][n] with entries uniform in [lo, hi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(R, n)).astype(np.float32)


def random_binary(B: int, n: int, seed: int = 0, p: float = 0.5) -> np.ndarray:
    """A uint8 batch [B][n] of binary vectors with P(x_i = 1) = p."""
    rng = np.random.default_rng(seed)
    return (rng.random((B, n)) < p).astype(np.uint8)


# ---------------------------------------------------------------- third-order (HUBO) instances
class Hubo3:
    """A third-order Ising cost function
    H(s) = const + sum h s + sum J s_pi s_pj + sum K s_ti s_tj s_tk."""

    def __init__(self, n, h, pairs, triples, const=0.0):
        self.n = int(n)
        self.h = np.asarray(h, dtype=np.float64)
        self.pairs = tuple(pairs)        # (pi, pj, J)
        self.triples = tuple(triples)    # (ti, tj, tk, K)
        self.const = float(const)


def hubo_chain_3body(N: int, seed: int = 0) -> Hubo3:
    """One-dimensional spin glass with nearest-neighbour two- and three-body
    terms (Sec. "HUBO", eq. nn): h_i, J_i, K_i ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(N)
    J = rng.standard_normal(max(N - 1, 0))
    K = rng.standard_normal(max(N - 2, 0))
    i1 = np.arange(max(N - 1, 0), dtype=np.int64)
    i2 = np.arange(max(N - 2, 0), dtype=np.int64)
    return Hubo3(N, h, (i1, i1 + 1, J), (i2, i2 + 1, i2 + 2, K))


def max3sat_weighted(N: int, seed: int = 0) -> Hubo3:
    """Weighted MAX 3-SAT on consecutive triples (Sec. "HUBO", eq. mw3s):
    clause i weighs w_i ~ U[0, 1] and contributes (w_i/8) prod_{m=0..2}
    (1 + l_m s_{i+m}), l_m = (-1)^{c_m}, c_m ~ {0, 1}; the product is expanded
    into its constant, field, pair and triple terms."""
    rng = np.random.default_rng(seed)
    M = max(N - 2, 0)
    w = rng.uniform(0.0, 1.0, size=M)
    c = rng.integers(0, 2, size=(M, 3))
    l = 1.0 - 2.0 * c                     # (-1)^c
    i = np.arange(M, dtype=np.int64)
    idx = [i, i + 1, i + 2]
    e = w / 8.0
    h = np.zeros(N)
    for m in range(3):
        np.add.at(h, idx[m], e * l[:, m])
    pi = np.concatenate([idx[0], idx[0], idx[1]])
    pj = np.concatenate([idx[1], idx[2], idx[2]])
    pv = np.concatenate([e * l[:, 0] * l[:, 1], e * l[:, 0] * l[:, 2], e * l[:, 1] * l[:, 2]])
    K = e * l[:, 0] * l[:, 1] * l[:, 2]
    return Hubo3(N, h, (pi, pj, pv), (idx[0], idx[1], idx[2], K), const=float(e.sum()))


class Xorsat3R3X:
    """A planted 3-regular 3-XORSAT instance: the equations (T, b), the
    planted assignment and the third-order Ising cost built from them."""

    def __init__(self, T, b, x_planted, hubo, E0):
        self.T = T                    # [m][3] int64, the variables of equation i (distinct, sorted)
        self.b = b                    # [m] uint8, right-hand sides
        self.x_planted = x_planted    # [n] uint8
        self.s_planted = (2 * x_planted.astype(np.int8) - 1).astype(np.int8)
        self.hubo = hubo              # Hubo3: sum_i K_i s_i1 s_i2 s_i3, K_i = (-1)^b_i
        self.E0 = E0                  # ground energy, -m


def _three_regular_triples(n: int, rng, max_rounds: int = 100000) -> np.ndarray:
    """m = n triples of distinct variables, every variable in exactly three of
    them and no triple twice: three copies of every variable dealt at random
    into rows of three, then rows that repeat a variable or an earlier row
    swap one entry with a random entry elsewhere (which keeps every
    variable's count at three) until none is left."""
    if n < 4:
        raise ValueError("a 3-regular 3-XORSAT instance needs n >= 4")
    T = rng.permutation(np.repeat(np.arange(n, dtype=np.int64), 3)).reshape(n, 3)
    for _ in range(max_rounds):
        S = np.sort(T, axis=1)
        bad = (S[:, 0] == S[:, 1]) | (S[:, 1] == S[:, 2])
        _, first = np.unique(S, axis=0, return_index=True)
        again = np.ones(n, dtype=bool)
        again[first] = False
        rows = np.flatnonzero(bad | again)
        if rows.size == 0:
            return S
        for r in rows:
            q, a, c = int(rng.integers(n)), int(rng.integers(3)), int(rng.integers(3))
            T[r, a], T[q, c] = T[q, c], T[r, a]
    raise RuntimeError("no simple 3-regular triple system found")


def xorsat_3r3x(n: int, seed: int = 0) -> Xorsat3R3X:
    """Planted 3-regular 3-XORSAT (Sec. "3-regular 3-XORSAT equation
    planting"): m = n equations sum_{j in T_i} x_j = b_i (mod 2) over three
    distinct variables each, every variable in exactly three equations. A
    uniformly random x* fixes b = A x* (mod 2), so the system has a solution.

    With sigma_j = (-1)^{x_j} the equations read prod sigma = (-1)^{b_i} and
    the cost is -sum_i (-1)^{b_i} prod sigma. The library's spins are
    s = 2x - 1 = -sigma, and a product of three flips sign, so the cost is
    sum_i K_i s_i1 s_i2 s_i3 with K_i = (-1)^{b_i}. Each term is at least -1
    and equals -1 exactly when equation i holds: the ground energy is -m,
    reached at s* = 2x* - 1 and at every other solution of the system."""
    rng = np.random.default_rng(seed)
    T = _three_regular_triples(n, rng)
    x = rng.integers(0, 2, size=n).astype(np.uint8)
    b = (x[T[:, 0]] ^ x[T[:, 1]] ^ x[T[:, 2]]).astype(np.uint8)
    K = 1.0 - 2.0 * b.astype(np.float64)
    empty = np.zeros(0, dtype=np.int64)
    hubo = Hubo3(n, np.zeros(n), (empty, empty, np.zeros(0)), (T[:, 0], T[:, 1], T[:, 2], K))
    return Xorsat3R3X(T, b, x, hubo, -float(n))


# ----------------------------------------------------------------------------- annealer topologies
# Both are graphs of line segments (qubits) on a grid: a vertical and a
# horizontal segment that cross are joined by an internal coupler, collinear
# neighbouring segments by an external coupler, and paired parallel segments
# by an odd coupler (Boothby et al., "Next-generation topology of D-Wave
# quantum processors", 2020, for Pegasus; the Zephyr topology white paper of
# 2021 for Zephyr).

# Pegasus: per-track offsets of the segments of the standard topology (track k
# of a vertical / horizontal bundle), in units of the 12-track tile.
_PEG_OFF_V = np.array([2, 2, 2, 2, 10, 10, 10, 10, 6, 6, 6, 6], dtype=np.int64)
_PEG_OFF_H = np.array([6, 6, 6, 6, 2, 2, 2, 2, 10, 10, 10, 10], dtype=np.int64)


def pegasus_edges(m: int):
    """The Pegasus graph P_m, fabric only: (n, u, v) with edges u < v.

    Qubit (o, w, k, z), o in {0 vertical, 1 horizontal}, w in [0, m),
    k in [0, 12), z in [0, m - 1), is the segment on track 12 w + k spanning
    [12 z + off_o[k], 12 z + off_o[k] + 12) along its direction. Internal
    couplers join crossing vertical and horizontal segments, external ones
    (o, w, k, z) and (o, w, k, z + 1), odd ones tracks 2i and 2i + 1 of the
    same (o, w, z). Qubits without an internal coupler (at the boundary) are
    not part of the fabric and are dropped; the rest are numbered in order of
    (o, w, k, z)."""
    if m < 2:
        raise ValueError("Pegasus needs m >= 2")
    M1 = m - 1

    def idx(o, w, k, z):
        return ((o * m + w) * 12 + k) * M1 + z

    w, k, z = np.meshgrid(np.arange(m), np.arange(12), np.arange(M1), indexing="ij")
    w, k, z = w.ravel(), k.ravel(), z.ravel()
    us, vs = [], []
    for o in (0, 1):
        e = z + 1 < M1
        us.append(idx(o, w[e], k[e], z[e]))
        vs.append(idx(o, w[e], k[e], z[e] + 1))
        e = k % 2 == 0
        us.append(idx(o, w[e], k[e], z[e]))
        vs.append(idx(o, w[e], k[e] + 1, z[e]))
    # internal: each vertical segment crosses the 12 rows of its span; row y is
    # track k' = y % 12 of horizontal bundle w' = y // 12, whose segment over
    # column x = 12 w + k is z' = (x - off_H[k']) // 12
    x = 12 * w + k
    y0 = 12 * z + _PEG_OFF_V[k]
    for dy in range(12):
        y = y0 + dy
        wp, kp = y // 12, y % 12
        zp = np.floor_divide(x - _PEG_OFF_H[kp], 12)
        e = (wp < m) & (zp >= 0) & (zp < M1)
        us.append(idx(0, w[e], k[e], z[e]))
        vs.append(idx(1, wp[e], kp[e], zp[e]))
    u = np.concatenate(us)
    v = np.concatenate(vs)
    nfull = 2 * m * 12 * M1
    internal = np.zeros(nfull, dtype=bool)
    cut = sum(a.shape[0] for a in us[:4])          # the external and odd couplers come first
    internal[u[cut:]] = True
    internal[v[cut:]] = True
    keep = internal[u] & internal[v]
    new = np.cumsum(internal) - 1
    u, v = new[u[keep]], new[v[keep]]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    return int(internal.sum()), lo.astype(np.int64), hi.astype(np.int64)


def _pair_uniform(lo: np.ndarray, hi: np.ndarray, n: int, seed: int) -> np.ndarray:
    """A value uniform in [-1, 1) per unordered pair (lo < hi), from a
    counter-based hash of (seed, lo n + hi) (SplitMix64's finaliser): the same
    at (i, j) and (j, i) without an edge list."""
    x = (lo.astype(np.uint64) * np.uint64(n) + hi.astype(np.uint64)) ^ np.uint64((seed * 0x9E3779B97F4A7C15) & (2 ** 64 - 1))
    with np.errstate(over="ignore"):
        x = x + np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    return ((x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) * 2.0 - 1.0


def pegasus_qubo(m: int, seed: int = 0) -> SparseCoupling:
    """Random QUBO on the Pegasus fabric P_m (Sec. "Pegasus topology"):
    Q_ij ~ U[-1, 1) on every coupler, linear terms c_i ~ U[-1, 1). Stored as
    a symmetric float32 CSR with Q_ij / 2 at both (i, j) and (j, i), so that a
    pair contributes Q_ij x_i x_j to E(x) = sum_ij Q_ij x_i x_j + c x."""
    n, u, v = pegasus_edges(m)
    q = _pair_uniform(u, v, n, seed)
    rowptr, col, val = _csr_from_edges(n, u, v, (0.5 * q).astype(np.float32))
    lin = np.random.default_rng(seed + 1).uniform(-1.0, 1.0, size=n)
    return SparseCoupling(n, rowptr, col, val, lin)


def zephyr_csr(m: int, t: int = 4):
    """The Zephyr graph Z_{m,t} as a symmetric CSR pattern: (n, rowptr, col).

    Qubit (o, w, k, j, z), o in {0 vertical, 1 horizontal}, w in [0, 2m],
    k in [0, t), j in {0, 1}, z in [0, m), is the segment on track (k, j) of
    bundle w spanning half-tiles [2 z + j, 2 z + j + 2) along its direction
    (the j = 1 tracks staggered by one half-tile). Internal couplers join
    crossing segments (each crosses the 2t tracks of the two bundles of its
    span: 4t of them away from the boundary), external ones (..., z) and
    (..., z + 1), odd ones the two overlapping segments of the other track of
    the same (o, w, k). n = 4 t m (2 m + 1); degree at most 4 t + 4.
    Built as a table of every qubit's neighbours (4 t + 4 columns), so that no
    global sort of the ~n (2t + 2) entries is needed."""
    if m < 1 or t < 1:
        raise ValueError("Zephyr needs m >= 1 and t >= 1")
    W = 2 * m + 1
    n = 2 * W * t * 2 * m

    def idx(o, w, k, j, z):
        return (((o * W + w) * t + k) * 2 + j) * m + z

    D = 4 * t + 4
    half = n // 2                                      # qubits of one orientation, in (w, k, j, z) order
    it = np.int64 if n > 2 ** 31 - 2 else np.int32
    nb = np.empty((n, D), dtype=it)
    w, k, j, z = (a.ravel().astype(it) for a in
                  np.meshgrid(np.arange(W), np.arange(t), np.arange(2), np.arange(m), indexing="ij"))
    for o in (0, 1):
        blk = nb[o * half:(o + 1) * half]              # rows of this orientation, contiguous
        cols = []
        # external
        cols.append(np.where(z + 1 < m, idx(o, w, k, j, z + 1), -1))
        cols.append(np.where(z >= 1, idx(o, w, k, j, z - 1), -1))
        # odd: the segments of the other track of (o, w, k) that overlap this one
        zb = np.where(j == 0, z - 1, z + 1)
        cols.append(idx(o, w, k, 1 - j, z))
        cols.append(np.where((zb >= 0) & (zb < m), idx(o, w, k, 1 - j, zb), -1))
        # internal: bundles w' in {2z + j, 2z + j + 1} of the other orientation;
        # track (k', j') of bundle w' covers this qubit's bundle w when
        # j' <= w < 2m + j', with the segment z' = (w - j') // 2
        for dw in (0, 1):
            wp = 2 * z + j + dw
            for kp in range(t):
                for jp in (0, 1):
                    cols.append(np.where((jp <= w) & (w < 2 * m + jp), idx(1 - o, wp, kp, jp, (w - jp) // 2), -1))
        assert len(cols) == D
        for c, v in enumerate(cols):
            blk[:, c] = v
        del cols
    nb.sort(axis=1)                                    # -1 (absent) first, then ascending columns
    deg = (nb >= 0).sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rowptr[1:])
    col = nb[nb >= 0].astype(np.int32)
    return n, rowptr, col


def zephyr_qubo(m: int, t: int = 4, seed: int = 0) -> SparseCoupling:
    """Random QUBO on the Zephyr graph Z_{m,t} (Sec. "Zephyr topology"):
    Q_ij ~ U[-1, 1) on every coupler, c_i ~ U[-1, 1); symmetric float32 CSR
    with Q_ij / 2 at both positions, as pegasus_qubo."""
    n, rowptr, col = zephyr_csr(m, t)
    val = np.empty(col.shape[0], dtype=np.float32)
    step = 1 << 22                                     # rows per chunk (bounded temporaries)
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        p0, p1 = int(rowptr[r0]), int(rowptr[r1])
        rows = np.repeat(np.arange(r0, r1, dtype=np.int64), np.diff(rowptr[r0:r1 + 1]))
        c64 = col[p0:p1].astype(np.int64)
        val[p0:p1] = 0.5 * _pair_uniform(np.minimum(rows, c64), np.maximum(rows, c64), n, seed)
    lin = np.random.default_rng(seed + 1).uniform(-1.0, 1.0, size=n)
    return SparseCoupling(n, rowptr, col, val, lin)


# ----------------------------------------------------------------------------- tile planting
# Coupling values of the four tile classes, in the convention of Sec. "Tile
# planting" (H_C = -sum over the tile's four edges of J_ij s_i s_j, target
# ground state all +1). The paper defines class C_i only by its ground-state
# count: i ground states, up to the global flip, one of them all +1. Here each
# tile is a frustrated square (one antiferromagnetic bond, J = -1) whose other
# bonds are ferromagnetic, i - 1 of them with J = +1 and 4 - i with J = +2.
# A frustrated square violates an odd number of bonds in every state, so its
# ground states are those that violate exactly one of its weakest bonds: i of
# them up to the flip, all +1 (which violates the -1 bond) among them, at
# energy -(sum |J|) + 2 = i - 6.
TILE_CLASS_J = {1: (-1, 2, 2, 2), 2: (-1, 1, 2, 2), 3: (-1, 1, 1, 2), 4: (-1, 1, 1, 1)}


class TilePlanted:
    """A tile-planted square-lattice Ising instance: the couplings in the
    library's Ising convention (sp), the planted ground state, its energy and
    the class of every tile."""

    def __init__(self, sp, s_planted, E0, tile_class, L):
        self.sp = sp                  # SparseCoupling, H(s) = sum_{i<j} J_ij s_i s_j (h = 0)
        self.s_planted = s_planted    # [n] int8, +-1: a ground state
        self.x_planted = ((s_planted.astype(np.int16) + 1) // 2).astype(np.uint8)
        self.E0 = E0                  # ground energy of H (sum of the tiles' minima)
        self.tile_class = tile_class  # [L*L/2] int8, the class 1..4 of tile t
        self.L = L


def tile_plaquettes(L: int) -> np.ndarray:
    """The tiles of the periodic L x L square lattice (L even): the plaquettes
    of one colour of the checkerboard, those with lower-left corner (x, y) and
    x + y even. Returns [L*L/2][4][2] site indices of the tile's four edges in
    the order bottom, right, top, left; site (x, y) is y*L + x. Every lattice
    edge lies in exactly one tile and every site in two."""
    ys, xs = np.divmod(np.arange(L * L, dtype=np.int64), L)
    keep = (xs + ys) % 2 == 0
    x, y = xs[keep], ys[keep]
    x1, y1 = (x + 1) % L, (y + 1) % L
    a, b, c, d = y * L + x, y * L + x1, y1 * L + x1, y1 * L + x   # corners counter-clockwise
    return np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([d, c], 1), np.stack([a, d], 1)], 1)


def tile_planted_ising(L: int, p=(0.0, 0.2, 0.0, 0.8), seed: int = 0, gauge: bool = True) -> TilePlanted:
    """Tile-planted instance on the periodic L x L square lattice (Sec. "Tile
    planting"): every tile of the checkerboard draws its class C_i with
    probability p[i-1] and its four coupling values (TILE_CLASS_J) in a random
    order over its four edges. All tiles then share the ground state all +1,
    so the lattice does too, with energy sum_tiles (i - 6). With gauge, a
    random s* in {+-1}^n hides it: J_ij -> s*_i s*_j J_ij, ground state s*.
    The paper's benchmark draws p = (0, p2, 0, 1 - p2), p2 = 0.2 (easy) or 0.8
    (hard), L in [10, 300]. The couplings are returned in the library's Ising
    convention, H(s) = sum_{i<j} J_ij s_i s_j (that is, -J of the tile
    Hamiltonian), as int8 CSR with h = 0."""
    if L < 4 or L % 2:
        raise ValueError("tile planting needs an even L >= 4 (a periodic checkerboard with distinct neighbours)")
    p = np.asarray(p, dtype=np.float64)
    if p.shape != (4,) or np.any(p < 0) or abs(p.sum() - 1.0) > 1e-12:
        raise ValueError("p must be four probabilities summing to 1")
    rng = np.random.default_rng(seed)
    n = L * L
    tiles = tile_plaquettes(L)
    cls = (rng.choice(4, size=tiles.shape[0], p=p) + 1).astype(np.int8)
    table = np.array([TILE_CLASS_J[i] for i in range(1, 5)], dtype=np.int8)
    J = rng.permuted(table[cls - 1], axis=1)           # tile-convention couplings, per edge of each tile
    s = (2 * rng.integers(0, 2, size=n) - 1).astype(np.int8) if gauge else np.ones(n, dtype=np.int8)
    u, v = tiles[:, :, 0].reshape(-1), tiles[:, :, 1].reshape(-1)
    Jg = (J.reshape(-1) * s[u] * s[v]).astype(np.int8)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    rowptr, col, val = _csr_from_edges(n, lo, hi, (-Jg).astype(np.int8))
    E0 = float(np.sum(cls.astype(np.int64) - 6))
    return TilePlanted(SparseCoupling(n, rowptr, col, val, np.zeros(n, dtype=np.float64)), s, E0, cls, L)
