"""Third-order (HUBO) instances of Sec. "HUBO": the oracle's energy against
hand values and the global-flip identity, the generators' expansion against
the product form, and the library's reduction to second order (eq.
reduction) against the oracle by enumeration. CPU only (the reduction is host
code of the library)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2501_19221_gb300 import instances as I


def _all_spins(n):
    return np.array(list(itertools.product([-1, 1], repeat=n)), dtype=np.int8)


def test_hubo3_energy_by_hand():
    """n = 4: h = (1, 0, -2, 0), J_01 = 3, K_123 = -1.5 at s = (1, -1, 1, -1):
    1 - 2 + 3(1)(-1) - 1.5(-1)(1)(-1) = -5.5."""
    E = O.hubo3_energy(4, [1, 0, -2, 0], ([0], [1], [3.0]), ([1], [2], [3], [-1.5]), [[1, -1, 1, -1]])
    assert E[0] == -5.5


def test_hubo3_energy_global_flip():
    """Flipping every spin negates the odd-order terms and keeps the pairs:
    H(s) + H(-s) = 2 sum J s s (catches a dropped or mis-signed term)."""
    inst = I.hubo_chain_3body(9, seed=3)
    S = _all_spins(9)
    pi, pj, J = inst.pairs
    pair_only = O.hubo3_energy(9, None, inst.pairs, None, S)
    assert np.allclose(O.hubo3_energy(9, inst.h, inst.pairs, inst.triples, S) +
                       O.hubo3_energy(9, inst.h, inst.pairs, inst.triples, -S), 2 * pair_only, atol=1e-12)
    assert np.allclose(pair_only, (S[:, pi] * S[:, pj]) @ J)


def test_max3sat_expansion_equals_clause_product():
    """The expanded MAX 3-SAT cost equals sum_i (w_i/8) prod (1 + l s) on every
    assignment, i.e. the weight of the clauses whose three literals are all
    false."""
    N = 8
    inst = I.max3sat_weighted(N, seed=5)
    rng = np.random.default_rng(5)
    w = rng.uniform(0.0, 1.0, size=N - 2)
    l = 1.0 - 2.0 * rng.integers(0, 2, size=(N - 2, 3))
    S = _all_spins(N).astype(np.float64)
    direct = np.zeros(S.shape[0])
    for i in range(N - 2):
        direct += w[i] / 8 * (1 + l[i, 0] * S[:, i]) * (1 + l[i, 1] * S[:, i + 1]) * (1 + l[i, 2] * S[:, i + 2])
    E = inst.const + O.hubo3_energy(N, inst.h, inst.pairs, inst.triples, S)
    assert np.allclose(E, direct, atol=1e-12)


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2501_19221_gb300 import binding
    return binding


def _reduced_energy(red, S_all):
    """sum_{i<j} J s s + sum lin s + offset of the reduced instance, by the
    oracle's Ising energy on its dense upper triangle."""
    n = red["n"]
    J = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(red["rowptr"]))
    up = red["col"] > rows
    J[rows[up], red["col"][up]] = red["val"][up]
    return np.array([O.ising_energy(J, red["lin"], s) for s in S_all]) + red["offset"]


@pytest.mark.parametrize("kind", ["chain", "max3sat", "random"])
def test_reduction_minimum_over_auxiliaries_equals_hubo(B, kind):
    """For every assignment of the original spins, the minimum over the
    auxiliary spins of the reduced second-order cost equals the third-order
    cost (eq. reduction), with both signs of K and shared pairs."""
    if kind == "chain":
        inst = I.hubo_chain_3body(7, seed=1)
    elif kind == "max3sat":
        inst = I.max3sat_weighted(7, seed=2)
    else:
        rng = np.random.default_rng(9)
        n = 6
        trip = np.array([rng.choice(n, 3, replace=False) for _ in range(5)])
        pairs = np.array([rng.choice(n, 2, replace=False) for _ in range(4)])
        inst = I.Hubo3(n, rng.normal(size=n), (pairs[:, 0], pairs[:, 1], rng.normal(size=4)),
                       (trip[:, 0], trip[:, 1], trip[:, 2], rng.normal(size=5)))
    n = inst.n
    red = B.veloxq_hubo3_reduce(n, inst.h, inst.pairs, inst.triples)
    n3 = inst.triples[0].shape[0]
    assert red["n"] == n + n3
    # structurally symmetric with equal values, sorted, no diagonal
    rows = np.repeat(np.arange(red["n"]), np.diff(red["rowptr"]))
    M = {(int(r), int(c)): v for r, c, v in zip(rows, red["col"], red["val"])}
    assert all(M[(c, r)] == v for (r, c), v in M.items()) and all(r != c for r, c in M)
    for i in range(red["n"]):
        seg = red["col"][red["rowptr"][i]:red["rowptr"][i + 1]]
        assert np.all(np.diff(seg) > 0)
    S = _all_spins(n)
    A = _all_spins(n3)
    full = np.concatenate([np.repeat(S, len(A), axis=0), np.tile(A, (len(S), 1))], axis=1)
    Ered = _reduced_energy(red, full).reshape(len(S), len(A)).min(axis=1)
    Ehubo = O.hubo3_energy(n, inst.h, inst.pairs, inst.triples, S)
    assert np.allclose(Ered, Ehubo, atol=1e-9)


def test_reduction_rejects_bad_terms(B):
    with pytest.raises(B.VeloxqError):
        B.veloxq_hubo3_reduce(3, None, None, ([0], [0], [1], [1.0]))       # repeated index
    with pytest.raises(B.VeloxqError):
        B.veloxq_hubo3_reduce(3, None, ([0], [5], [1.0]), None)            # out of range


@pytest.mark.parametrize("kind", ["chain", "max3sat"])
def test_oracle_reduction_pinned_and_equal_to_library(B, kind):
    """The oracle's own reduction satisfies the same min-over-auxiliaries
    identity, and the library's merged CSR holds the same couplings (sums of
    the oracle's unmerged pairs, up to summation order) and fields."""
    inst = I.hubo_chain_3body(7, seed=4) if kind == "chain" else I.max3sat_weighted(7, seed=6)
    n = inst.n
    N, (qi, qj, qv), lin, off = O.hubo3_reduce(n, inst.h, inst.pairs, inst.triples)
    n3 = N - n
    S = _all_spins(n)
    A = _all_spins(n3)
    full = np.concatenate([np.repeat(S, len(A), axis=0), np.tile(A, (len(S), 1))], axis=1)
    Ered = O.hubo3_energy(N, lin, (qi, qj, qv), None, full) + off
    assert np.allclose(Ered.reshape(len(S), len(A)).min(axis=1),
                       O.hubo3_energy(n, inst.h, inst.pairs, inst.triples, S), atol=1e-9)
    red = B.veloxq_hubo3_reduce(n, inst.h, inst.pairs, inst.triples)
    Jo = np.zeros((N, N))
    np.add.at(Jo, (np.minimum(qi, qj), np.maximum(qi, qj)), qv)
    rows = np.repeat(np.arange(N), np.diff(red["rowptr"]))
    up = red["col"] > rows
    Jl = np.zeros((N, N))
    Jl[rows[up], red["col"][up]] = red["val"][up]
    assert np.allclose(Jl, Jo, rtol=0, atol=1e-12)
    assert np.allclose(red["lin"], lin, rtol=0, atol=1e-12) and red["offset"] == pytest.approx(off, abs=1e-12)


@pytest.mark.parametrize("kind", ["chain", "max3sat", "random"])
def test_local_numbering_is_a_relabeling(B, kind):
    """veloxq_hubo3_reduce_local is the default reduction with its spins
    renumbered: index is a permutation, and couplings, fields and offset
    agree under it; every auxiliary spin comes right after the largest
    original spin of its term (or after the auxiliaries anchored there)."""
    if kind == "chain":
        inst = I.hubo_chain_3body(40, seed=1)
    elif kind == "max3sat":
        inst = I.max3sat_weighted(40, seed=2)
    else:
        inst = I.xorsat_3r3x(40, seed=3).hubo
    n = inst.n
    a = B.veloxq_hubo3_reduce(n, inst.h, inst.pairs, inst.triples)
    b = B.veloxq_hubo3_reduce(n, inst.h, inst.pairs, inst.triples, local=True)
    P = b["index"]
    N = a["n"]
    assert b["n"] == N and np.array_equal(np.sort(P), np.arange(N))
    assert b["offset"] == a["offset"]
    assert np.array_equal(b["lin"][P], a["lin"])

    def dense(r):
        M = np.zeros((N, N))
        rows = np.repeat(np.arange(N), np.diff(r["rowptr"]))
        M[rows, r["col"]] = r["val"]
        return M

    assert np.array_equal(dense(b)[np.ix_(P, P)], dense(a))
    ti, tj, tk, _ = inst.triples
    anchor = np.maximum(np.maximum(ti, tj), tk)
    orig = P[:n]
    assert np.all(np.diff(orig) >= 1)                       # originals keep their order
    assert np.all(P[n:] > orig[anchor])
    nxt = np.append(orig[1:], N)
    assert np.all(P[n:] < nxt[anchor])                      # before the next original spin
    if kind == "chain":
        q = np.arange(n - 2)
        assert np.array_equal(P[n:], 2 * q + 3)
