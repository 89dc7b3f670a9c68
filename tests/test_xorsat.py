"""Planted 3-regular 3-XORSAT instances (Sec. "3-regular 3-XORSAT equation
planting"): the generator's structure, the planted ground energy pinned by
an independent solve of the equations over GF(2) and by enumeration, and
the second-order form (eq. reduction) by enumeration. CPU only."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2501_19221_gb300 import instances as I


def _gf2_solve(A: np.ndarray, b: np.ndarray):
    """Gaussian elimination over GF(2) of A x = b: (a solution with the free
    variables at 0, or None; the rank of A)."""
    M = np.concatenate([A.astype(np.uint8), b.astype(np.uint8)[:, None]], axis=1)
    m, n = A.shape
    row, pivots = 0, []
    for col in range(n):
        hit = np.flatnonzero(M[row:, col]) + row
        if hit.size == 0:
            continue
        M[[row, hit[0]]] = M[[hit[0], row]]
        others = np.flatnonzero(M[:, col])
        others = others[others != row]
        M[others] ^= M[row]
        pivots.append(col)
        row += 1
        if row == m:
            break
    if np.any(M[row:, n]):
        return None, row
    x = np.zeros(n, dtype=np.uint8)
    for r, col in enumerate(pivots):
        x[col] = M[r, n]
    return x, row


def _incidence(inst):
    n = inst.x_planted.shape[0]
    A = np.zeros((inst.T.shape[0], n), dtype=np.uint8)
    A[np.arange(inst.T.shape[0])[:, None], inst.T] = 1
    return A


def _energy(inst, S):
    h = inst.hubo
    return O.hubo3_energy(h.n, h.h, h.pairs, h.triples, np.asarray(S, dtype=np.float64))


@pytest.mark.parametrize("n", [4, 7, 1000])
def test_structure(n):
    """m = n equations of three distinct variables, each variable in exactly
    three, no equation twice, b = A x* (mod 2)."""
    inst = I.xorsat_3r3x(n, seed=n)
    T = inst.T
    assert T.shape == (n, 3)
    assert np.all(np.bincount(T.ravel(), minlength=n) == 3)
    assert np.all((T[:, 0] < T[:, 1]) & (T[:, 1] < T[:, 2]))
    assert len({tuple(r) for r in T.tolist()}) == n
    A = _incidence(inst)
    assert np.array_equal(A.astype(np.int64) @ inst.x_planted % 2, inst.b)
    assert inst.E0 == -n


@pytest.mark.parametrize("n,seed", [(200, 0), (1000, 3)])
def test_gf2_solution_reaches_planted_energy(n, seed):
    """Any solution of the equations, found here by elimination and not from
    the planted assignment, has energy -m, and every term is -1 there; the
    planted assignment too."""
    inst = I.xorsat_3r3x(n, seed=seed)
    x, rank = _gf2_solve(_incidence(inst), inst.b)
    assert x is not None and rank <= n
    s = 2 * x.astype(np.float64) - 1
    assert _energy(inst, s[None, :])[0] == inst.E0
    assert _energy(inst, inst.s_planted[None, :])[0] == inst.E0
    # one flipped variable breaks exactly its three equations: -m + 6
    s[0] = -s[0]
    assert _energy(inst, s[None, :])[0] == inst.E0 + 6


@pytest.mark.parametrize("n,seed", [(8, 1), (10, 2), (12, 5)])
def test_enumeration_minimum_and_degeneracy(n, seed):
    """Brute force: the minimum is -m and it is reached by exactly the
    2^(n - rank A) solutions of the system."""
    inst = I.xorsat_3r3x(n, seed=seed)
    S = np.array(list(itertools.product([-1, 1], repeat=n)), dtype=np.float64)
    E = _energy(inst, S)
    _, rank = _gf2_solve(_incidence(inst), inst.b)
    assert E.min() == inst.E0
    assert np.sum(E == inst.E0) == 2 ** (n - rank)


def test_reduced_form_keeps_the_ground_energy():
    """The second-order form (one auxiliary spin per equation, eq. reduction,
    by the oracle's reduction): over all 2^(n+m) spins its minimum is -m."""
    inst = I.xorsat_3r3x(8, seed=4)
    h = inst.hubo
    N, pairs, lin, off = O.hubo3_reduce(h.n, h.h, h.pairs, h.triples)
    assert N == 16
    S = np.array(list(itertools.product([-1, 1], repeat=N)), dtype=np.float64)
    E = O.hubo3_energy(N, lin, pairs, None, S) + off
    assert E.min() == pytest.approx(inst.E0, abs=1e-9)
