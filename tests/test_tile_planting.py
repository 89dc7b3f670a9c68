"""Tile-planted square lattices (Sec. "Tile planting"): the generator against
what the paper's definition fixes, checked without the generator's own
arithmetic.

* Each tile class C_i has exactly i ground states up to the global flip, one
  of them all +1 (enumeration of the 16 states of a square).
* The tiles of one checkerboard colour cover every edge of the periodic
  square lattice exactly once (the lattice's edge set written out here).
* The planted state is a ground state of the whole lattice and its energy is
  the generator's E0 (exhaustive search over 2^16 states at L = 4 through the
  oracle's App. A conversion, and the oracle's Ising energy at larger L).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2501_19221_gb300 import instances as I

SQUARE = [(0, 1), (1, 2), (2, 3), (3, 0)]       # a tile's four edges around its corners


def _square_energies(J):
    """H = -sum J_e s_a s_b over the square's edges for all 16 states."""
    out = {}
    for s in itertools.product((-1, 1), repeat=4):
        out[s] = -sum(J[e] * s[a] * s[b] for e, (a, b) in enumerate(SQUARE))
    return out


@pytest.mark.parametrize("cls", [1, 2, 3, 4])
def test_tile_class_has_i_ground_states_including_all_up(cls):
    """The defining property of C_i, for every order of its values around the
    square (the generator permutes them per tile)."""
    for J in set(itertools.permutations(I.TILE_CLASS_J[cls])):
        E = _square_energies(J)
        emin = min(E.values())
        ground = [s for s, e in E.items() if e == emin]
        assert len(ground) == 2 * cls                   # i states and their flips
        assert (1, 1, 1, 1) in ground
        assert emin == cls - 6                           # the per-tile term of E0


def _lattice_edges(L):
    """Every nearest-neighbour pair of the periodic L x L lattice, site y*L + x."""
    e = set()
    for y in range(L):
        for x in range(L):
            i = y * L + x
            for j in (y * L + (x + 1) % L, ((y + 1) % L) * L + x):
                e.add((min(i, j), max(i, j)))
    return e


@pytest.mark.parametrize("L", [4, 6, 10])
def test_tiles_cover_every_lattice_edge_once(L):
    tiles = I.tile_plaquettes(L)
    assert tiles.shape == (L * L // 2, 4, 2)
    seen = [tuple(sorted((int(a), int(b)))) for a, b in tiles.reshape(-1, 2)]
    assert len(seen) == len(set(seen)) == 2 * L * L
    assert set(seen) == _lattice_edges(L)
    # every site lies in exactly two tiles
    per_tile_sites = [set(t.reshape(-1).tolist()) for t in tiles]
    assert all(len(s) == 4 for s in per_tile_sites)
    occ = np.zeros(L * L, dtype=int)
    for s in per_tile_sites:
        occ[list(s)] += 1
    assert np.all(occ == 2)


@pytest.mark.parametrize("gauge", [False, True])
def test_csr_is_the_lattice_with_class_values(gauge):
    L = 8
    t = I.tile_planted_ising(L, p=(0.1, 0.4, 0.2, 0.3), seed=5, gauge=gauge)
    sp = t.sp
    assert sp.n == L * L and sp.nnz == 4 * L * L and sp.val.dtype == np.int8
    assert np.all(np.diff(sp.rowptr) == 4) and not np.any(sp.lin)
    D = sp.to_dense(np.int64)
    assert np.array_equal(D, D.T) and not np.any(np.diag(D))
    iu, ju = np.nonzero(np.triu(D))
    assert set(zip(iu.tolist(), ju.tolist())) == _lattice_edges(L)
    # undo the gauge and the sign convention: each tile carries its class's values
    s = t.s_planted.astype(np.int64)
    for tile, c in zip(I.tile_plaquettes(L), t.tile_class):
        vals = sorted(int(-D[a, b] * s[a] * s[b]) for a, b in tile)
        assert tuple(vals) == tuple(sorted(I.TILE_CLASS_J[int(c)]))
    if not gauge:
        assert np.all(t.s_planted == 1)


@pytest.mark.parametrize("p,seed", [((0.0, 0.2, 0.0, 0.8), 0), ((0.0, 0.8, 0.0, 0.2), 1),
                                     ((0.25, 0.25, 0.25, 0.25), 2), ((1.0, 0.0, 0.0, 0.0), 3)])
def test_planted_energy_is_the_ground_energy_by_enumeration(p, seed):
    """L = 4 (16 spins): the minimum over all 2^16 states is E0, reached by the
    planted state; via App. A, H(s) = 2 E(x) + C."""
    t = I.tile_planted_ising(4, p=p, seed=seed)
    sp = t.sp
    prob, C = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    Emin, _, count = O.bruteforce(prob)
    assert 2 * Emin + C == t.E0
    assert 2 * O.energy(prob, t.x_planted[None])[0] + C == t.E0
    # the ground states come at least in the pair s*, -s*
    assert count >= 2


@pytest.mark.parametrize("L,p2", [(12, 0.2), (20, 0.8)])
def test_planted_state_energy_and_single_flips(L, p2):
    t = I.tile_planted_ising(L, p=(0.0, p2, 0.0, 1.0 - p2), seed=7)
    sp = t.sp
    J = np.triu(sp.to_dense(np.float64))
    s = t.s_planted.astype(np.int8)
    assert O.ising_energy(J, np.zeros(sp.n), s) == t.E0
    assert t.E0 == np.sum(t.tile_class.astype(np.int64) - 6)
    # a ground state: no single flip lowers the energy
    prob, C = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    X = np.repeat(t.x_planted[None], sp.n, axis=0)
    X[np.arange(sp.n), np.arange(sp.n)] ^= 1
    assert np.all(2 * O.energy(prob, X) + C >= t.E0)


def test_class_frequencies_follow_p():
    t = I.tile_planted_ising(100, p=(0.0, 0.2, 0.0, 0.8), seed=0)
    k = np.bincount(t.tile_class, minlength=5)[1:]
    m = t.tile_class.shape[0]
    assert k[0] == 0 and k[2] == 0
    assert abs(k[1] - 0.2 * m) <= 5 * np.sqrt(m * 0.2 * 0.8)


def test_rejects_odd_or_tiny_lattices_and_bad_p():
    for L in (2, 5, 7):
        with pytest.raises(ValueError):
            I.tile_planted_ising(L)
    with pytest.raises(ValueError):
        I.tile_planted_ising(6, p=(0.5, 0.5, 0.5, 0.0))
