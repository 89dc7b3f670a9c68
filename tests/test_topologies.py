"""The annealer topologies the paper benchmarks (Sec. "Pegasus topology",
Sec. "Zephyr topology"), pinned to the sizes the paper and D-Wave publish and
to the structure their definitions imply: the paper's P_2 of 40 qubits and
Z_1 of 48 qubits with a native K_{8,8}, its P_150 of about 5e5 and Z_150 of
about 7.2e5 variables and its Z_1750 of more than 9.8e7, and the 5640 qubits
and 40,484 couplers of the Pegasus P_16 fabric (Boothby et al. 2020)."""
import itertools

import numpy as np
import pytest

from paper_2501_19221_gb300 import instances as I


def _adjacency(n, rowptr, col):
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return set(zip(rows.tolist(), col.tolist()))


def test_pegasus_published_sizes():
    n2, u2, _ = I.pegasus_edges(2)
    assert n2 == 40                                   # the paper's P_2 on 40 qubits
    n16, u16, _ = I.pegasus_edges(16)
    assert (n16, u16.shape[0]) == (5640, 40484)       # the P_16 fabric of D-Wave Advantage
    n150, _, _ = I.pegasus_edges(150)
    assert 4.5e5 < n150 < 5.5e5                       # "approximately 5e5 variables" at P_150


@pytest.mark.parametrize("m", [2, 3, 6, 16])
def test_pegasus_structure(m):
    """Simple graph, degree at most 15 (12 internal + 2 external + 1 odd),
    every qubit of the fabric with an internal coupler, and the interior at
    the full degree of 15; a K_4 from two odd-coupled pairs that cross."""
    n, u, v = I.pegasus_edges(m)
    assert np.all(u < v) and np.all(v < n)
    key = u * n + v
    assert np.unique(key).shape[0] == key.shape[0]
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    assert deg.max() == 15 if m >= 6 else deg.max() <= 15
    assert deg.min() >= 1
    E = set(zip(u.tolist(), v.tolist()))
    adj = {i: set() for i in range(n)}
    for a, b in E:
        adj[a].add(b)
        adj[b].add(a)
    found = False
    for a, b in E:
        common = adj[a] & adj[b]
        for c, d in itertools.combinations(sorted(common), 2):
            if d in adj[c]:
                found = True
                break
        if found:
            break
    assert found


def test_zephyr_published_sizes():
    n1, rp1, col1 = I.zephyr_csr(1)
    assert n1 == 48                                   # the paper's Z_1 on 48 qubits
    n150 = 4 * 4 * 150 * (2 * 150 + 1)
    assert abs(n150 - 7.2e5) < 0.01 * 7.2e5           # "approximately 7.2e5 variables" at Z_150
    assert I.zephyr_csr(150)[0] == n150
    assert 4 * 4 * 1750 * (2 * 1750 + 1) > 9.8e7      # "more than 9.8e7 variables" at Z_1750
    n12 = I.zephyr_csr(12)[0]
    assert n12 == 4800 > 4580                          # the imperfect Z_12 of Advantage2 has 4580 working qubits


def test_zephyr_z1_holds_k88():
    """The paper: Z_1 embeds K_{8,8} directly. The 8 vertical qubits of the
    middle bundle and the 8 horizontal qubits of the middle bundle are all
    coupled to one another."""
    n, rp, col = I.zephyr_csr(1)
    A = _adjacency(n, rp, col)
    W, t, m = 3, 4, 1

    def idx(o, w, k, j, z):
        return (((o * W + w) * t + k) * 2 + j) * m + z

    V = [idx(0, 1, k, j, 0) for k in range(t) for j in range(2)]
    H = [idx(1, 1, k, j, 0) for k in range(t) for j in range(2)]
    assert all((a, b) in A for a in V for b in H)


@pytest.mark.parametrize("m,t", [(1, 4), (2, 4), (6, 4), (12, 4), (3, 2)])
def test_zephyr_structure(m, t):
    """Symmetric pattern without self-loops, sorted columns, n = 4tm(2m+1),
    degree at most 4t + 4 and exactly that away from the boundary (from
    m = 3 on), and the edge count the definition implies: 16 t^2 m^2
    internal + 2 t (2m + 1)(2m - 1) odd + 4 t (2m + 1)(m - 1) external."""
    n, rp, col = I.zephyr_csr(m, t)
    assert n == 4 * t * m * (2 * m + 1)
    deg = np.diff(rp)
    assert deg.max() <= 4 * t + 4
    if m >= 3:
        assert deg.max() == 4 * t + 4
    rows = np.repeat(np.arange(n), deg)
    assert np.all(rows != col)
    for i in range(0, n, max(1, n // 97)):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0)
    A = _adjacency(n, rp, col)
    assert all((b, a) in A for a, b in A)
    edges = rp[-1] // 2
    assert edges == 4 * t * t * m * m * 4 + 2 * t * (2 * m + 1) * (2 * m - 1) + 4 * t * (2 * m + 1) * (m - 1)


def test_topology_qubos_symmetric_and_seeded():
    """The random QUBOs on both graphs store each coupler's value at both
    positions, are reproducible from the seed and differ between seeds."""
    for make in (lambda s: I.pegasus_qubo(4, seed=s), lambda s: I.zephyr_qubo(3, seed=s)):
        a, b, c = make(0), make(0), make(1)
        assert np.array_equal(a.val, b.val) and np.array_equal(a.lin, b.lin)
        assert not np.array_equal(a.val, c.val)
        rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
        d = dict(zip(zip(rows.tolist(), a.col.tolist()), a.val.tolist()))
        assert all(d[(j, i)] == v for (i, j), v in d.items())
        assert np.all(np.abs(a.val) <= 0.5) and np.all(np.abs(a.lin) <= 1.0)
