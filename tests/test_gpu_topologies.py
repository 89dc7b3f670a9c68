"""Random QUBOs on the annealer topologies the paper benchmarks (Sec.
"Pegasus topology", Sec. "Zephyr topology") through the library: the field,
one fused step and a solve against the FP64 oracle, on the resident and the
streaming kernels, the automatic path choice, and the Zephyr Z_150 (7.2e5
variables) and Z_1750 (9.8e7) instances at full size on sampled rows."""
import numpy as np
import pytest

import oracle as O
from paper_2501_19221_gb300 import instances as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2501_19221_gb300 import binding
    return binding


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


GRAPHS = {"pegasus_p16": lambda: I.pegasus_qubo(16, seed=0), "zephyr_z12": lambda: I.zephyr_qubo(12, seed=0)}


def _make(B, name):
    sp = GRAPHS[name]()
    ctx = B.veloxq_create_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    p = O.problem_from_csr(sp.n, sp.rowptr, sp.col, sp.val.astype(np.float64), sp.lin)
    return sp, ctx, p


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("path", [1, 2])
def test_topology_one_step(B, name, path):
    """One fused step: the field within 1e-5 of |Qoff||S| elementwise and the
    state within 2e-5 of the oracle's FP64 step (the bar of the FP32 paths)."""
    sp, ctx, p = _make(B, name)
    n, R, K, k = sp.n, 64, 100, 40
    sched = B.make_schedule(c0=0.3, dt=0.45, path=path)
    S = I.uniform_state(R, n, -1.0, 1.0, seed=1)
    Y = I.uniform_state(R, n, -0.6, 0.6, seed=2)
    St, Yt, Ft = _cuda(S), _cuda(Y), torch.empty(R, n, device="cuda")
    B.veloxq_steps_dev(ctx, R, k, 1, K, sched, St, Yt, Ft)
    torch.cuda.synchronize()
    a = O.schedule(K, [0.0, 1.0])
    S1, Y1, F = O.bsb_step(p, S, Y, a[k], np.float32(0.45), 1.0, np.float32(0.3))
    assert np.all(np.abs(Ft.cpu().numpy() - F) <= 1e-5 * O.abs_field(p, S.astype(np.float64)) + 1e-30)
    Sg, Yg = St.cpu().numpy(), Yt.cpu().numpy()
    bad = (np.abs(Sg - S1) > 2e-5) | (np.abs(Yg - Y1) > 2e-5)
    # the only admissible disagreement: one side at a wall the other is within 1e-4 of
    near = np.minimum(np.abs(np.abs(Sg) - 1.0), np.abs(np.abs(S1) - 1.0)) <= 1e-4
    assert np.all((near & (np.sign(Sg) == np.sign(S1)))[bad])


@pytest.mark.parametrize("name", list(GRAPHS))
def test_topology_solve(B, name):
    """1024 replicas (the paper's 2^10 samples per run): the returned energy is
    the oracle's energy of the returned vector within its FP64 bound, the best
    of the per-replica energies, and far below random vectors."""
    sp, ctx, p = _make(B, name)
    out = B.veloxq_solve(ctx, 1024, 1000, B.make_schedule(readout_every=50), seed=3)
    Ex = O.energy(p, out["x"])[0]
    tol = (p.nnz + p.n) * 2.0 ** -52 * (np.abs(p.ev).sum() + np.abs(p.c).sum())
    assert abs(Ex - out["E"]) <= tol
    assert out["E"] == np.min(out["E_per_replica"])
    assert out["E"] < np.min(O.energy(p, I.random_binary(256, sp.n, seed=4)))


def test_zephyr_z150_full_size(B):
    """Z_150, the paper's largest Zephyr instance with a quality claim (7.2e5
    variables), on the streaming kernel: the field of sampled rows against the
    oracle's field of the couplers touching them, and a solve whose energy the
    energy entry point reproduces."""
    sp = I.zephyr_qubo(150, seed=0)
    n, R = sp.n, 64
    ctx = B.veloxq_create_csr(n, sp.rowptr, sp.col, sp.val, sp.lin)
    rows = np.sort(np.random.default_rng(5).choice(n, size=96, replace=False))
    rp = sp.rowptr
    ri = np.concatenate([np.full(rp[r + 1] - rp[r], r, dtype=np.int64) for r in rows])
    cj = np.concatenate([sp.col[rp[r]:rp[r + 1]] for r in rows]).astype(np.int64)
    qv = np.concatenate([sp.val[rp[r]:rp[r + 1]] for r in rows]).astype(np.float64)
    # every coupler touching a sampled row once, stored at both positions as in
    # the instance (the oracle forms Qs = (Q + Q^T)/2 from them)
    pi, pj = np.minimum(ri, cj), np.maximum(ri, cj)
    _, first = np.unique(pi * n + pj, return_index=True)
    pi, pj, qv = pi[first], pj[first], qv[first]
    ps = O.Problem(n, np.concatenate([pi, pj]), np.concatenate([pj, pi]), np.concatenate([qv, qv]), np.zeros(n))
    S = I.uniform_state(R, n, seed=6)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, _cuda(S), F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()[:, rows].astype(np.float64)
    Sd = S.astype(np.float64)
    ref = O.field(ps, Sd)[:, rows]
    sc = O.abs_field(ps, Sd)[:, rows]
    assert np.all(np.abs(Fg - ref) <= 1e-5 * sc + 1e-30)
    out = B.veloxq_solve(ctx, R, 200, B.make_schedule(readout_every=0), seed=1)
    assert B.veloxq_last_timing(ctx).path == 2
    again = B.veloxq_energy(ctx, out["x"][None])
    assert abs(again["E"][0] - out["E"]) <= 1e-9 * max(1.0, abs(out["E"]))


def test_auto_path_by_where_couplings_fit(B):
    """The automatic path: the resident kernel when the couplings fit in
    shared memory (Chimera C16, int8 in packed words), the streaming step
    when they do not (float couplings of Pegasus P_16 and Zephyr Z_12, which
    the resident kernel would re-read from L2 every step)."""
    sp = I.chimera_ising(16, 16, 4, seed=0)
    ctx = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    B.veloxq_solve(ctx, 1024, 10, B.make_schedule(), seed=1)
    assert B.veloxq_last_timing(ctx).path == 1
    for name in GRAPHS:
        sp, ctx, _ = _make(B, name)
        B.veloxq_solve(ctx, 1024, 10, B.make_schedule(), seed=1)
        assert B.veloxq_last_timing(ctx).path == 2


def test_zephyr_z1750_full_size(B):
    """Z_1750, the paper's largest instance (9.8e7 variables, 1.96e9 CSR
    entries), with 2 replicas as the bench runs it: the field of sampled rows
    against the oracle's field of the couplers touching them, and a short
    solve whose energy the energy entry point reproduces."""
    sp = I.zephyr_qubo(1750, seed=0)
    n, R = sp.n, 2
    assert n > 9.8e7
    ctx = B.veloxq_create_csr(n, sp.rowptr, sp.col, sp.val, sp.lin)
    rows = np.sort(np.random.default_rng(7).choice(n, size=48, replace=False))
    rp = sp.rowptr
    ri = np.concatenate([np.full(rp[r + 1] - rp[r], r, dtype=np.int64) for r in rows])
    cj = np.concatenate([sp.col[rp[r]:rp[r + 1]] for r in rows]).astype(np.int64)
    qv = np.concatenate([sp.val[rp[r]:rp[r + 1]] for r in rows]).astype(np.float64)
    pi, pj = np.minimum(ri, cj), np.maximum(ri, cj)
    _, first = np.unique(pi * n + pj, return_index=True)
    pi, pj, qv = pi[first], pj[first], qv[first]
    ps = O.Problem(n, np.concatenate([pi, pj]), np.concatenate([pj, pi]), np.concatenate([qv, qv]), np.zeros(n))
    S = I.uniform_state(R, n, seed=8)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, _cuda(S), F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()[:, rows].astype(np.float64)
    Sd = S.astype(np.float64)
    ref = O.field(ps, Sd)[:, rows]
    sc = O.abs_field(ps, Sd)[:, rows]
    assert np.all(np.abs(Fg - ref) <= 1e-5 * sc + 1e-30)
    del S, Sd, F
    out = B.veloxq_solve(ctx, R, 20, B.make_schedule(readout_every=0), seed=1)
    assert B.veloxq_last_timing(ctx).path == 2
    again = B.veloxq_energy(ctx, out["x"][None])
    assert abs(again["E"][0] - out["E"]) <= 1e-9 * max(1.0, abs(out["E"]))
