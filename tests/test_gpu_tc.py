"""Tensor-core (tcgen05) dense local field, BF16 and FP8 E4M3 with per-row
scales, FP32 accumulation, against the FP64 oracle.

Bounds from the operand rounding. BF16 rounds each operand to 8 significant
bits (relative error <= 2^-9). E4M3 keeps 4 (<= 2^-4 for normal values, an
absolute 2^-10 of the scale below 2^-6). Qoff is one E4M3 term of Qoff_ij /
q_i, q_i = amax_i / 448. S is v = 448 s in two E4M3 terms for FP8 (hi =
e4m3(v), lo = e4m3(v - hi): relative 2^-8 plus the lo term's absolute
2^-10 / 448), or in one term for FP8_ONE_TERM (2^-4). With uQ, uS the
relative and aQ_i, aS the absolute parts,
    |dF_ir| <= (uQ + uS + uQ uS) (|Qoff| |S|)_ir
               + aQ_i (1 + uS) sum_j |S_jr| + aS (1 + uQ) sum_j |Qoff_ij|
               + FP32 accumulation.
The normwise bar of the mixed-precision field is 3e-2; BF16 and FP8 (two
terms) meet it, FP8_ONE_TERM does not (both operands rounded to 4 bits: about
3.7%) and its tests hold it to its own estimate instead.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2501_19221_gb300 import instances as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BF16, FP8, FP8_ONE_TERM = 1, 2, 3
# relative rounding of (Qoff, S) per precision
U = {BF16: (2.0 ** -9, 2.0 ** -9), FP8: (2.0 ** -4, 2.0 ** -8 + 2.0 ** -23), FP8_ONE_TERM: (2.0 ** -4, 2.0 ** -4)}
# normwise bars: the 3e-2 of the mixed-precision field for BF16 and FP8; the
# one-term form's own estimate (sqrt(2) x 2.7%) with margin
NORM_BAR = {BF16: 1e-2, FP8: 3e-2, FP8_ONE_TERM: 4.5e-2}


def _report(key, value):
    """Record a measured error when VELOXQ_REPORT_DIR names a folder."""
    d = os.environ.get("VELOXQ_REPORT_DIR")
    if not d:
        return
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, "tc_errors.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    data[key] = float(value)
    json.dump(data, open(path, "w"), indent=1, sort_keys=True)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2501_19221_gb300 import binding
    return binding


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _qoff_rows(Q, rows):
    """Rows of Qoff = offdiag((Q + Q^T)/2) for the given row indices."""
    Qd = np.asarray(Q, dtype=np.float64)
    Qs = 0.5 * (Qd[rows, :] + Qd[:, rows].T)
    Qs[np.arange(len(rows)), rows] = 0.0
    return Qs


def _elem_bound(prec, scale, Qoff_rows=None, S=None):
    """Elementwise bound on |F_gpu - F| ([R][rows]) from the module docstring;
    scale = (|Qoff| |S|) for the same entries."""
    uq, us = U[prec]
    b = (uq + us + uq * us) * scale + 1e-6 * scale
    if prec != BF16:
        aq = np.abs(Qoff_rows).max(axis=1) / 448.0 * 2.0 ** -10          # per row
        a_s = 2.0 ** -10 / 448.0                                          # S's absolute part
        b = b + (1 + us) * aq[None, :] * np.abs(S).sum(axis=1)[:, None]
        b = b + (1 + uq) * a_s * np.abs(Qoff_rows).sum(axis=1)[None, :]
    return b


PRECS = [BF16, FP8, FP8_ONE_TERM]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,R", [(300, 1), (300, 64), (300, 300), (20, 7), (129, 257)])
def test_tc_field_matches_oracle(B, prec, n, R):
    Q, _ = I.sk_qubo(n, seed=3)
    c = np.zeros(n)
    ctx = B.veloxq_create_dense(Q, c)
    S = I.uniform_state(R, n, seed=5)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, prec, _cuda(S), F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy().astype(np.float64)
    p = O.problem_from_dense(Q.astype(np.float64))
    ref = O.field(p, S.astype(np.float64))
    scale = O.abs_field(p, S.astype(np.float64))
    bound = _elem_bound(prec, scale, _qoff_rows(Q, np.arange(n)), S)
    assert np.all(np.abs(Fg - ref) <= bound + 1e-30), np.max(np.abs(Fg - ref) / (scale + 1e-30))
    err = np.linalg.norm(Fg - ref) / np.linalg.norm(ref)
    assert err <= NORM_BAR[prec], err


@pytest.mark.parametrize("prec", PRECS)
def test_tc_field_full_size_sampled_rows(B, prec):
    """n = 8192, 1024 replicas (the dense benchmark shape), sampled rows."""
    n, R = 8192, 1024
    Q, c = I.sk_qubo(n, seed=0)
    ctx = B.veloxq_create_dense(Q, c)
    S = I.uniform_state(R, n, seed=7)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, prec, _cuda(S), F)
    torch.cuda.synchronize()
    rows = np.random.default_rng(1).choice(n, size=96, replace=False)
    Fg = F[:, torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    ref = O.field_dense_rows(Q, S, rows)
    scale = O.abs_field_dense_rows(Q, S, rows)
    assert np.all(np.abs(Fg - ref) <= _elem_bound(prec, scale, _qoff_rows(Q, rows), S))
    err = np.linalg.norm(Fg - ref) / np.linalg.norm(ref)
    _report(f"field_n8192_R1024_prec{prec}", err)
    assert err <= NORM_BAR[prec], err
    # FP32 CUDA-core form on the same sample, for the report
    B.veloxq_field_dev(ctx, R, 0, _cuda(S), F)
    torch.cuda.synchronize()
    F32 = F[:, torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    e32 = np.linalg.norm(F32 - ref) / np.linalg.norm(ref)
    _report("field_n8192_R1024_fp32", e32)
    assert e32 <= 1e-5


@pytest.mark.parametrize("prec", PRECS)
def test_tc_step_fuses_the_update(B, prec):
    """One fused step: s, y follow the FP32 update of the oracle up to the
    propagated field error (dy = dt c0 dF / 2, ds = dt a0 dy)."""
    n, R, K, k = 300, 64, 100, 40
    Q, c = I.sk_qubo(n, seed=4)
    c = np.random.default_rng(1).normal(size=n) * 0.05
    ctx = B.veloxq_create_dense(Q, c)
    dt, c0 = np.float32(0.5), np.float32(0.7)
    sched = B.make_schedule(dt=float(dt), c0=float(c0), prec=prec)
    S = I.uniform_state(R, n, -1, 1, seed=2)
    Y = I.uniform_state(R, n, -0.4, 0.4, seed=3)
    St, Yt, Ft = _cuda(S), _cuda(Y), torch.empty(R, n, device="cuda")
    B.veloxq_steps_dev(ctx, R, k, 1, K, sched, St, Yt, Ft)
    torch.cuda.synchronize()
    p = O.problem_from_dense(Q.astype(np.float64), c)
    a = O.schedule(K, [0.0, 1.0])
    S1, Y1, F = O.bsb_step(p, S, Y, a[k], float(dt), 1.0, float(c0))
    dF = _elem_bound(prec, O.abs_field(p, S.astype(np.float64)), _qoff_rows(Q, np.arange(n)), S)
    dy = float(dt) * float(c0) * 0.5 * dF + 2e-5
    ds = float(dt) * dy + 2e-5
    Sg, Yg = St.cpu().numpy(), Yt.cpu().numpy()
    wall = (np.abs(Sg) == 1.0) | (np.abs(S1) == 1.0)
    free = ~wall
    assert np.all(np.abs(Yg - Y1)[free] <= dy[free])
    assert np.all(np.abs(Sg - S1)[free] <= ds[free])
    # at a wall both sides agree on the sign, or the other side is within ds of it
    assert np.all((np.sign(Sg) == np.sign(S1))[wall] | (np.abs(np.abs(S1) - 1) <= ds)[wall])


def _first_50(B, prec, teacher_forced):
    """Errors of the field of each of the first 50 steps from the same Philox
    start: against the FP64 field of the GPU's own state before the step
    (teacher-forced), or against the FP64 trajectory (free-running)."""
    n, R, K, seed = 512, 64, 1000, 3
    Q, c = I.sk_qubo(n, seed=5)
    ctx = B.veloxq_create_dense(Q, c)
    p = O.problem_from_dense(Q.astype(np.float64), c)
    c0 = float(np.float32(2.0 / O.spectral_radius(p)))
    sched = B.make_schedule(c0=c0, prec=prec)
    St = torch.empty(R, n, device="cuda")
    Yt = torch.empty(R, n, device="cuda")
    Ft = torch.empty(R, n, device="cuda")
    B.veloxq_init_state_dev(ctx, R, seed, 0.1, St, Yt)
    S0, Y0 = O.init_state(n, R, seed, 0.1)
    ref = None if teacher_forced else O.bsb_run(p, R, 50, 0.5, 1.0, c0, [0.0, 49.0 / (K - 1)], 0, S0, Y0, n_snap=50)
    errs = []
    for k in range(50):
        Sk = St.cpu().numpy().astype(np.float64)
        B.veloxq_steps_dev(ctx, R, k, 1, K, sched, St, Yt, Ft)
        torch.cuda.synchronize()
        Fr = O.field(p, Sk) if teacher_forced else ref["F_snap"][k]
        errs.append(np.linalg.norm(Ft.cpu().numpy() - Fr) / np.linalg.norm(Fr))
    return errs


@pytest.mark.parametrize("prec", PRECS)
def test_tc_first_50_steps_teacher_forced(B, prec):
    """The mixed-precision bar, 3e-2 normwise on each of the first 50 steps'
    fields, for BF16 and FP8 (two S terms); the one-term form against its own
    estimate."""
    errs = _first_50(B, prec, True)
    _report(f"first_50_steps_teacher_forced_prec{prec}", max(errs))
    bar = 3e-2 if prec in (BF16, FP8) else NORM_BAR[FP8_ONE_TERM]
    assert max(errs) <= bar, (max(errs), errs[:5])


@pytest.mark.parametrize("prec", PRECS)
def test_tc_first_50_steps_free_running(B, prec):
    """Free-running from the same start: the field error then also carries the
    trajectory's divergence from the FP64 one (every step's rounding is fed
    back through the dynamics), which the FP32 form holds to 1e-5 elsewhere.
    Recorded; held to twice the teacher-forced bar so that a broken step
    still fails."""
    errs = _first_50(B, prec, False)
    _report(f"first_50_steps_free_running_prec{prec}", max(errs))
    bar = 2 * (3e-2 if prec in (BF16, FP8) else NORM_BAR[FP8_ONE_TERM])
    assert max(errs) <= bar, (max(errs), errs[:5])


@pytest.mark.parametrize("prec", PRECS)
def test_tc_solve_outputs_consistent(B, prec):
    n = 300
    Q, c = I.sk_qubo(n, seed=6)
    ctx = B.veloxq_create_dense(Q, c)
    p = O.problem_from_dense(Q.astype(np.float64), c)
    out = B.veloxq_solve(ctx, 96, 400, B.make_schedule(prec=prec, readout_every=40), seed=1)
    Ex = O.energy(p, out["x"])[0]
    tol = (p.nnz + n) * 2.0 ** -52 * np.sum(np.abs(Q)) + 1e-12
    assert abs(Ex - out["E"]) <= tol
    assert out["E"] == np.min(out["E_per_replica"])
    # it actually optimises: far below random vectors
    assert out["E"] < np.min(O.energy(p, I.random_binary(256, n, seed=2)))
    t = B.veloxq_last_timing(ctx)
    # one launch per run of steps up to a readout: 400 steps, a readout every 40
    assert t.path == 3 and t.main_launches == 10


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,R", [(2048, 256), (3000, 300)])
def test_tc_field_mid_sizes(B, prec, n, R):
    """Mid-size shapes (8 and 24 pair tiles, ragged row and replica tiles):
    the field matches the oracle within the rounding bound on sampled rows
    (tile boundaries included), and two runs give the same bits."""
    Q, _ = I.sk_qubo(n, seed=11)
    ctx = B.veloxq_create_dense(Q, np.zeros(n))
    S = I.uniform_state(R, n, seed=12)
    F = torch.empty(R, n, device="cuda")
    F2 = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, prec, _cuda(S), F)
    B.veloxq_field_dev(ctx, R, prec, _cuda(S), F2)
    torch.cuda.synchronize()
    assert torch.equal(F, F2)
    rows = np.sort(np.random.default_rng(2).choice(n, size=128, replace=False))
    rows = np.unique(np.concatenate([rows, [0, 255, 256, n - 1]]))
    Fg = F[:, torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    ref = O.field_dense_rows(Q, S, rows)
    scale = O.abs_field_dense_rows(Q, S, rows)
    assert np.all(np.abs(Fg - ref) <= _elem_bound(prec, scale, _qoff_rows(Q, rows), S))
    assert np.linalg.norm(Fg - ref) / np.linalg.norm(ref) <= NORM_BAR[prec]


@pytest.mark.parametrize("method", [0, 2])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,R", [(3000, 1024), (1500, 768), (700, 96)])
def test_tc_run_equals_single_steps(B, prec, method, n, R):
    """Several steps in one launch (the solve's form: tiles of consecutive
    steps overlap, each waiting for the column block of the state it reads;
    column blocks in groups of two for BF16 and one-term FP8, the last group
    of R = 768 a single block) give bit for bit the state and last field of
    the same steps launched one at a time: the per-tile arithmetic is the
    same, only the schedule differs."""
    if method == 2 and prec == FP8_ONE_TERM:
        pytest.skip("Parallel Annealing's FP8 forms are the same run")
    Q, c = I.sk_qubo(n, seed=13)
    ctx = B.veloxq_create_dense(Q, c)
    sched = B.make_schedule(prec=prec, method=method)
    K, k0, steps = 100, 7, 20
    runs = []
    for one_launch in (True, False):
        St = torch.empty(R, n, device="cuda")
        Yt = torch.empty(R, n, device="cuda")
        Ft = torch.empty(R, n, device="cuda")
        B.veloxq_init_state_dev(ctx, R, 5, 0.3, St, Yt)
        if one_launch:
            B.veloxq_steps_dev(ctx, R, k0, steps, K, sched, St, Yt, Ft)
        else:
            for k in range(k0, k0 + steps):
                B.veloxq_steps_dev(ctx, R, k, 1, K, sched, St, Yt, Ft)
        torch.cuda.synchronize()
        runs.append((St, Yt, Ft))
    for a, b in zip(*runs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
def test_tc_steps_deterministic(B, prec):
    """Ten fused steps in one launch at the dense benchmark's shape (n = 8192,
    1024 replicas: 128 pair tiles per step over the pairs): two runs from the
    same state give the same bits."""
    n, R = 8192, 1024
    Q, c = I.sk_qubo(n, seed=0)
    ctx = B.veloxq_create_dense(Q, c)
    sched = B.make_schedule(prec=prec)
    outs = []
    for _ in range(2):
        St = torch.empty(R, n, device="cuda")
        Yt = torch.empty(R, n, device="cuda")
        B.veloxq_init_state_dev(ctx, R, 3, 0.1, St, Yt)
        B.veloxq_steps_dev(ctx, R, 0, 10, 200, sched, St, Yt, None)
        torch.cuda.synchronize()
        outs.append((St, Yt))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
