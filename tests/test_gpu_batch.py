"""The persistent batched tensor-core kernel (veloxq_solve_batch with dense
BF16 contexts): one-step parity of every instance against the FP64 oracle,
exact outputs, and solution quality on Wishart planted instances."""
import numpy as np
import pytest

import oracle as O
from paper_2501_19221_gb300 import instances as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -9       # BF16 operand rounding
# relative rounding of (Qoff, S) per field precision: BF16; FP8 with S in two
# E4M3 terms; FP8 with one term (E4M3 keeps 4 significant bits)
UQS = {1: (2.0 ** -9, 2.0 ** -9), 2: (2.0 ** -4, 2.0 ** -8 + 2.0 ** -23), 3: (2.0 ** -4, 2.0 ** -4)}


def _field_bound(prec, Q, S, rows=None):
    """Elementwise bound on the field error of one batched step ([R][rows]):
    (uQ + uS + uQ uS)(|Qoff||S|) plus, for E4M3, the absolute error of its
    subnormal range (2^-10 of the row scale for Qoff, 2^-10/448 for S)."""
    rows = np.arange(Q.shape[0]) if rows is None else np.asarray(rows)
    uq, us = UQS[prec]
    Qd = np.asarray(Q, dtype=np.float64)
    Qr = 0.5 * (Qd[rows, :] + Qd[:, rows].T)
    Qr[np.arange(len(rows)), rows] = 0.0
    b = (uq + us + uq * us) * (np.abs(S).astype(np.float64) @ np.abs(Qr).T) + 1e-6
    if prec != 1:
        aq = np.abs(Qr).max(axis=1) / 448.0 * 2.0 ** -10
        b = b + (1 + us) * aq[None, :] * np.abs(S).sum(axis=1)[:, None]
        b = b + (1 + uq) * 2.0 ** -10 / 448.0 * np.abs(Qr).sum(axis=1)[None, :]
    return b


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2501_19221_gb300 import binding
    return binding


def _sk(n, seed):
    Q, _ = I.sk_qubo(n, seed=seed)
    c = np.random.default_rng(seed).normal(size=n) * 0.05
    return Q, c


@pytest.mark.parametrize("prec,R", [(1, 16), (1, 64), (1, 128), (2, 16), (2, 64), (2, 128), (3, 64)])
def test_batch_one_step_parity(B, prec, R):
    """K = 1 from the Philox start: every instance's state equals the oracle's
    FP32-input FP64 step up to the field bound of the precision (BF16; FP8
    with S in two E4M3 terms; FP8 with one) propagated through the update."""
    sizes = [20, 100, 129, 300, 511, 640, 128, 64]
    insts = [_sk(n, 10 + i) for i, n in enumerate(sizes)]
    ctxs = [B.veloxq_create_dense(Q, c) for Q, c in insts]
    dt, c0 = np.float32(0.5), np.float32(0.3)
    sched = B.make_schedule(prec=prec, readout_every=0, c0=float(c0), dt=float(dt))
    out = B.veloxq_solve_batch(ctxs, R, 1, sched, seed=4)
    assert B.veloxq_last_timing(ctxs[0]).main_launches == 1
    for (Q, c), ctx in zip(insts, ctxs):
        n = Q.shape[0]
        S = torch.empty(R, n, device="cuda")
        Y = torch.empty(R, n, device="cuda")
        B.veloxq_batch_state_dev(ctx, R, S, Y)
        torch.cuda.synchronize()
        p = O.problem_from_dense(Q.astype(np.float64), c)
        S0, Y0 = O.init_state(n, R, 4, 0.1)
        ref = O.bsb_run(p, R, 1, float(dt), 1.0, float(c0), [0.0, 1.0], 0, S0, Y0)
        dF = _field_bound(prec, Q, S0)
        dy = float(dt) * float(c0) * 0.5 * dF + 2e-6
        ds = float(dt) * dy + 2e-6
        assert np.all(np.abs(Y.cpu().numpy() - ref["Y"]) <= dy)
        assert np.all(np.abs(S.cpu().numpy() - ref["S"]) <= ds)
    assert len(out["E"]) == len(sizes)


@pytest.mark.parametrize("prec,method", [(1, 0), (2, 0), (3, 0), (2, 2)])
def test_batch_outputs_exact_and_consistent(B, prec, method):
    sizes = [37, 200, 150, 480, 99]
    insts = [_sk(n, 30 + i) for i, n in enumerate(sizes)]
    ctxs = [B.veloxq_create_dense(Q, c) for Q, c in insts]
    out = B.veloxq_solve_batch(ctxs, 64, 200, B.make_schedule(prec=prec, readout_every=0, method=method), seed=2)
    t = B.veloxq_last_timing(ctxs[0])
    assert t.main_launches == 1
    for (Q, c), x, E in zip(insts, out["x"], out["E"]):
        p = O.problem_from_dense(Q.astype(np.float64), c)
        Ex = O.energy(p, x)[0]
        tol = (p.nnz + p.n) * 2.0 ** -52 * (np.sum(np.abs(Q)) + np.sum(np.abs(c)))
        assert abs(Ex - E) <= tol
        assert E < np.min(O.energy(p, I.random_binary(128, p.n, seed=1)))


def test_batch_wishart_quality_matches_plain_fp32(B):
    """Wishart planted instances (Sec. Wishart ensemble), alpha = 0.75: the
    batched BF16 solve never goes below the planted ground energy, and its
    mean relative gap to it is within 0.02 of the plain FP32 form's gap on the
    same instances, schedule and seed (the dynamics, not the precision, set
    the quality)."""
    sizes = [100, 160, 240, 320, 128, 200]
    ctxs, E0s = [], []
    for i, n in enumerate(sizes):
        w = I.wishart_ising(n, 0.75, seed=50 + i)
        ctxs.append(B.veloxq_create_ising_dense(-w["J"], None))
        E0s.append(0.5 * w["Jt_diag"].sum())
    out = B.veloxq_solve_batch(ctxs, 64, 1000, B.make_schedule(prec=1, readout_every=0), seed=1)
    gaps_b, gaps_f = [], []
    for ctx, E, E0 in zip(ctxs, out["E"], E0s):
        off = ctx.info.ising_offset
        H = 2 * E + off
        assert H >= E0 - 1e-6 * abs(E0)
        gaps_b.append((H - E0) / abs(E0))
        f = B.veloxq_solve(ctx, 64, 1000, B.make_schedule(readout_every=0, path=3), seed=1)
        gaps_f.append((2 * f["E"] + off - E0) / abs(E0))
    assert np.mean(gaps_b) <= np.mean(gaps_f) + 0.02, (gaps_b, gaps_f)


def test_batch_falls_back_when_not_supported(B):
    """Other schedules (readouts during the run, FP32) solve each context in turn."""
    sizes = [40, 70]
    insts = [_sk(n, 60 + i) for i, n in enumerate(sizes)]
    ctxs = [B.veloxq_create_dense(Q, c) for Q, c in insts]
    a = B.veloxq_solve_batch(ctxs, 32, 100, B.make_schedule(readout_every=10), seed=3)
    for ctx, E in zip(ctxs, a["E"]):
        single = B.veloxq_solve(ctx, 32, 100, B.make_schedule(readout_every=10), seed=3)
        assert single["E"] == E


def _sym_normal(n, seed):
    """A symmetric dense instance with N(0, 1/n) couplings, zero diagonal
    (float32; the SK recipe, cheap enough for hundreds of instances)."""
    g = np.random.default_rng(seed).standard_normal((n, n), dtype=np.float32)
    Q = (g + g.T) * np.float32(1.0 / np.sqrt(2.0 * n))
    np.fill_diagonal(Q, 0.0)
    return Q


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_config4_shapes_one_step(B, prec):
    """The batched-instance workload's own shapes in ONE launch: 512
    instances with n drawn uniformly from [100, 2000] (the Wishart batch's
    sizes), 64 replicas, one step from the Philox start. For every instance,
    sampled rows (the first and last of each 128-row tile boundary pair and a
    few random ones) of S and Y match the oracle's FP64 step (field of the
    sampled rows by a library matmul, bias of those rows, the oracle's update)
    within the BF16 field bound propagated through the update."""
    R, dt, c0 = 64, np.float32(0.5), np.float32(0.3)
    sizes = I.wishart_sizes(512, 100, 2000, seed=0)
    ctxs, refs = [], []
    rng = np.random.default_rng(123)
    for m, n in enumerate(sizes):
        n = int(n)
        Q = _sym_normal(n, 5000 + m)
        c = np.zeros(n)
        ctxs.append(B.veloxq_create_dense(Q, c))
        rows = {0, n - 1, min(127, n - 1), min(128, n - 1)}
        rows |= set(rng.choice(n, size=4, replace=False).tolist())
        rows = np.array(sorted(rows))
        S0, Y0 = O.init_state(n, R, 4, 0.1)
        F = O.field_dense_rows(Q, S0, rows)
        b = O.bias_dense_rows(Q, c, rows)
        S1, Y1 = O.update("bsb", F, b, 0.0, float(dt), 1.0, float(c0), S0[:, rows], Y0[:, rows])
        dF = _field_bound(prec, Q, S0, rows)
        refs.append((rows, S1, Y1, dF))
    sched = B.make_schedule(prec=prec, readout_every=0, c0=float(c0), dt=float(dt))
    B.veloxq_solve_batch(ctxs, R, 1, sched, seed=4, want_x=False)
    assert B.veloxq_last_timing(ctxs[0]).main_launches == 1
    for ctx, (rows, S1, Y1, dF) in zip(ctxs, refs):
        n = ctx.info.n
        S = torch.empty(R, n, device="cuda")
        Y = torch.empty(R, n, device="cuda")
        B.veloxq_batch_state_dev(ctx, R, S, Y)
        torch.cuda.synchronize()
        ti = torch.as_tensor(rows, device="cuda")
        Sg, Yg = S[:, ti].cpu().numpy(), Y[:, ti].cpu().numpy()
        dy = float(dt) * float(c0) * 0.5 * dF + 2e-6
        ds = float(dt) * dy + 2e-6
        assert np.all(np.abs(Yg - Y1) <= dy), n
        assert np.all(np.abs(Sg - S1) <= ds), n
    for ctx in ctxs:
        ctx.destroy()


def test_two_batches_on_two_streams(B):
    """Two batches headed by different contexts, on two streams and from two
    host threads at once, give exactly the results each gives alone: the
    batched launch's scratch belongs to the batch's first context."""
    import threading
    sets = [[_sk(n, 70 + 10 * k + i) for i, n in enumerate(sizes)]
            for k, sizes in enumerate(([90, 300, 210, 64], [150, 37, 400]))]
    ctx_sets = [[B.veloxq_create_dense(Q, c) for Q, c in s] for s in sets]
    sched = B.make_schedule(prec=1, readout_every=0)
    alone = [B.veloxq_solve_batch(cs, 32, 150, sched, seed=5 + k) for k, cs in enumerate(ctx_sets)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for cs, st in zip(ctx_sets, streams):
        for cx in cs:
            B.veloxq_set_stream(cx, st.cuda_stream)
    got, errs = [None, None], []

    def run(k):
        try:
            got[k] = B.veloxq_solve_batch(ctx_sets[k], 32, 150, sched, seed=5 + k)
        except Exception as e:                      # reported below
            errs.append(e)

    th = [threading.Thread(target=run, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    for a, g in zip(alone, got):
        assert np.array_equal(a["E"], g["E"])
        for xa, xg in zip(a["x"], g["x"]):
            assert np.array_equal(xa, xg)
    for cs in ctx_sets:
        for cx in cs:
            cx.destroy()


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_forms_agree(B, prec, monkeypatch):
    """Every form of the launch the autotuner chooses from (4 or 6 pipeline
    stages; an instance's 64 replicas in one work item or in groups of 32 or
    16 on separate CTAs) gives the same final states and energies: the
    replicas are independent and each keeps its own arithmetic."""
    sizes = [150, 77, 300, 129, 512]
    insts = [_sk(n, 90 + i) for i, n in enumerate(sizes)]
    ctxs = [B.veloxq_create_dense(Q, c) for Q, c in insts]
    sched = B.make_schedule(prec=prec, readout_every=0)
    results = {}
    for form in ("6 64", "4 64", "6 32", "4 16"):
        monkeypatch.setenv("VELOXQ_BATCH_FORM", form)
        out = B.veloxq_solve_batch(ctxs, 64, 60, sched, seed=8)
        t = B.veloxq_last_timing(ctxs[0])
        assert (t.batch_stages, t.batch_group) == tuple(int(v) for v in form.split())
        states = []
        for ctx in ctxs:
            n = ctx.info.n
            S = torch.empty(64, n, device="cuda")
            Y = torch.empty(64, n, device="cuda")
            B.veloxq_batch_state_dev(ctx, 64, S, Y)
            torch.cuda.synchronize()
            states.append((S.cpu().numpy(), Y.cpu().numpy()))
        results[form] = (out["E"], states)
    E0, st0 = results["6 64"]
    for form, (E, st) in results.items():
        assert np.array_equal(E, E0), form
        for (S, Y), (S0, Y0) in zip(st, st0):
            assert np.array_equal(S, S0) and np.array_equal(Y, Y0), form
    monkeypatch.setenv("VELOXQ_BATCH_FORM", "5 64")
    with pytest.raises(B.VeloxqError, match="VELOXQ_BATCH_FORM"):
        B.veloxq_solve_batch(ctxs, 64, 2, sched, seed=8)


def test_batch_tune_cache_file(B, tmp_path, monkeypatch):
    """The autotuner keeps what it picked in the file VELOXQ_TUNE_CACHE names,
    one "key=stages group" line per kind of batch, and the launch runs in that
    form."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("VELOXQ_TUNE_CACHE", str(path))
    monkeypatch.delenv("VELOXQ_BATCH_FORM", raising=False)
    sizes = [211, 97, 333]                      # a kind of batch no other test uses
    ctxs = [B.veloxq_create_dense(*_sk(n, 120 + i)) for i, n in enumerate(sizes)]
    B.veloxq_solve_batch(ctxs, 48, 20, B.make_schedule(prec=1, readout_every=0), seed=1)
    t = B.veloxq_last_timing(ctxs[0])
    lines = [ln for ln in path.read_text().splitlines() if ln.startswith("batch|")]
    assert len(lines) == 1 and "|R48|" in lines[0]
    st, grp = (int(v) for v in lines[0].split("=")[1].split())
    assert (st, grp) == (t.batch_stages, t.batch_group) and st in (4, 6) and 48 % grp == 0


def test_batch_graph_replays_with_new_seeds(B, monkeypatch):
    """The captured batch solve is replayed for a new seed: seeds 5, 6, 5 in a
    row give two different results and the first one again, bit for bit,
    each equal to an uncaptured run (a fresh batch of the same instances)."""
    monkeypatch.delenv("VELOXQ_BATCH_FORM", raising=False)
    sizes = [120, 260, 64, 333]
    insts = [_sk(n, 140 + i) for i, n in enumerate(sizes)]
    ctxs = [B.veloxq_create_dense(Q, c) for Q, c in insts]
    sched = B.make_schedule(prec=1, readout_every=0)
    runs = [B.veloxq_solve_batch(ctxs, 32, 80, sched, seed=s) for s in (5, 6, 5)]
    assert np.array_equal(runs[0]["E"], runs[2]["E"])
    assert all(np.array_equal(a, b) for a, b in zip(runs[0]["x"], runs[2]["x"]))
    assert not np.array_equal(runs[0]["E"], runs[1]["E"])
    t = B.veloxq_last_timing(ctxs[0])
    assert t.main_launches == 1 and t.launches <= 4
    fresh = [B.veloxq_create_dense(Q, c) for Q, c in insts]
    ref = B.veloxq_solve_batch(fresh, 32, 80, sched, seed=6)
    assert np.array_equal(ref["E"], runs[1]["E"])
