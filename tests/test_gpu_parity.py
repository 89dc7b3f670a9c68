"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs. Tolerances follow the arithmetic:

* integer energies: bit-exact int64;
* real energies: |dE| <= (nnz + n) 2^-52 sum|terms| (FP64 summation of the
  oracle; the library's fixed-point sums are exact to 2^-S);
* FP32 local field: |dF_ir| <= 1e-5 (|Qoff| |S|)_ir and normwise <= 1e-5;
* one FP32 update step: |ds|, |dy| <= 2e-5 absolute, except where one side hit
  a wall (s = +-1, y = 0) and the other is within 1e-4 of it.
"""
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


# ----------------------------------------------------------------- instances
def inst_dense_int20(B):
    Q, c = I.dense_int_qubo(20, seed=0)
    return B.veloxq_create_dense(Q, c), O.problem_from_dense(Q, c)


def inst_dense_int_nonsym(B):
    rng = np.random.default_rng(11)
    n = 70
    Q = rng.integers(-9, 10, size=(n, n)).astype(np.int32)
    c = rng.integers(-4, 5, size=n).astype(np.float64)
    return B.veloxq_create_dense(Q, c), O.problem_from_dense(Q, c)


def inst_dense_sk(B, n=300):
    Q, c = I.sk_qubo(n, seed=1)
    c = np.random.default_rng(2).normal(size=n) * 0.1
    return B.veloxq_create_dense(Q, c), O.problem_from_dense(Q.astype(np.float64), c)


def inst_chimera(B, m=4):
    sp = I.chimera_ising(m, m, 4, seed=0)
    ctx = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    p, C = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    return ctx, p


def inst_sparse_ragged_int(B):
    sp = I.random_sparse_qubo(333, 5, seed=5, vtype=np.int32, lo=-40, hi=40, empty_rows=7)
    c = np.random.default_rng(3).integers(-3, 4, size=sp.n).astype(np.float64)
    return B.veloxq_create_csr(sp.n, sp.rowptr, sp.col, sp.val, c), O.problem_from_csr(sp.n, sp.rowptr, sp.col, sp.val, c)


def inst_sparse_real(B):
    sp = I.random_sparse_qubo(257, 6, seed=6, vtype=np.float64, empty_rows=3)
    vals = sp.val * np.random.default_rng(4).uniform(0.5, 1.5, size=sp.val.shape)   # non-symmetric values
    c = np.random.default_rng(5).normal(size=sp.n)
    return (B.veloxq_create_csr(sp.n, sp.rowptr, sp.col, vals, c),
            O.problem_from_csr(sp.n, sp.rowptr, sp.col, vals, c))


def inst_lattice(B, L=6):
    sp = I.cubic_lattice_ising(L, seed=1)
    ctx = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    p, _ = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    return ctx, p


INSTANCES = {
    "dense_int20": inst_dense_int20,
    "dense_int_nonsym": inst_dense_int_nonsym,
    "dense_sk": inst_dense_sk,
    "chimera_c4": inst_chimera,
    "sparse_ragged_int": inst_sparse_ragged_int,
    "sparse_real": inst_sparse_real,
    "lattice_l6": inst_lattice,
}


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _abs_terms(p, X):
    """sum_i,j |Q_ij| x_i x_j + sum |c_i| x_i, for the FP64 tolerance."""
    q = O.Problem(p.n, p.er, p.ec, np.abs(p.ev), np.abs(p.c))
    return O.energy(q, X)


# ----------------------------------------------------------------- init
def test_init_state_bitexact(B):
    ctx, _ = inst_chimera(B)
    n = ctx.info.n
    for R, seed, sigma in [(37, 2**40 + 12345, 0.1), (1, 0, 1.0), (64, 7, 0.25)]:
        S = torch.empty(R, n, device="cuda")
        Y = torch.empty(R, n, device="cuda")
        B.veloxq_init_state_dev(ctx, R, seed, sigma, S, Y)
        torch.cuda.synchronize()
        S0, Y0 = O.init_state(n, R, seed, sigma)
        assert np.array_equal(S.cpu().numpy(), S0)
        assert np.array_equal(Y.cpu().numpy(), Y0)


# ----------------------------------------------------------------- energies
@pytest.mark.parametrize("name", ["dense_int20", "dense_int_nonsym", "chimera_c4", "sparse_ragged_int", "lattice_l6"])
def test_energy_integer_bitexact(B, name):
    ctx, p = INSTANCES[name](B)
    n = p.n
    X = np.concatenate([I.random_binary(61, n, seed=1), I.random_binary(3, n, seed=2, p=0.9),
                        np.zeros((1, n), np.uint8), np.ones((1, n), np.uint8)])
    out = B.veloxq_energy(ctx, X)
    ref = O.energy(p, X)
    assert ref.dtype == np.int64
    assert np.array_equal(out["E_int"], ref)
    assert np.array_equal(out["E"], ref.astype(np.float64))
    # device entry point, same values
    Xd = _cuda(X, torch.uint8)
    Ed = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
    Eid = torch.empty(X.shape[0], dtype=torch.int64, device="cuda")
    B.veloxq_energy_dev(ctx, Xd, Ed, Eid)
    torch.cuda.synchronize()
    assert np.array_equal(Eid.cpu().numpy(), ref)
    # empty batch
    assert B.veloxq_energy(ctx, np.zeros((0, n), np.uint8))["E"].shape == (0,)


@pytest.mark.parametrize("name", ["dense_sk", "sparse_real"])
def test_energy_real_fp64(B, name):
    ctx, p = INSTANCES[name](B)
    X = np.concatenate([I.random_binary(40, p.n, seed=3), np.ones((1, p.n), np.uint8)])
    E = B.veloxq_energy(ctx, X)["E"]
    ref = O.energy(p, X)
    tol = (p.nnz + p.n) * 2.0 ** -52 * _abs_terms(p, X)
    assert np.all(np.abs(E - ref) <= tol), np.max(np.abs(E - ref) / tol)


# ----------------------------------------------------------------- field
@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("R", [1, 3, 6, 64])
def test_field_fp32(B, name, R):
    ctx, p = INSTANCES[name](B)
    S = I.uniform_state(R, p.n, seed=R + 17)
    F = torch.empty(R, p.n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, _cuda(S), F)
    torch.cuda.synchronize()
    F = F.cpu().numpy().astype(np.float64)
    ref = O.field(p, S.astype(np.float64))
    scale = O.abs_field(p, S.astype(np.float64))
    assert np.all(np.abs(F - ref) <= 1e-5 * scale + 1e-30)
    nr = np.linalg.norm(ref)
    if nr > 0:
        assert np.linalg.norm(F - ref) / nr <= 1e-5


# ----------------------------------------------------------------- one step
def _check_step(S_gpu, Y_gpu, S_ref, Y_ref, atol=2e-5):
    ds = np.abs(S_gpu - S_ref)
    dy = np.abs(Y_gpu - Y_ref)
    bad = (ds > atol) | (dy > atol)
    if np.any(bad):
        # the only admissible disagreement: one side hit the wall, the other is at it
        g_wall = (np.abs(S_gpu) == 1.0) & (Y_gpu == 0.0)
        r_wall = (np.abs(S_ref) == 1.0) & (Y_ref == 0.0)
        near = np.minimum(np.abs(np.abs(S_gpu) - 1.0), np.abs(np.abs(S_ref) - 1.0)) <= 1e-4
        ok = (g_wall ^ r_wall) & near & (np.sign(S_gpu) == np.sign(S_ref))
        assert np.all(ok[bad]), (np.argwhere(bad & ~ok)[:5], ds.max(), dy.max())
    return int(bad.sum())


STEP_CASES = [
    ("chimera_c4", 1), ("chimera_c4", 2), ("sparse_ragged_int", 1), ("sparse_ragged_int", 2),
    ("sparse_real", 1), ("sparse_real", 2), ("lattice_l6", 2), ("dense_int20", 3), ("dense_sk", 3),
    ("dense_int_nonsym", 3),
]


@pytest.mark.parametrize("name,path", STEP_CASES)
@pytest.mark.parametrize("R", [5, 64])
def test_one_step(B, name, path, R):
    ctx, p = INSTANCES[name](B)
    n = p.n
    K, k = 100, 37
    sched = B.make_schedule(c0=0.3, dt=0.45, path=path)
    S = I.uniform_state(R, n, -1.0, 1.0, seed=1)
    Y = I.uniform_state(R, n, -0.6, 0.6, seed=2)
    St, Yt = _cuda(S), _cuda(Y)
    Ft = torch.empty(R, n, device="cuda")
    B.veloxq_steps_dev(ctx, R, k, 1, K, sched, St, Yt, Ft)
    torch.cuda.synchronize()
    a = O.schedule(K, [0.0, 1.0])
    S1, Y1, F = O.bsb_step(p, S, Y, a[k], np.float32(0.45), 1.0, np.float32(0.3))
    Fg = Ft.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Fg - F) <= 1e-5 * O.abs_field(p, S.astype(np.float64)) + 1e-30)
    _check_step(St.cpu().numpy(), Yt.cpu().numpy(), S1, Y1)


# ----------------------------------------------------------------- 50 steps
@pytest.mark.parametrize("name,path", [("chimera_c4", 1), ("chimera_c4", 2), ("lattice_l6", 1), ("lattice_l6", 2),
                                       ("dense_int20", 3), ("dense_sk", 3), ("sparse_real", 2)])
def test_first_50_steps_free_running(B, name, path):
    """Philox start, K = 5000 schedule, the field of each of the first 50 steps
    within 1e-5 normwise of the FP64 trajectory of the oracle."""
    ctx, p = INSTANCES[name](B)
    n, R, K, seed = p.n, 32, 5000, 99
    rho = O.spectral_radius(p)
    c0 = np.float32(2.0 / rho)
    sched = B.make_schedule(c0=float(c0), path=path)
    St = torch.empty(R, n, device="cuda")
    Yt = torch.empty(R, n, device="cuda")
    Ft = torch.empty(R, n, device="cuda")
    B.veloxq_init_state_dev(ctx, R, seed, 0.1, St, Yt)
    S0, Y0 = O.init_state(n, R, seed, 0.1)
    # 50 oracle steps whose knots {a_0, a_49} reproduce a_k = k/(K-1) of the K-step schedule
    ref = O.bsb_run(p, R, 50, 0.5, 1.0, float(c0), [0.0, 49.0 / (K - 1)], 0, S0, Y0, n_snap=50)
    worst = 0.0
    for k in range(50):
        B.veloxq_steps_dev(ctx, R, k, 1, K, sched, St, Yt, Ft)
        torch.cuda.synchronize()
        Fg = Ft.cpu().numpy().astype(np.float64)
        Fr = ref["F_snap"][k]
        nr = np.linalg.norm(Fr)
        err = np.linalg.norm(Fg - Fr) / nr if nr > 0 else np.linalg.norm(Fg)
        worst = max(worst, err)
    assert worst <= 1e-5, worst
    Sg = St.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Sg - ref["S_snap"][49]) / np.linalg.norm(ref["S_snap"][49]) <= 1e-5


@pytest.mark.parametrize("name,path", [("chimera_c4", 1), ("chimera_c4", 2), ("dense_sk", 3)])
def test_multi_step_launch_equals_single_steps(B, name, path):
    """The in-kernel step loop (resident) and the per-step launches agree bit for bit."""
    ctx, p = INSTANCES[name](B)
    n, R, K = p.n, 8, 300
    sched = B.make_schedule(c0=0.2, path=path)
    S = I.uniform_state(R, n, -0.3, 0.3, seed=4)
    Y = I.uniform_state(R, n, -0.3, 0.3, seed=5)
    S1, Y1 = _cuda(S), _cuda(Y)
    S2, Y2 = _cuda(S), _cuda(Y)
    B.veloxq_steps_dev(ctx, R, 0, 120, K, sched, S1, Y1)
    for k in range(120):
        B.veloxq_steps_dev(ctx, R, k, 1, K, sched, S2, Y2)
    torch.cuda.synchronize()
    assert torch.equal(S1, S2) and torch.equal(Y1, Y2)


def test_resident_and_stream_paths_identical(B):
    """Both sparse kernels do the same FP32 arithmetic in the same order: the
    same solve gives bitwise the same per-replica energies and best vector."""
    ctx, p = inst_chimera(B, 4)
    a = B.veloxq_solve(ctx, 48, 400, B.make_schedule(path=1, readout_every=25), seed=3)
    b = B.veloxq_solve(ctx, 48, 400, B.make_schedule(path=2, readout_every=25), seed=3)
    assert np.array_equal(a["E_per_replica"], b["E_per_replica"])
    assert np.array_equal(a["x"], b["x"]) and a["E_int"] == b["E_int"]


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("m,R", [(4, 40), (4, 304), (4, 600), (4, 640), (16, 600), (16, 1024)])
def test_resident_variants_match_stream(B, method, m, R):
    """Every replicas-per-CTA and rows-per-thread variant the plan picks
    (Chimera C4: 1, 2, 4 and 8 replicas per CTA, one row per thread; C16: 4
    and 8 replicas per CTA with rows in pairs) does the streaming kernel's
    FP32 operations in the same order: bitwise the same per-replica energies,
    for each integrator."""
    ctx, _ = inst_chimera(B, m)
    kw = dict(readout_every=25, method=method, dt=0.3)
    a = B.veloxq_solve(ctx, R, 120, B.make_schedule(path=1, **kw), seed=3)
    b = B.veloxq_solve(ctx, R, 120, B.make_schedule(path=2, **kw), seed=3)
    assert np.array_equal(a["E_per_replica"], b["E_per_replica"])
    assert np.array_equal(a["x"], b["x"])


@pytest.mark.parametrize("method", [0, 2])
@pytest.mark.parametrize("R", [8, 64])
def test_resident_runtime_slot_count_matches_stream(B, method, R):
    """Chimera C_{4,4} with shores of 6 (degree 8: eight slots per row, a
    count the kernel reads at run time, unlike the six of C_{m,m,4} and the
    lattices): bitwise the streaming kernel's energies."""
    sp = I.chimera_ising(4, 4, 6, seed=1)
    assert np.max(np.diff(sp.rowptr)) == 8
    ctx = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    kw = dict(readout_every=25, method=method, dt=0.3)
    a = B.veloxq_solve(ctx, R, 120, B.make_schedule(path=1, **kw), seed=5)
    b = B.veloxq_solve(ctx, R, 120, B.make_schedule(path=2, **kw), seed=5)
    assert np.array_equal(a["E_per_replica"], b["E_per_replica"])
    assert np.array_equal(a["x"], b["x"])


# ----------------------------------------------------------------- solve
def test_solve_dense_int20_reaches_ground_state(B):
    ctx, p = inst_dense_int20(B)
    Emin, _, _ = O.bruteforce(p)
    out = B.veloxq_solve(ctx, 128, 2000, B.make_schedule(), seed=0)
    assert out["E_int"] == Emin
    assert O.energy(p, out["x"])[0] == out["E_int"]
    assert np.min(out["E_per_replica"]) == out["E"]
    assert np.all(out["E_per_replica"] >= Emin)


@pytest.mark.parametrize("name,path", [("chimera_c4", 1), ("chimera_c4", 2), ("sparse_ragged_int", 0),
                                       ("sparse_real", 0), ("dense_sk", 0), ("dense_int_nonsym", 0)])
def test_solve_outputs_consistent(B, name, path):
    """The returned x has the returned energy; E is the minimum over replicas
    (lowest index on ties) and every replica's best is a real readout."""
    ctx, p = INSTANCES[name](B)
    out = B.veloxq_solve(ctx, 40, 300, B.make_schedule(path=path, readout_every=20), seed=5)
    Ex = O.energy(p, out["x"])[0]
    if p.integer:
        assert Ex == out["E_int"]
    else:
        tol = (p.nnz + p.n) * 2.0 ** -52 * _abs_terms(p, out["x"][None])[0]
        assert abs(Ex - out["E"]) <= tol
    assert out["E"] == np.min(out["E_per_replica"])


@pytest.mark.parametrize("name,path", [("chimera_c4", 1), ("dense_int20", 3), ("lattice_l6", 2)])
def test_solve_energy_distribution_matches_oracle(B, name, path):
    """Final per-replica best energies: GPU (FP32) vs oracle (FP64) from the
    same Philox start; after the bifurcation the runs may part, so compare
    distributions (two-sample KS) and means."""
    from scipy.stats import ks_2samp
    ctx, p = INSTANCES[name](B)
    R, K, seed = 64, 600, 21
    rho = O.spectral_radius(p)
    c0 = float(np.float32(2.0 / rho))
    out = B.veloxq_solve(ctx, R, K, B.make_schedule(path=path, c0=c0, readout_every=50), seed=seed)
    S0, Y0 = O.init_state(p.n, R, seed, 0.1)
    ref = O.bsb_run(p, R, K, 0.5, 1.0, c0, [0.0, 1.0], 50, S0, Y0)
    g, r = out["E_per_replica"], ref["best_E"]
    assert ks_2samp(g, r).pvalue > 1e-3
    spread = max(np.std(r), 1e-9)
    assert abs(np.mean(g) - np.mean(r)) <= 0.5 * spread + 1e-9


# ----------------------------------------------------------------- context facts
@pytest.mark.parametrize("name", list(INSTANCES))
def test_rho_and_K0(B, name):
    ctx, p = INSTANCES[name](B)
    info = ctx.info
    rho = O.spectral_radius(p)
    assert info.rho <= rho * (1 + 1e-6) and info.rho >= rho * (1 - 2e-2)
    _, K0 = O.bias(p)
    assert info.K0 == pytest.approx(K0, rel=1e-12, abs=1e-12)


def test_rho_multi_launch_sparse(B):
    """A sparse problem too large for the one-CTA power iteration (n = 13824)
    takes the Lanczos estimate (rows walked backwards on odd steps).
    Ferromagnetic periodic cubic lattice: rho = 6 exactly."""
    L = I.cubic_lattice_ising(24, seed=0)
    ctx = B.veloxq_create_csr(L.n, L.rowptr, L.col, np.abs(L.val).astype(np.int32))
    assert 6.0 * (1 - 2e-2) <= ctx.info.rho <= 6.0 * (1 + 1e-6)


def test_rho_multi_launch_dense_unaligned(B):
    """Dense, n % 4 != 0 and above the CSR size: the GEMV's scalar loop."""
    n = 517
    Q, c = I.sk_qubo(n, seed=3)
    ctx = B.veloxq_create_dense(Q, c)
    rho = O.spectral_radius(O.problem_from_dense(Q.astype(np.float64), c))
    assert rho * (1 - 2e-2) <= ctx.info.rho <= rho * (1 + 1e-6)


def test_rho_lanczos_wishart_and_sk(B):
    """The Lanczos estimate on dense spectra of the benchmark families: a
    Wishart planted instance (negative semi-definite coupling, rho at the
    Marchenko-Pastur edge) and an SK instance above the CSR size, against the
    oracle's dense eigensolver: from below, within 2%."""
    w = I.wishart_ising(1200, 0.75, seed=8)
    ctx = B.veloxq_create_ising_dense(-w["J"], None)
    Qd, _ = O.ising_to_qubo(-w["J"], np.zeros(1200))
    rho = O.spectral_radius(O.problem_from_dense(Qd))
    assert rho * (1 - 2e-2) <= ctx.info.rho <= rho * (1 + 1e-6)
    Q, c = I.sk_qubo(3000, seed=9)
    ctx = B.veloxq_create_dense(Q, c)
    rho = O.spectral_radius(O.problem_from_dense(Q.astype(np.float64), c))
    assert rho * (1 - 2e-2) <= ctx.info.rho <= rho * (1 + 1e-6)


def test_ising_offset_matches_oracle(B):
    sp = I.chimera_ising(3, 3, 4, seed=2)
    h = np.random.default_rng(1).integers(-2, 3, size=sp.n).astype(np.float64)
    ctx = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, h)
    p, C = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, h)
    assert ctx.info.ising_offset == pytest.approx(C)
    X = I.random_binary(16, sp.n, seed=4)
    assert np.array_equal(B.veloxq_energy(ctx, X)["E_int"], O.energy(p, X))
    w = I.wishart_ising(60, 0.75, seed=3)
    ctxd = B.veloxq_create_ising_dense(-w["J"], None)
    Qd, Cd = O.ising_to_qubo(-w["J"], np.zeros(60))
    assert ctxd.info.ising_offset == pytest.approx(Cd, rel=1e-12)
    t = ((w["t"].astype(int) + 1) // 2).astype(np.uint8)
    E0 = 0.5 * w["Jt_diag"].sum()
    # the planted state has Ising energy E0: 2 E(x*) + C = E0
    Ex = B.veloxq_energy(ctxd, t[None])["E"][0]
    assert 2 * Ex + ctxd.info.ising_offset == pytest.approx(E0, rel=1e-9)


# ----------------------------------------------------------------- errors and edges
def test_malformed_inputs_rejected(B):
    rp = np.array([0, 2, 3, 4], dtype=np.int64)
    bad_order = np.array([2, 1, 0, 0], dtype=np.int32)
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_create_csr(3, rp, bad_order, np.ones(4, np.int32))
    assert e.value.status == B.VELOXQ_EINVAL and "increasing" in e.value.message
    asym = np.array([1, 2, 0, 1], dtype=np.int32)          # rows {1,2}, {0}, {1}: (0,2) has no (2,0)
    rp2 = np.array([0, 2, 3, 4], dtype=np.int64)
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_create_csr(3, rp2, asym, np.ones(4, np.int32))
    assert e.value.status == B.VELOXQ_EUNSUPPORTED
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_create_csr(2, np.array([0, 1, 2]), np.array([1, 0]), np.array([np.nan, 1.0]))
    assert e.value.status == B.VELOXQ_EINVAL
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_create_ising_csr(2, np.array([0, 1, 2]), np.array([0, 1]), np.array([1, 1], np.int8))
    assert e.value.status == B.VELOXQ_EINVAL
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_create_csr(2, np.array([0, 2, 1]), np.array([0, 1]), np.array([1, 1], np.int32))
    assert e.value.status == B.VELOXQ_EINVAL
    ctx, _ = inst_chimera(B)
    for bad in [dict(dt=-1.0), dict(sigma0=float("nan")), dict(readout_every=-2), dict(prec=7)]:
        with pytest.raises(B.VeloxqError) as e:
            B.veloxq_solve(ctx, 4, 10, B.make_schedule(**bad))
        assert e.value.status == B.VELOXQ_EINVAL
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_solve(ctx, 0, 10)
    assert e.value.status == B.VELOXQ_EINVAL
    with pytest.raises(B.VeloxqError) as e:      # beyond the 2^20 replica limit: refused before any launch
        B.veloxq_solve(ctx, (1 << 20) + 1, 10)
    assert e.value.status == B.VELOXQ_EINVAL and "2^20" in e.value.message
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_solve(ctx, 4, 10, B.make_schedule(prec=B.VELOXQ_PREC_FP8))
    assert e.value.status == B.VELOXQ_EUNSUPPORTED


def test_real_couplings_beyond_fixed_point_range(B):
    """Real couplings whose absolute sum reaches 2^61 cannot keep exact int64
    fixed-point energies: creation refuses them (dense and sparse) instead of
    overflowing silently; just below the limit they are accepted and the
    energy of a vector is the oracle's within its FP64 bound."""
    big = np.array([[0.0, 3e18], [3e18, 0.0]])                 # sum |Q| = 6e18 > 2^61
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_create_dense(big)
    assert e.value.status == B.VELOXQ_EUNSUPPORTED and "2^61" in e.value.message
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_create_csr(2, np.array([0, 1, 2]), np.array([1, 0], np.int32), np.array([3e18, 3e18]))
    assert e.value.status == B.VELOXQ_EUNSUPPORTED
    ok = np.array([[0.0, 5e17], [5e17, 0.25]])                 # sum |Q| just above 1e18 < 2^61
    ctx = B.veloxq_create_dense(ok)
    X = np.array([[1, 1], [1, 0], [0, 1]], np.uint8)
    E = B.veloxq_energy(ctx, X)["E"]
    Eo = O.energy(O.problem_from_dense(ok), X)
    assert np.all(np.abs(E - Eo) <= 4 * 2.0 ** -52 * np.sum(np.abs(ok)))


def test_degenerate_sizes(B):
    # n = 1, no couplings: E(x) = c x, best is x = [c < 0]
    ctx = B.veloxq_create_csr(1, np.array([0, 0]), np.zeros(0, np.int32), np.zeros(0, np.int32), np.array([-3.0]))
    out = B.veloxq_solve(ctx, 1, 1)
    assert out["E_int"] in (0, -3)
    out = B.veloxq_solve(ctx, 4, 200, B.make_schedule(c0=1.0))
    assert out["E_int"] == -3 and out["x"].tolist() == [1]
    ctxd = B.veloxq_create_dense(np.array([[5]], np.int32), np.array([-7.0]))
    assert B.veloxq_energy(ctxd, np.array([[1]], np.uint8))["E_int"][0] == -2
    # every row empty: b = c drives each spin on its own
    n = 50
    c = np.where(np.arange(n) % 2 == 0, -1.0, 1.0)
    ctxe = B.veloxq_create_csr(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int8), c)
    out = B.veloxq_solve(ctxe, 3, 500, B.make_schedule(c0=1.0))
    assert out["E_int"] == -25
    # R = 1, K = 1 on every path
    for name, path in [("chimera_c4", 1), ("chimera_c4", 2), ("dense_sk", 3)]:
        ctx, p = INSTANCES[name](B)
        o = B.veloxq_solve(ctx, 1, 1, B.make_schedule(path=path))
        assert O.energy(p, o["x"])[0] == pytest.approx(o["E"], rel=1e-9, abs=1e-9)


# ----------------------------------------------------------------- full-size cases
def test_chimera_c16_full_size(B):
    """The benchmark workload (C16, 1024 replicas, 5000 steps, as timed): one
    step at full R against the oracle field, and the full solve's outputs."""
    sp = I.chimera_ising(16, 16, 4, seed=0)
    ctx = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    p, C = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    n, R = sp.n, 1024
    S = I.uniform_state(R, n, seed=8)
    Y = I.uniform_state(R, n, -0.5, 0.5, seed=9)
    St, Yt, Ft = _cuda(S), _cuda(Y), torch.empty(R, n, device="cuda")
    B.veloxq_steps_dev(ctx, R, 10, 1, 5000, B.make_schedule(c0=0.2), St, Yt, Ft)
    torch.cuda.synchronize()
    F = O.field(p, S.astype(np.float64))
    assert np.all(np.abs(Ft.cpu().numpy() - F) <= 1e-5 * O.abs_field(p, S.astype(np.float64)) + 1e-30)
    a = O.schedule(5000, [0.0, 1.0])
    S1, Y1 = O.bsb_update(F, O.bias(p)[0], a[10], 0.5, 1.0, float(np.float32(0.2)), S, Y)
    _check_step(St.cpu().numpy(), Yt.cpu().numpy(), S1, Y1)
    out = B.veloxq_solve(ctx, R, 5000, B.make_schedule(), seed=0)
    assert O.energy(p, out["x"])[0] == out["E_int"]
    assert out["E"] == out["E_per_replica"].min()
    # random states are far above what the solver reaches
    assert out["E_int"] < np.min(O.energy(p, I.random_binary(64, n, seed=1)))


def test_lattice_l100_stream_sampled_rows(B):
    """Periodic 3-D lattice at n = 10^6 with 256 replicas (streaming kernel):
    the field of sampled rows against the oracle, and exact energies."""
    L, R = 100, 256
    sp = I.cubic_lattice_ising(L, seed=0)
    ctx = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    n = sp.n
    rows = np.random.default_rng(0).choice(n, size=200, replace=False)
    # oracle problem restricted to the entries touching the sampled rows (selection only)
    p, _ = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    keep = np.isin(p.er, rows) | np.isin(p.ec, rows)
    psub = O.Problem(n, p.er[keep], p.ec[keep], p.ev[keep], p.c, p.ev_i64[keep], p.c_i64)
    S = I.uniform_state(R, n, seed=3)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, _cuda(S), F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()[:, rows].astype(np.float64)
    Sd = S.astype(np.float64)
    ref = O.field(psub, Sd)[:, rows]
    sc = O.abs_field(psub, Sd)[:, rows]
    assert np.all(np.abs(Fg - ref) <= 1e-5 * sc + 1e-30)
    X = I.random_binary(4, n, seed=5)
    assert np.array_equal(B.veloxq_energy(ctx, X)["E_int"], O.energy(p, X))


def test_lattice_l464_full_size(B):
    """The periodic lattice at L = 464 (n = 99,897,344) with 2 replicas, as
    the bench runs it (streaming kernel, rows of a regular graph indexed
    without row pointers): the field of sampled rows against the oracle, and
    a solve whose returned energy the energy entry point reproduces."""
    L, R = 464, 2
    sp = I.cubic_lattice_ising(L, seed=0)
    n = sp.n
    ctx = B.veloxq_create_ising_csr(n, sp.rowptr, sp.col, sp.val, sp.lin)
    rows = np.random.default_rng(1).choice(n, size=64, replace=False)
    # coupled pairs touching the sampled rows (selection only); each row has 6 entries
    ri = np.repeat(rows, 6)
    cj = sp.col.reshape(n, 6)[rows].reshape(-1).astype(np.int64)
    jv = sp.val.reshape(n, 6)[rows].reshape(-1).astype(np.float64)
    pi, pj = np.minimum(ri, cj), np.maximum(ri, cj)
    key = pi * n + pj
    _, first = np.unique(key, return_index=True)
    psub, _ = O.ising_pairs_to_qubo(n, pi[first], pj[first], jv[first])
    S = I.uniform_state(R, n, seed=2)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, _cuda(S), F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()[:, rows].astype(np.float64)
    Sd = S.astype(np.float64)
    ref = O.field(psub, Sd)[:, rows]
    sc = O.abs_field(psub, Sd)[:, rows]
    assert np.all(np.abs(Fg - ref) <= 1e-5 * sc + 1e-30)
    del S, Sd, F
    out = B.veloxq_solve(ctx, R, 50, B.make_schedule(readout_every=0), seed=0)
    assert out["E"] == np.min(out["E_per_replica"])
    again = B.veloxq_energy(ctx, out["x"][None])
    assert again["E_int"][0] == out["E_int"]
