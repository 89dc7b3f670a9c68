"""The two further integrators of App. B on every kernel path, against the
FP64 oracle: adiabatic SB as printed (quartic term, no walls) and Parallel
Annealing (the field of the binarised spins, momentum, clip).

Tolerances follow the arithmetic of each step:
* FP32 field: |dF| <= 1e-5 (|Qoff| |o|), o the method's operand;
* one FP32 step: |ds|, |dy| <= 2e-5 (no walls for aSB; PA's clip is exact);
* the resident and streaming kernels do the same FP32 operations in the same
  order, so they agree bit for bit;
* PA's operand is +-1, exact in BF16 and in FP8 (+-448): on a +-1 instance
  the BF16 field is exact and the FP8 one exact up to the FP32 rounding of
  its row scale.
"""
import numpy as np
import pytest

import oracle as O
from paper_2501_19221_gb300 import instances as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

METHOD = {"asb": 1, "pa": 2}


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


def inst_chimera(B, m=4):
    sp = I.chimera_ising(m, m, 4, seed=0)
    p, _ = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    return B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin), p


def inst_lattice(B, L=6):
    sp = I.cubic_lattice_ising(L, seed=1)
    p, _ = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    return B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin), p


def inst_sparse_real(B):
    sp = I.random_sparse_qubo(257, 6, seed=6, vtype=np.float64, empty_rows=3)
    vals = sp.val * np.random.default_rng(4).uniform(0.5, 1.5, size=sp.val.shape)
    c = np.random.default_rng(5).normal(size=sp.n)
    return (B.veloxq_create_csr(sp.n, sp.rowptr, sp.col, vals, c),
            O.problem_from_csr(sp.n, sp.rowptr, sp.col, vals, c))


def inst_dense_sk(B, n=300):
    Q, _ = I.sk_qubo(n, seed=1)
    c = np.random.default_rng(2).normal(size=n) * 0.1
    return B.veloxq_create_dense(Q, c), O.problem_from_dense(Q.astype(np.float64), c)


def inst_dense_int20(B):
    Q, c = I.dense_int_qubo(20, seed=0)
    return B.veloxq_create_dense(Q, c), O.problem_from_dense(Q, c)


INSTANCES = {"chimera_c4": inst_chimera, "lattice_l6": inst_lattice, "sparse_real": inst_sparse_real,
             "dense_sk": inst_dense_sk, "dense_int20": inst_dense_int20}

CASES = [("chimera_c4", 1), ("chimera_c4", 2), ("lattice_l6", 2), ("sparse_real", 1), ("sparse_real", 2),
         ("dense_sk", 3), ("dense_int20", 3)]


@pytest.mark.parametrize("method", ["asb", "pa"])
@pytest.mark.parametrize("name,path", CASES)
@pytest.mark.parametrize("R", [5, 64])
def test_one_step(B, method, name, path, R):
    ctx, p = INSTANCES[name](B)
    n = p.n
    K, k = 100, 37
    dt, c0, alpha = np.float32(0.45), np.float32(0.3), np.float32(0.8)
    sched = B.make_schedule(c0=float(c0), dt=float(dt), path=path, method=METHOD[method], momentum=float(alpha))
    S = I.uniform_state(R, n, -1.0, 1.0, seed=1)
    Y = I.uniform_state(R, n, -0.6, 0.6, seed=2)
    St, Yt = _cuda(S), _cuda(Y)
    Ft = torch.empty(R, n, device="cuda")
    B.veloxq_steps_dev(ctx, R, k, 1, K, sched, St, Yt, Ft)
    torch.cuda.synchronize()
    a = O.schedule(K, [0.0, 1.0])
    S1, Y1, F = O.step(method, p, S, Y, a[k], float(dt), 1.0, float(c0), float(alpha))
    op = O.field_operand(method, S)
    assert np.all(np.abs(Ft.cpu().numpy() - F) <= 1e-5 * O.abs_field(p, op) + 1e-30)
    assert np.max(np.abs(St.cpu().numpy() - S1)) <= 2e-5
    assert np.max(np.abs(Yt.cpu().numpy() - Y1)) <= 2e-5
    if method == "pa":
        assert np.max(np.abs(St.cpu().numpy())) <= 1.0     # the clip


@pytest.mark.parametrize("method", ["asb", "pa"])
@pytest.mark.parametrize("name,path", [("chimera_c4", 1), ("chimera_c4", 2), ("dense_sk", 3)])
def test_first_20_steps_free_running(B, method, name, path):
    """Philox start: 20 free-running steps stay within 1e-4 normwise of the
    FP64 trajectory (PA's sign can only flip where |x| is at rounding level,
    which this seed does not meet)."""
    ctx, p = INSTANCES[name](B)
    n, R, K, seed = p.n, 32, 400, 99
    c0 = np.float32(2.0 / O.spectral_radius(p))
    sched = B.make_schedule(c0=float(c0), dt=0.3, path=path, method=METHOD[method], momentum=0.9)
    St = torch.empty(R, n, device="cuda")
    Yt = torch.empty(R, n, device="cuda")
    B.veloxq_init_state_dev(ctx, R, seed, 0.1, St, Yt)
    S0, Y0 = O.init_state(n, R, seed, 0.1)
    ref = O.bsb_run(p, R, 20, float(np.float32(0.3)), 1.0, float(c0), [0.0, 19.0 / (K - 1)], 0, S0, Y0, n_snap=20,
                    method=method, alpha=float(np.float32(0.9)))
    B.veloxq_steps_dev(ctx, R, 0, 20, K, sched, St, Yt)
    torch.cuda.synchronize()
    Sg = St.cpu().numpy().astype(np.float64)
    Sr = ref["S_snap"][19]
    assert np.linalg.norm(Sg - Sr) / np.linalg.norm(Sr) <= 1e-4


@pytest.mark.parametrize("method,R", [("asb", 48), ("pa", 48), ("pa", 6), ("pa", 5)])
def test_resident_and_stream_paths_identical(B, method, R):
    """The same solve on both sparse paths gives the same bits (for Parallel
    Annealing with vectors of 4, 2 and 1 replicas on the streaming path)."""
    ctx, p = inst_chimera(B, 4)
    kw = dict(readout_every=25, method=METHOD[method], dt=0.3)
    a = B.veloxq_solve(ctx, R, 400, B.make_schedule(path=1, **kw), seed=3)
    b = B.veloxq_solve(ctx, R, 400, B.make_schedule(path=2, **kw), seed=3)
    assert np.array_equal(a["E_per_replica"], b["E_per_replica"])
    assert np.array_equal(a["x"], b["x"]) and a["E_int"] == b["E_int"]
    assert O.energy(p, a["x"][None, :])[0] == a["E_int"]


@pytest.mark.parametrize("path", [1, 3])
def test_pa_solve_reaches_ground_state_n20(B, path):
    """Parallel Annealing through the library finds the enumerated ground state
    of the dense n = 20 instance, resident and dense paths."""
    ctx, p = inst_dense_int20(B)
    Emin, _, _ = O.bruteforce(p)
    out = B.veloxq_solve(ctx, 128, 2000, B.make_schedule(path=path, method=2), seed=0)
    assert out["E_int"] == Emin
    assert O.energy(p, out["x"][None, :])[0] == Emin


def test_pa_low_precision_field_exact_on_pm1_instance(B):
    """Dense +-1 couplings (a Chimera C8 Ising instance in dense form, J =
    +-1, h = 0, so Qoff = +-1/2): PA's operand is +-1, and the tensor-core
    field of one PA step is the exact field of sign(x) in BF16, and in FP8
    (Qoff/q_i = +-448 exactly) up to the three FP32 roundings of the row scale
    q_i / 448."""
    sp = I.chimera_ising(8, 8, 4, seed=3)
    J = np.triu(sp.to_dense(), 1)
    ctx = B.veloxq_create_ising_dense(J.astype(np.float32), None)
    p, _ = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    n, R = sp.n, 256
    S = I.uniform_state(R, n, -1.0, 1.0, seed=7)
    Y = I.uniform_state(R, n, -0.5, 0.5, seed=8)
    got = {}
    for prec in (1, 2, 3):
        St, Yt = _cuda(S), _cuda(Y)
        Ft = torch.empty(R, n, device="cuda")
        B.veloxq_steps_dev(ctx, R, 3, 1, 10, B.make_schedule(path=3, prec=prec, method=2, c0=0.2), St, Yt, Ft)
        torch.cuda.synchronize()
        F = O.field(p, O.field_operand("pa", S))
        Fg = Ft.cpu().numpy().astype(np.float64)
        got[prec] = (Fg, St.cpu().numpy(), Yt.cpu().numpy())
        if prec == 1:
            assert np.array_equal(Fg, F)
        else:
            assert np.all(np.abs(Fg - F) <= 4e-7 * np.abs(F))
    # PA's operand is exact in one E4M3 term: FP8 runs it as FP8_ONE_TERM does, bit for bit
    for a, b in zip(got[2], got[3]):
        assert np.array_equal(a, b)


def test_method_errors(B):
    ctx, _ = inst_dense_sk(B, 64)
    for prec in (2, 3):
        with pytest.raises(B.VeloxqError, match="EUNSUPPORTED|status -5"):
            B.veloxq_solve(ctx, 16, 4, B.make_schedule(prec=prec, method=1), seed=0)
    with pytest.raises(B.VeloxqError, match="status -1"):
        B.veloxq_solve(ctx, 16, 4, B.make_schedule(prec=4), seed=0)
    with pytest.raises(B.VeloxqError):
        B.veloxq_solve(ctx, 16, 4, B.make_schedule(method=3), seed=0)
    with pytest.raises(B.VeloxqError):
        B.veloxq_solve(ctx, 16, 4, B.make_schedule(method=2, momentum=1.0), seed=0)
    lat, _ = inst_lattice(B, 4)
    with pytest.raises(B.VeloxqError, match="status -5"):
        B.veloxq_grad(lat, 8, 10, B.make_schedule(method=2), 0, 5)


def test_pa_batch_matches_per_instance_quality(B):
    """The persistent batch kernel runs PA as well: outputs are exact energies
    of the returned vectors."""
    sizes = [37, 200, 150]
    insts = [I.sk_qubo(n, seed=40 + i) for i, n in enumerate(sizes)]
    ctxs = [B.veloxq_create_dense(Q, c) for Q, c in insts]
    out = B.veloxq_solve_batch(ctxs, 64, 300, B.make_schedule(prec=1, readout_every=0, method=2, dt=0.1), seed=2)
    assert B.veloxq_last_timing(ctxs[0]).main_launches == 1
    for (Q, c), x, E in zip(insts, out["x"], out["E"]):
        p = O.problem_from_dense(Q.astype(np.float64), c)
        tol = (p.nnz + p.n) * 2.0 ** -52 * (np.sum(np.abs(Q)) + np.sum(np.abs(c)))
        assert abs(O.energy(p, x)[0] - E) <= tol
