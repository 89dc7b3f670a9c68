"""Exact readout energies of dense instances on the tensor cores (digit
planes of the fixed-point couplings, BF16 operands, FP32 accumulation),
against the oracle.

Integer instances: bit-exact int64 energies. Real-valued instances: the
FP64 oracle within the fixed-point rounding bound (the same bar as the
CUDA-core kernel), and bit-identical to the CUDA-core kernel, which forms
the same fixed-point sum in another order (both are exact integer sums).
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


def _states(n, seed):
    return np.concatenate([I.random_binary(29, n, seed=seed), I.random_binary(3, n, seed=seed + 1, p=0.95),
                           np.zeros((1, n), np.uint8), np.ones((1, n), np.uint8)])


def _dev_energy(B, ctx, X):
    """The device entry point (CUDA-core kernel)."""
    Xd = torch.as_tensor(X, device="cuda")
    E = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
    Ei = torch.empty(X.shape[0], dtype=torch.int64, device="cuda") if ctx.info.is_integer else None
    B.veloxq_energy_dev(ctx, Xd, E, Ei)
    torch.cuda.synchronize()
    return E.cpu().numpy(), (Ei.cpu().numpy() if Ei is not None else None)


def _abs_terms(p, X):
    q = O.Problem(p.n, p.er, p.ec, np.abs(p.ev), np.abs(p.c))
    return O.energy(q, X)


@pytest.mark.parametrize("n,lo,hi", [(1024, -8, 8), (1100, -(2 ** 27), 2 ** 27), (1031, -3, 3)])
def test_integer_bitexact(B, n, lo, hi):
    """Non-symmetric int32 couplings: 1 to 4 digit planes, ragged K padding."""
    rng = np.random.default_rng(n)
    Q = rng.integers(lo, hi + 1, size=(n, n)).astype(np.int32)
    c = rng.integers(-50, 51, size=n).astype(np.float64)
    ctx = B.veloxq_create_dense(Q, c)
    p = O.problem_from_dense(Q, c)
    X = _states(n, 7)
    out = B.veloxq_energy(ctx, X)
    ref = O.energy(p, X)
    assert np.array_equal(out["E_int"], ref)
    assert np.array_equal(out["E"], ref.astype(np.float64))
    E_dev, Ei_dev = _dev_energy(B, ctx, X)
    assert np.array_equal(Ei_dev, ref)


def test_zero_couplings(B):
    """Q = 0 off the diagonal: one plane of zeros, E = sum x_i (Q_ii + c_i)."""
    n = 1024
    Q = np.diag(np.arange(n) % 7 - 3).astype(np.int32)
    c = np.ones(n)
    ctx = B.veloxq_create_dense(Q, c)
    X = _states(n, 3)
    ref = X.astype(np.int64) @ (np.diag(Q).astype(np.int64) + 1)
    assert np.array_equal(B.veloxq_energy(ctx, X)["E_int"], ref)


@pytest.mark.parametrize("kind", ["sk", "wide"])
def test_real_matches_oracle_and_cuda_cores(B, kind):
    """SK couplings (about 5 planes) and couplings spread over eight decades
    (all 8 planes); n % 16 != 0."""
    n = 1100
    rng = np.random.default_rng(5)
    if kind == "sk":
        Q, _ = I.sk_qubo(n, seed=2)
    else:
        Q = (rng.choice([-1.0, 1.0], size=(n, n)) * 10.0 ** rng.uniform(-6, 2, size=(n, n))).astype(np.float32)
        Q[0, 1] = 3.0e7   # most of sum |Q|: its fixed-point value is near 2^60
    c = rng.normal(size=n)
    ctx = B.veloxq_create_dense(Q, c)
    p = O.problem_from_dense(Q.astype(np.float64), c)
    X = _states(n, 11)
    E = B.veloxq_energy(ctx, X)["E"]
    ref = O.energy(p, X)
    tol = (p.nnz + p.n) * 2.0 ** -52 * _abs_terms(p, X)
    assert np.all(np.abs(E - ref) <= tol), np.max(np.abs(E - ref) / tol)
    E_dev, _ = _dev_energy(B, ctx, X)
    assert np.array_equal(E, E_dev)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_readouts(B, prec):
    """Readouts inside the captured step loop (FP32, BF16 and FP8 field
    paths): the reported best energy is the oracle's energy of the returned
    configuration, and no replica reports an energy below it."""
    n = 1056
    rng = np.random.default_rng(9)
    Q = rng.integers(-20, 21, size=(n, n)).astype(np.int32)
    Q = np.triu(Q) + np.triu(Q, 1).T
    c = rng.integers(-5, 6, size=n).astype(np.float64)
    ctx = B.veloxq_create_dense(Q, c)
    p = O.problem_from_dense(Q, c)
    sched = B.make_schedule(prec=prec, readout_every=10)
    out = B.veloxq_solve(ctx, 40, 60, sched, seed=3)
    assert out["E_int"] == O.energy(p, out["x"][None, :])[0]
    assert out["E"] == float(out["E_int"])
    assert np.min(out["E_per_replica"]) == out["E"]
