"""Third-order instances (Sec. "HUBO") through the library: reduced to second
order by veloxq_hubo3_reduce, solved on the GPU, and checked against the
oracle's third-order energy and exhaustive minimum."""
import itertools

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


@pytest.mark.parametrize("kind,path", [("chain", 1), ("chain", 2), ("max3sat", 1)])
def test_reduced_solve_reaches_hubo_minimum(B, kind, path):
    N = 14
    inst = I.hubo_chain_3body(N, seed=7) if kind == "chain" else I.max3sat_weighted(N, seed=8)
    red = B.veloxq_hubo3_reduce(N, inst.h, inst.pairs, inst.triples)
    ctx = B.veloxq_create_ising_csr(red["n"], red["rowptr"], red["col"], red["val"], red["lin"])
    out = B.veloxq_solve(ctx, 128, 2000, B.make_schedule(path=path), seed=1)
    S = np.array(list(itertools.product([-1, 1], repeat=N)), dtype=np.int8)
    H = O.hubo3_energy(N, inst.h, inst.pairs, inst.triples, S)
    s = (2 * out["x"].astype(np.int8) - 1)
    # the returned energy is the reduced cost of the returned spins (2E + C, App. A), whose
    # minimum over the auxiliary spins is the third-order cost of the original ones
    N2, (qi, qj, qv), lin, off = O.hubo3_reduce(N, inst.h, inst.pairs, inst.triples)
    Hred = O.hubo3_energy(N2, lin, (qi, qj, qv), None, s[None, :])[0] + off
    assert Hred == pytest.approx(2 * out["E"] + ctx.info.ising_offset + red["offset"], abs=1e-9)
    Hs = O.hubo3_energy(N, inst.h, inst.pairs, inst.triples, s[None, :N])[0]
    assert Hs <= Hred + 1e-9
    assert Hs == pytest.approx(H.min(), abs=1e-9)


@pytest.mark.parametrize("path", [1, 2])
def test_3r3x_reduced_solve_reaches_planted_energy(B, path):
    """Planted 3-regular 3-XORSAT, n = 24 equations and variables, reduced to
    48 spins: the solve returns a configuration whose original spins satisfy
    every equation (third-order cost -m). The FP64 oracle's dynamics from
    the same initial states put 207 of 256 replicas there."""
    inst = I.xorsat_3r3x(24, seed=1)
    h = inst.hubo
    red = B.veloxq_hubo3_reduce(h.n, h.h, h.pairs, h.triples)
    ctx = B.veloxq_create_ising_csr(red["n"], red["rowptr"], red["col"], red["val"], red["lin"])
    rho = ctx.info.rho
    out = B.veloxq_solve(ctx, 256, 2000, B.make_schedule(path=path, c0=float(np.float32(2.0 / rho))), seed=1)
    s = 2 * out["x"].astype(np.int8) - 1
    Hs = O.hubo3_energy(h.n, h.h, h.pairs, h.triples, s[None, :h.n].astype(np.float64))[0]
    assert 2 * out["E"] + ctx.info.ising_offset + red["offset"] >= Hs - 1e-9
    assert Hs == inst.E0


def test_stream_chunked_thread_order(B):
    """A random sparse graph whose state outgrows L2 (3R3X, 1e5 equations,
    2e5 spins, 256 replicas: 205 MB per state array): the timed choice of the
    streaming step takes a chunked thread order (every row of a replica chunk
    before the next chunk, so the neighbours' states gathered stay in L2), and
    its field matches the oracle on replicas from several chunks."""
    inst = I.xorsat_3r3x(10 ** 5, seed=0)
    h = inst.hubo
    red = B.veloxq_hubo3_reduce(h.n, h.h, h.pairs, h.triples)
    ctx = B.veloxq_create_ising_csr(red["n"], red["rowptr"], red["col"], red["val"], red["lin"])
    R, n = 256, red["n"]
    B.veloxq_solve(ctx, R, 4, B.make_schedule(path=2, readout_every=0), seed=2)
    t = B.veloxq_last_timing(ctx)
    assert t.path == 2 and t.stream_gather in (1, 4)
    assert t.stream_chunk > 0 and R % t.stream_chunk == 0
    S = I.uniform_state(R, n, seed=3)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, torch.as_tensor(S, device="cuda"), F)
    torch.cuda.synchronize()
    rows = np.r_[0:3, t.stream_chunk - 1:t.stream_chunk + 2, R - 3:R]
    N, (qi, qj, qv), lin, _ = O.hubo3_reduce(h.n, h.h, h.pairs, h.triples)
    p, _ = O.ising_pairs_to_qubo(N, qi, qj, qv, lin)
    Ss = S[rows].astype(np.float64)
    ref = O.field(p, Ss)
    scale = O.abs_field(p, Ss)
    assert np.all(np.abs(F.cpu().numpy()[rows].astype(np.float64) - ref) <= 1e-5 * scale + 1e-30)


def test_stream_chunked_order_bitwise_equal_to_unchunked(B):
    """Replicas are independent and seeded by index, so the first 64
    replicas of a 256-replica solve (chunked thread order: 205 MB per state
    array) and a 64-replica solve (51 MB, never chunked) do the same FP32
    operations: bitwise the same per-replica energies."""
    inst = I.xorsat_3r3x(10 ** 5, seed=2)
    h = inst.hubo
    red = B.veloxq_hubo3_reduce(h.n, h.h, h.pairs, h.triples)
    ctx = B.veloxq_create_ising_csr(red["n"], red["rowptr"], red["col"], red["val"], red["lin"])
    sched = B.make_schedule(path=2, readout_every=10)
    big = B.veloxq_solve(ctx, 256, 30, sched, seed=7)
    assert B.veloxq_last_timing(ctx).stream_chunk > 0
    small = B.veloxq_solve(ctx, 64, 30, sched, seed=7)
    assert B.veloxq_last_timing(ctx).stream_chunk == 0
    assert np.array_equal(big["E_per_replica"][:64], small["E_per_replica"])


def test_hubo_chain_5e7_full_size(B):
    """The third-order chain at the paper's largest scale (Sec. "HUBO": a
    chain of N = 5e7 spins, reduced by eq. reduction to 1e8 second-order
    spins, float couplings, auxiliary spins numbered next to their terms), as
    the bench runs it: the field of sampled rows against the oracle's field
    of the coupled pairs touching them (built from the reduced couplings,
    which the CPU tests pin to the oracle's own reduction), and a solve whose
    returned energy the energy entry point reproduces and whose third-order
    cost bounds the reduced one."""
    N, R = 5 * 10 ** 7, 2
    inst = I.hubo_chain_3body(N, seed=0)
    red = B.veloxq_hubo3_reduce(inst.n, inst.h, inst.pairs, inst.triples, local=True)
    n = red["n"]
    assert n == 2 * N - 2
    ctx = B.veloxq_create_ising_csr(n, red["rowptr"], red["col"], red["val"], red["lin"])
    rp = red["rowptr"]
    rows = np.sort(np.random.default_rng(3).choice(n, size=64, replace=False))
    ri = np.concatenate([np.full(rp[r + 1] - rp[r], r, dtype=np.int64) for r in rows])
    cj = np.concatenate([red["col"][rp[r]:rp[r + 1]] for r in rows]).astype(np.int64)
    jv = np.concatenate([red["val"][rp[r]:rp[r + 1]] for r in rows])
    pi, pj = np.minimum(ri, cj), np.maximum(ri, cj)
    _, first = np.unique(pi * n + pj, return_index=True)
    psub, _ = O.ising_pairs_to_qubo(n, pi[first], pj[first], jv[first])
    S = I.uniform_state(R, n, seed=4)
    F = torch.empty(R, n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, torch.as_tensor(S, device="cuda"), F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()[:, rows].astype(np.float64)
    Sd = S.astype(np.float64)
    ref = O.field(psub, Sd)[:, rows]
    sc = O.abs_field(psub, Sd)[:, rows]
    assert np.all(np.abs(Fg - ref) <= 1e-5 * sc + 1e-30)
    del S, Sd, F
    out = B.veloxq_solve(ctx, R, 30, B.make_schedule(readout_every=0), seed=0)
    assert out["E"] == np.min(out["E_per_replica"])
    again = B.veloxq_energy(ctx, out["x"][None])
    assert abs(again["E"][0] - out["E"]) <= 1e-9 * max(1.0, abs(out["E"]))
