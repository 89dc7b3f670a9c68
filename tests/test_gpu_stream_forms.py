"""The gather forms of the streaming step (one, four or six couplings at a
time) and its replica chunking, each fixed through VELOXQ_STREAM_FORM: the
same CSR summation order, so every form gives the same bits as the
one-at-a-time loop, and each form's field is the oracle's (App. B:
F = Qoff S) on ragged rows, empty rows, rows of a regular lattice and one
hub row of 3000 couplings."""
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


def _hub_graph():
    """Mean degree 12 plus vertex 0 coupled to 3000 others."""
    rng = np.random.default_rng(9)
    n = 6000
    m = 6 * n
    u = rng.integers(1, n, size=m)
    v = rng.integers(1, n, size=m)
    hub = rng.choice(np.arange(1, n), size=3000, replace=False)
    u = np.concatenate([u, np.zeros(3000, dtype=np.int64)])
    v = np.concatenate([v, hub])
    keep = u != v
    lo, hi = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    key = np.unique(lo * n + hi)
    lo, hi = key // n, key % n
    w = rng.uniform(-1.0, 1.0, size=lo.shape[0]).astype(np.float32)
    rowptr, col, val = I._csr_from_edges(n, lo, hi, w)
    return I.SparseCoupling(n, rowptr, col, val.astype(np.float32), rng.uniform(-1, 1, n))


# mean degree 40: rows of about 20 to 65 couplings, five empty rows, integer
# weights (the 8-bit copy); the float weights of the Zephyr Z_6 QUBO; the
# 3-D +-J lattice (every row 6 couplings, no row pointers read); the hub graph
GRAPHS = {
    "ragged_int": lambda: (I.random_sparse_qubo(3000, 40.0, seed=7, vtype=np.float32, empty_rows=5), "qubo"),
    "zephyr_z6": lambda: (I.zephyr_qubo(6, seed=1), "qubo"),
    "lattice_l12": lambda: (I.cubic_lattice_ising(12, seed=2), "ising"),
    "hub": lambda: (_hub_graph(), "qubo"),
}


def _create(B, sp, kind):
    make = B.veloxq_create_csr if kind == "qubo" else B.veloxq_create_ising_csr
    return make(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)


def _oracle_problem(sp, kind):
    if kind == "qubo":
        return O.problem_from_csr(sp.n, sp.rowptr, sp.col, sp.val.astype(np.float64), sp.lin)
    return O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)[0]


def _forms(R, lattice):
    """The forms ("gather chunk", chunk in replicas) valid for R replicas in
    vectors of 4."""
    gathers = (1, 4, 6) if lattice else (1, 4)
    out = [f"{g} 0" for g in gathers]
    for chunk in (32, 64, 128):                 # 8, 16 and 32 vectors per chunk
        if chunk < R and R % chunk == 0:
            out += [f"{g} {chunk}" for g in gathers]
    return out


def _run(B, g, monkeypatch, form, R, method, steps=60):
    sp, kind = g
    monkeypatch.setenv("VELOXQ_STREAM_FORM", form)
    ctx = _create(B, sp, kind)
    sched = B.make_schedule(path=2, method=method, readout_every=20)
    out = B.veloxq_solve(ctx, R, steps, sched, seed=11)
    t = B.veloxq_last_timing(ctx)
    assert t.path == 2
    gth, c = (int(v) for v in form.split())
    assert t.stream_gather == gth and t.stream_chunk == c
    return out


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("R", [32, 64, 256, 512])
@pytest.mark.parametrize("method", [0, 1, 2])
def test_forms_bit_identical(B, monkeypatch, name, R, method):
    g = GRAPHS[name]()
    ref = None
    for form in _forms(R, name.startswith("lattice")):
        out = _run(B, g, monkeypatch, form, R, method)
        if ref is None:
            ref = out
            continue
        assert np.array_equal(out["E_per_replica"], ref["E_per_replica"]), form
        assert np.array_equal(out["x"], ref["x"]), form


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("form", ["1 0", "4 32"])
def test_form_field_against_oracle(B, monkeypatch, name, form):
    """One step through a fixed form (set by a solve of the same replica
    count first): the field within 1e-5 of |Qoff||S| elementwise of the
    oracle's FP64 field, including the empty rows (zero); the field entry
    point gives the same bits."""
    sp, kind = GRAPHS[name]()
    R = 128
    monkeypatch.setenv("VELOXQ_STREAM_FORM", form)
    ctx = _create(B, sp, kind)
    B.veloxq_solve(ctx, R, 2, B.make_schedule(path=2), seed=1)
    t = B.veloxq_last_timing(ctx)
    assert (t.stream_gather, t.stream_chunk) == tuple(int(v) for v in form.split())
    p = _oracle_problem(sp, kind)
    S = I.uniform_state(R, sp.n, -1.0, 1.0, seed=3)
    Y = I.uniform_state(R, sp.n, -0.5, 0.5, seed=4)
    St, Yt, Ft = _cuda(S), _cuda(Y), torch.empty(R, sp.n, device="cuda")
    B.veloxq_steps_dev(ctx, R, 0, 1, 100, B.make_schedule(path=2), St, Yt, Ft)
    torch.cuda.synchronize()
    Sd = S.astype(np.float64)
    F = Ft.cpu().numpy().astype(np.float64)
    ref = O.field(p, Sd)
    assert np.all(np.abs(F - ref) <= 1e-5 * O.abs_field(p, Sd) + 1e-30)
    if name == "ragged_int":
        assert np.all(F[:, :5] == 0.0)
    F2 = torch.empty(R, sp.n, device="cuda")
    B.veloxq_field_dev(ctx, R, B.VELOXQ_PREC_FP32, _cuda(S), F2)
    torch.cuda.synchronize()
    assert np.array_equal(F2.cpu().numpy(), Ft.cpu().numpy())


def test_stream_form_rejected(B, monkeypatch):
    """Forms that do not fit are refused with EINVAL: six couplings at a time
    on rows that are not all of six, and a chunk the replicas do not split
    into."""
    sp, kind = GRAPHS["zephyr_z6"]()
    for form in ("6 0", "1 48"):
        monkeypatch.setenv("VELOXQ_STREAM_FORM", form)
        ctx = _create(B, sp, kind)
        with pytest.raises(B.VeloxqError) as e:
            B.veloxq_solve(ctx, 128, 10, B.make_schedule(path=2), seed=1)
        assert e.value.status == B.VELOXQ_EINVAL and "VELOXQ_STREAM_FORM" in e.value.message
