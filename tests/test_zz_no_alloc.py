"""veloxq_energy_dev_noalloc: the energy entry point for callers that cannot
allocate device memory during a call (code inside a custom allocator that must
not re-enter cudaMalloc, processes with a fixed device-memory budget, loops
that cannot absorb an allocation's synchronisation). It must give the same
energies as veloxq_energy_dev, call after call, while its scratch is a fixed
array shared by all calls; and those energies are the oracle's. This file is
collected last so that a run stopping at its first failure has run every other
test before it."""
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


def _both(B, ctx, X, integer):
    n_b = X.shape[0]
    Xd = torch.as_tensor(X, device="cuda")
    E1 = torch.empty(n_b, dtype=torch.float64, device="cuda")
    E2 = torch.empty(n_b, dtype=torch.float64, device="cuda")
    I1 = torch.empty(n_b, dtype=torch.int64, device="cuda") if integer else None
    I2 = torch.empty(n_b, dtype=torch.int64, device="cuda") if integer else None
    B.veloxq_energy_dev(ctx, Xd, E1, I1)
    B.veloxq_energy_dev_noalloc(ctx, Xd, E2, I2)
    torch.cuda.synchronize()
    return E1.cpu().numpy(), E2.cpu().numpy(), (I1.cpu().numpy() if integer else None), \
        (I2.cpu().numpy() if integer else None)


def test_noalloc_energy_matches_allocating_entry_point_twice(B):
    sp = I.chimera_ising(8, 8, 4, seed=3)
    sparse = B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    Q, c = I.sk_qubo(300, seed=2)
    dense = B.veloxq_create_dense(Q, c)
    p_sparse, _ = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
    p_dense = O.problem_from_dense(Q.astype(np.float64), c)
    for ctx, p, n, integer in [(sparse, p_sparse, sp.n, True), (dense, p_dense, 300, False)]:
        for call in range(2):                      # two calls in a row share the scratch
            X = I.random_binary(97 + 31 * call, n, seed=call + 5)
            E1, E2, I1, I2 = _both(B, ctx, X, integer)
            # same kernels, same fixed-point sums: identical results
            assert np.array_equal(E1, E2)
            Eo = O.energy(p, X)
            if integer:
                assert np.array_equal(I1, I2)
                assert np.array_equal(I2, Eo)            # exact int64 energies
            else:
                # within the oracle's own FP64 summation bound
                tol = (p.nnz + n) * 2.0 ** -52 * (np.sum(np.abs(Q)) + np.sum(np.abs(c)))
                assert np.all(np.abs(E2 - Eo) <= tol)


def test_noalloc_rejects_batches_beyond_its_scratch(B):
    Q, c = I.sk_qubo(2048, seed=1)
    ctx = B.veloxq_create_dense(Q, c)              # 32 groups per vector -> at most 16384 vectors
    X = torch.zeros((16385, 2048), dtype=torch.uint8, device="cuda")
    E = torch.empty(16385, dtype=torch.float64, device="cuda")
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_energy_dev_noalloc(ctx, X, E)
    assert e.value.status == B.VELOXQ_EINVAL and "16384" in e.value.message
