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
