"""Failure detection without a GPU fault: the bounded device wait the
tensor-core kernels use is made to run out (a barrier that nothing arrives
on), reports ETIMEDOUT through its error word, and the device stays usable.
Host-side argument errors are covered in test_abi.py and test_gpu_parity.py."""
import numpy as np
import pytest

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


def test_bounded_wait_gives_up_and_device_stays_usable(B):
    for budget in (2_000, 2_000_000):            # about 1 us and 1 ms of SM cycles
        with pytest.raises(B.VeloxqError) as e:
            B.veloxq_selftest_timeout(budget)
        assert e.value.status == B.VELOXQ_ETIMEDOUT and "code 8" in e.value.message
    with pytest.raises(B.VeloxqError) as e:
        B.veloxq_selftest_timeout(10)
    assert e.value.status == B.VELOXQ_EINVAL
    # the context and the device are intact: tensor-core and resident solves still run
    Q, c = I.sk_qubo(256, seed=3)
    ctx = B.veloxq_create_dense(Q, c)
    out = B.veloxq_solve(ctx, 128, 50, B.make_schedule(prec=1, readout_every=0), seed=1)
    assert np.isfinite(out["E"])
    Qi, ci = I.dense_int_qubo(20, seed=0)
    ctx2 = B.veloxq_create_dense(Qi, ci)
    assert B.veloxq_solve(ctx2, 32, 200, B.make_schedule(), seed=0)["E_int"] <= 0
