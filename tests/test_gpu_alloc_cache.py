"""The library's cache of freed device buffers: contexts of different sizes
and paths created, solved and destroyed in turn (each reusing blocks the
previous ones freed) return the same results as the first round, and a
process with the cache switched off (VELOXQ_ALLOC_CACHE=0) returns the same
results again."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2501_19221_gb300 import instances as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2501_19221_gb300 import binding
    return binding


def _cases(B):
    """(name, make context, replicas, steps, schedule): the resident and
    streaming sparse paths, the FP32 dense step and the FP8 tensor-core step
    with its exact tensor-core readout."""
    ch = I.chimera_ising(4, 4, 4, seed=1)
    lat = I.cubic_lattice_ising(12, seed=2)
    Q1, c1 = I.sk_qubo(300, seed=3)
    Q2, c2 = I.sk_qubo(1024, seed=4)
    return [
        ("chimera_resident", lambda: B.veloxq_create_ising_csr(ch.n, ch.rowptr, ch.col, ch.val, ch.lin), 64, 300,
         B.make_schedule(path=1, readout_every=50)),
        ("lattice_stream", lambda: B.veloxq_create_ising_csr(lat.n, lat.rowptr, lat.col, lat.val, lat.lin), 64, 200,
         B.make_schedule(path=2, readout_every=50)),
        ("sk300_fp32", lambda: B.veloxq_create_dense(Q1, c1), 32, 100, B.make_schedule(readout_every=25)),
        ("sk1024_fp8", lambda: B.veloxq_create_dense(Q2, c2), 256, 100, B.make_schedule(prec=2, readout_every=0)),
    ]


def _run_all(B):
    out = {}
    for name, make, R, K, sched in _cases(B):
        ctx = make()
        r = B.veloxq_solve(ctx, R, K, sched, seed=11)
        ctx.destroy()
        out[name] = (float(r["E"]), r["x"].tobytes().hex(), [float(v) for v in r["E_per_replica"]])
    return out


def test_cached_blocks_give_identical_solves(B):
    first = _run_all(B)
    for _ in range(2):
        assert _run_all(B) == first


_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import tests.test_gpu_alloc_cache as T
from paper_2501_19221_gb300 import binding as B
print(json.dumps(T._run_all(B)))
"""


def test_cache_off_gives_the_same_solves(B):
    here = _run_all(B)
    env = dict(os.environ, VELOXQ_ALLOC_CACHE="0")
    res = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    there = json.loads(res.stdout.strip().splitlines()[-1])
    assert {k: [v[0], v[1], v[2]] for k, v in here.items()} == there
