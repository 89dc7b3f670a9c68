"""Replica parallelism across processes, on the host with gloo, world size 2:
seeds per rank, the max-over-ranks time and the best solution over ranks
(lowest energy, lowest rank on ties) that bench.py uses for N > 1. CPU only."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2501_19221_gb300 import replicas as RP  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 12
        if case == "distinct":
            E = [5.0, -3.0][rank]
        else:                                   # equal energies: the lowest rank wins
            E = -7.0
        x = np.full(n, rank + 1, dtype=np.uint8)
        Eb, xb, rb = RP.best_over_ranks(E, x, dist)
        tmax = RP.max_over_ranks([1.5, 4.25][rank], dist)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.concatenate([[Eb, rb, tmax, RP.rank_seed(7, rank)], xb.astype(np.float64)]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["distinct", "tie"])
def test_two_ranks_gloo(tmp_path, case):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, case, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    # every rank agrees on the winner and receives its vector
    assert np.array_equal(r0[:3], r1[:3]) and np.array_equal(r0[4:], r1[4:])
    if case == "distinct":
        assert r0[0] == -3.0 and r0[1] == 1 and np.all(r0[4:] == 2)
    else:
        assert r0[0] == -7.0 and r0[1] == 0 and np.all(r0[4:] == 1)
    assert r0[2] == 4.25                        # the longest rank's time
    assert r0[3] == 7 and r1[3] == 1007         # disjoint seeds per rank


def test_single_process_is_identity():
    x = np.arange(5, dtype=np.uint8)
    E, xb, r = RP.best_over_ranks(-1.5, x)
    assert E == -1.5 and r == 0 and np.array_equal(xb, x)
    assert RP.max_over_ranks(3.0) == 3.0
