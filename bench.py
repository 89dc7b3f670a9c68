#!/usr/bin/env python
"""Throughput benchmark of the VeloxQ hot path (ballistic simulated
bifurcation, arXiv:2501.19221 App. B) on one GB300.

A "step" of this benchmark is one complete solve of the workload: Philox
initial state, every integration step (field, fused update, walls, readout),
the exact readout energies, best-so-far and the argmin over replicas.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Metric: spin-updates/s = n * replicas * integration steps / solve time, with
the time-to-target of the mixed-precision forms against the plain FP32 form
on the same GPU and the roofline fraction of the dominant kernel.
Default workload: the dense SK instance n = 8192 (Q_ij ~ N(0,1)/sqrt(n)),
1024 replicas, 200 integration steps, the field in FP8 E4M3 on the tensor
cores (per-row scales for Qoff, two E4M3 terms for S, FP32 accumulation),
exact FP64-bounded readout energy after the last step.
With --gpus N (launched by torchrun) every rank solves its own replica of the
workload (weak scaling, no data-path collective); the time is the max over
ranks. --impl reference times the FP64 oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2501_19221_gb300 import instances as I

L2_FLUSH_BYTES = 256 << 20          # > 129 MB of L2

# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of
# the current kernel build (summaries and commands in profiles/); a kernel that
# changes after its capture must be removed from this table.
NCU_TRAFFIC = {
    ("k_resident", "chimera_c16"): 282_624,
    ("k_stream_step", "lattice_l100"): 4_104_791_000,
    ("k_stream_step", "hubo_chain_1e7"): 3_555_804_000,
    ("k_stream_step", "xorsat_3r3x_1e5"): 846_672_128,
    ("k_stream_step", "tile_planting_l300"): 314_659_499,
    ("k_adj_a+k_adj_b", "grad_l100"): 9_577_706_240,
    ("k_tc_step", "sk_n8192_fp8"): 291_477_740,     # per step: one 200-step launch, 58.30 GB / 200
    ("k_tc_step", "sk_n8192_bf16"): 435_910_845,    # per step: one 200-step launch, 87.18 GB / 200
    ("k_batch", "wishart_b512_k20"): 45_369_958_000,
    ("k_batch", "wishart_b512_k20_fp8"): 29_200_151_000,
}
SMEM_BYTES_PER_CLK_PER_SM = 128     # 32 banks x 4 bytes
FP32_LANES_PER_SM = 128
PREC_NAMES = {0: "fp32", 1: "bf16", 2: "fp8", 3: "fp8_one_term"}


def num_sms() -> int:
    """SMs of the current device (the derived peaks scale with it)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------- workloads
def workload(name: str, for_oracle: bool = False) -> dict:
    """The workload `name`. for_oracle: only what the oracle's timed sample
    needs (the full instance is not drawn when the sample is a smaller one)."""
    if name == "chimera_c16":
        sp = I.chimera_ising(16, 16, 4, seed=0)
        return {"name": name, "kind": "ising_csr", "sp": sp, "n": sp.n, "R": 1024, "K": 5000,
                "readout_every": 50, "desc": "Chimera C16 (16x16 K_{4,4} cells), J = +-1, h = 0, int8 CSR"}
    if name == "lattice_l100":
        sp = I.cubic_lattice_ising(100, seed=0)
        return {"name": name, "kind": "ising_csr", "sp": sp, "n": sp.n, "R": 256, "K": 400,
                "readout_every": 50, "desc": "periodic 3-D +-J lattice L=100, int8 CSR"}
    if name == "grad_l100":
        sp = I.cubic_lattice_ising(100, seed=0)
        return {"name": name, "kind": "grad", "sp": sp, "n": sp.n, "R": 256, "K": 400, "ckpt": 20,
                "readout_every": 0, "dt": 0.5, "knots": [0.0, 0.5, 1.0],
                "desc": "gradient of the mean relaxed energy w.r.t. dt, kappa and 3 schedule knots, periodic "
                        "3-D +-J lattice L=100, int8 CSR, 400 unrolled steps, checkpoint every 20"}
    if name in ("hubo_chain_1e7", "hubo_chain_5e7"):
        N = 10 ** 7 if name.endswith("1e7") else 5 * 10 ** 7
        inst = None if (for_oracle and N > 10 ** 7) else I.hubo_chain_3body(N, seed=0)
        n_red = N + max(N - 2, 0)             # one auxiliary spin per cubic term
        w = {"name": name, "kind": "hubo", "hubo": inst, "local": True, "n": n_red, "R": 8, "K": 200,
             "readout_every": 50,
             "desc": f"3-body +-Gaussian spin-glass chain (Sec. HUBO eq. nn), N = {N:.0e}, reduced to second order "
                     f"by eq. reduction (one auxiliary spin per cubic term, numbered next to it: n = {n_red}), "
                     "float CSR"}
        if N > 10 ** 7:
            # the oracle's sample: a chain of 1e6 spins drawn by the same recipe (the same local structure;
            # the whole instance does not fit one host process per core)
            w["oracle_chain"] = 10 ** 6
        return w
    if name == "xorsat_3r3x_1e5":
        x = I.xorsat_3r3x(10 ** 5, seed=0)
        return {"name": name, "kind": "hubo", "hubo": x.hubo, "E0_hubo": x.E0, "n": 2 * 10 ** 5, "R": 256,
                "K": 2000, "readout_every": 100,
                "desc": "planted 3-regular 3-XORSAT (Sec. 3R3X), 1e5 equations and variables, reduced to second "
                        "order by eq. reduction (n = 2e5), ground energy -1e5 by construction, float CSR"}
    if name in ("pegasus_p16", "zephyr_z12", "pegasus_p150", "zephyr_z150", "zephyr_z1750"):
        m = int(name.split("_")[1][1:])
        graph = "pegasus" if name.startswith("pegasus") else "zephyr"
        R, K = (1024, 1000) if m <= 16 else (2, 50) if m > 1000 else (256, 400)
        w = {"name": name, "kind": "qubo_csr", "graph": graph, "m": m, "R": R, "K": K, "readout_every": 50,
             "desc": f"random QUBO on the {graph.capitalize()} graph "
                     f"{'P' if graph == 'pegasus' else 'Z'}_{m}{'' if graph == 'pegasus' else ' (t = 4)'} "
                     "(Sec. " + ("Pegasus" if graph == "pegasus" else "Zephyr") + " topology), Q_ij, c_i ~ U[-1, 1), "
                     "float CSR"}
        if m > 1000:
            w["oracle_graph_m"] = 50          # the oracle's sample: Z_50 by the same recipe (same local structure)
        if not (for_oracle and m > 1000):
            w["sp"] = I.pegasus_qubo(m, seed=0) if graph == "pegasus" else I.zephyr_qubo(m, seed=0)
            w["n"] = w["sp"].n
        else:
            w["n"] = 4 * 4 * m * (2 * m + 1)
        return w
    if name in ("tile_planting_l300", "tile_planting_l300_easy"):
        p2 = 0.2 if name.endswith("easy") else 0.8
        tp = I.tile_planted_ising(300, p=(0.0, p2, 0.0, 1.0 - p2), seed=0)
        return {"name": name, "kind": "ising_csr", "sp": tp.sp, "E0_ising": tp.E0, "n": tp.sp.n, "R": 256,
                "K": 2000, "readout_every": 100,
                "desc": f"tile-planted periodic square lattice (Sec. Tile planting), L = 300 (n = 9e4), tile classes "
                        f"(0, {p2}, 0, {1 - p2:.1f}) ({'easy' if p2 < 0.5 else 'hard'} regime), gauge-hidden planted "
                        "ground state, int8 CSR"}
    if name == "lattice_l464":
        sp = I.cubic_lattice_ising(464, seed=0)
        return {"name": name, "kind": "ising_csr", "sp": sp, "n": sp.n, "R": 2, "K": 50,
                "readout_every": 50, "desc": "periodic 3-D +-J lattice L=464 (n ~ 1e8), int8 CSR"}
    if name in ("wishart_b512", "wishart_b512_fp8", "wishart_b128_k50", "wishart_b128_k50_fp8", "wishart_b512_k20",
                "wishart_b512_k20_fp8"):
        sizes = I.wishart_sizes(512, 100, 2000, seed=0)
        fp8 = name.endswith("fp8")
        small = "_b128_" in name
        if small:
            # the first 128 instances of the same batch, 50 steps: a case small enough for a full ncu capture
            sizes = sizes[:128]
        # the whole batch for 20 steps: the same sizes and L2 behaviour, short enough to capture
        K = 50 if small else 20 if "_k20" in name else 1000
        return {"name": name, "kind": "batch", "sizes": sizes, "n": int(sizes.sum()), "R": 64,
                "K": K, "readout_every": 0, "prec": 2 if fp8 else 1,
                "desc": ("the first 128 of the " if small else "") + "512 Wishart planted instances, n_i uniform in "
                        "[100, 2000], alpha 0.75, " + ("FP8 E4M3 field (S in two terms)" if fp8 else "BF16 field")
                        + ", one persistent launch" + (f", {K} steps" if K != 1000 else "")}
    if name in ("sk_n8192_fp32", "sk_n8192_bf16", "sk_n8192_fp8", "sk_n8192_fp8_one_term"):
        Q, c = I.sk_qubo(8192, seed=0)
        form = name[len("sk_n8192_"):]
        prec = {"fp32": 0, "bf16": 1, "fp8": 2, "fp8_one_term": 3}[form]
        what = {"fp32": "FP32 (CUDA cores)", "bf16": "BF16 (tensor cores)",
                "fp8": "FP8 E4M3 (tensor cores; per-row scales for Qoff, S as two E4M3 terms)",
                "fp8_one_term": "FP8 E4M3 (tensor cores; per-row scales for Qoff, S as one E4M3 term)"}[form]
        return {"name": name, "kind": "dense", "Q": Q, "c": c, "n": 8192, "R": 1024, "K": 200,
                "readout_every": 0, "prec": prec,
                "desc": f"SK n=8192, Q_ij ~ N(0,1)/sqrt(n), c = 0, seed 0; field in {what}, FP32 accumulation"}
    if name == "dense_n20":
        Q, c = I.dense_int_qubo(20, seed=0)
        return {"name": name, "kind": "dense", "Q": Q, "c": c, "n": 20, "R": 128, "K": 2000,
                "readout_every": 50, "desc": "dense int QUBO n=20, entries in [-8, 8]"}
    raise SystemExit(f"unknown workload {name}")


def batch_instances(w):
    """Wishart Ising couplings of the batch, as the Ising form -J (seeded per
    instance), and each instance's planted ground energy E0 = Tr(J~)/2."""
    if "inst" not in w:
        inst, e0 = [], []
        for m, n in enumerate(w["sizes"]):
            d = I.wishart_ising(int(n), 0.75, seed=1000 + m, dtype=np.float32)
            inst.append((-d["J"]).astype(np.float32))
            e0.append(0.5 * float(d["Jt_diag"].sum()))
        w["inst"], w["E0"] = inst, e0
    return w["inst"]


def reduce_hubo(B, w):
    """The library's second-order form of a third-order workload, kept in w;
    numbered for locality (each auxiliary spin next to its term) where the
    workload asks for it."""
    if "sp" not in w:
        inst = w["hubo"]
        red = B.veloxq_hubo3_reduce(inst.n, inst.h, inst.pairs, inst.triples, local=w.get("local", False))
        w["sp"] = I.SparseCoupling(red["n"], red["rowptr"], red["col"], red["val"], red["lin"])
        w["hubo_offset"] = red["offset"]
    return w["sp"]


def create(B, w, stream=None):
    if w["kind"] == "hubo":
        reduce_hubo(B, w)
    if w["kind"] == "qubo_csr":
        sp = w["sp"]
        return B.veloxq_create_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin, stream)
    if w["kind"] in ("ising_csr", "grad", "hubo"):
        sp = w["sp"]
        return B.veloxq_create_ising_csr(sp.n, sp.rowptr, sp.col, sp.val, sp.lin, stream)
    if w["kind"] == "batch":
        return [B.veloxq_create_ising_dense(J, None, stream) for J in batch_instances(w)]
    return B.veloxq_create_dense(w["Q"], w["c"], stream)


def input_arrays(w) -> list:
    if w["kind"] in ("ising_csr", "grad", "hubo", "qubo_csr"):
        sp = w["sp"]
        return [sp.rowptr, sp.col, sp.val, sp.lin]
    if w["kind"] == "batch":
        return list(batch_instances(w))
    return [w["Q"], w["c"]]


def oracle_problem(w):
    import oracle as O
    if w["kind"] == "hubo":
        inst = I.hubo_chain_3body(w["oracle_chain"], seed=0) if "oracle_chain" in w else w["hubo"]
        N, (qi, qj, qv), lin, _ = O.hubo3_reduce(inst.n, inst.h, inst.pairs, inst.triples)
        p, _ = O.ising_pairs_to_qubo(N, qi, qj, qv, lin)
        return p
    if w["kind"] in ("ising_csr", "grad"):
        sp = w["sp"]
        p, _ = O.ising_csr_to_qubo(sp.n, sp.rowptr, sp.col, sp.val, sp.lin)
        return p
    if w["kind"] == "qubo_csr":
        if "oracle_graph_m" in w:
            sp = I.zephyr_qubo(w["oracle_graph_m"], seed=0)
        else:
            sp = w["sp"]
        return O.problem_from_csr(sp.n, sp.rowptr, sp.col, sp.val.astype(np.float64), sp.lin)
    return O.problem_from_dense(w["Q"], w["c"])


def oracle_setup(w):
    """The oracle's problem and c0 = 2/rho for a workload (set-up, untimed).
    rho is the oracle's eigensolver value up to n = 6000; above, the timed
    sample only measures the arithmetic, and rho is the largest absolute row
    sum of Qoff (an upper bound of rho) so that set-up stays cheap."""
    import oracle as O
    p = oracle_problem(w)
    if p.n <= 6000:
        rho = O.spectral_radius(p)
    else:
        off = p.er != p.ec
        rowsum = np.bincount(p.er[off], weights=np.abs(p.ev[off]), minlength=p.n)
        rowsum += np.bincount(p.ec[off], weights=np.abs(p.ev[off]), minlength=p.n)
        rho = max(1e-12, 0.5 * float(rowsum.max()))
    return p, 2.0 / rho


def oracle_timed_run(w, p, c0, R_s: int, K_s: int, seed: int = 0, barrier=None) -> float:
    """Seconds of the FP64 oracle (single thread) on R_s replicas x the first
    K_s steps of the workload's schedule. With a barrier, the timed run starts
    when every process of the group is ready."""
    import oracle as O
    S0, Y0 = O.init_state(p.n, R_s, seed, 0.1)
    K = w["K"]
    knots = [0.0, (K_s - 1) / (K - 1) if K > 1 else 0.0]
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    if w["kind"] == "grad":
        O.bsb_grad(p, R_s, K_s, w["dt"], 1.0, c0, knots, S0, Y0)
    else:
        O.bsb_run(p, R_s, K_s, 0.5, 1.0, c0, knots, w["readout_every"], S0, Y0, method=w.get("method", "bsb"))
    return time.perf_counter() - t0


def oracle_sample_rate(w, R_s: int, K_s: int, seed: int = 0) -> tuple:
    """(spin-updates/s, seconds, variables) of one single-thread oracle sample."""
    p, c0 = oracle_setup(w)
    dt = oracle_timed_run(w, p, c0, R_s, K_s, seed)
    return p.n * R_s * K_s / dt, dt, p.n


def oracle_plan(w, target_s: float, max_R: int) -> tuple:
    """(R_s, K_s) for about target_s seconds of single-thread oracle work on
    the workload (at most max_R replicas and the workload's steps), from a
    one-replica calibration run of two steps."""
    rate0, _, n_s = oracle_sample_rate(w, 1, min(w["K"], 2))
    budget = max(1.0, target_s * rate0 / n_s)                   # replica-steps in the target
    R_s = int(min(w["R"], max_R, budget))
    K_s = int(min(w["K"], max(1, budget / max(1, R_s))))
    return max(1, R_s), K_s


def oracle_procs(w, R_s: int) -> int:
    """Processes of a replica-parallel oracle round: one per host core, fewer
    when their copies of the instance would not fit in half of the memory
    available (each holds the problem as coordinate lists, 24 B per stored
    entry, plus its state)."""
    cores = os.cpu_count() or 1
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    try:
        with open("/sys/fs/cgroup/memory.max") as f:
            v = f.read().strip()
            if v.isdigit():
                avail = min(avail, int(v)) if avail else int(v)
    except OSError:
        pass
    if "oracle_chain" in w:
        n_eff = 2 * int(w["oracle_chain"])
    elif "oracle_graph_m" in w:
        n_eff = 4 * 4 * w["oracle_graph_m"] * (2 * w["oracle_graph_m"] + 1)
    else:
        n_eff = int(w["n"])
    if "Q" in w:
        nnz = n_eff ** 2
    elif "sp" in w and "oracle_chain" not in w and "oracle_graph_m" not in w:
        nnz = int(np.asarray(w["sp"].rowptr)[-1]) + n_eff
    else:
        nnz = 8 * n_eff
    per_proc = 1.5 * 24 * nnz + 32 * n_eff * R_s + (512 << 20)
    if not avail:
        return cores
    return int(max(1, min(cores, 0.5 * avail // per_proc)))


def _crew_member(name, method, c0, seed, barrier, jobs, results):
    """A worker process of OracleCrew: builds the problem once, then runs the
    rounds it is given, each released by the shared barrier."""
    try:
        w = dict(workload(name, for_oracle=True), method=method)
        p = oracle_problem(w)
        while True:
            job = jobs.get()
            if job is None:
                break
            R_s, K_s = job
            results.put((seed, oracle_timed_run(w, p, c0, R_s, K_s, seed, barrier)))
    except Exception as e:                                   # reported by the parent
        results.put((seed, repr(e)))


class OracleCrew:
    """`procs` persistent oracle processes, one per host core, each with its
    own seed and its own copy of the problem (built once): a round runs the
    same sample in all of them at once, released together by a barrier
    (replica-parallel), and reports total spin-updates / the longest run.
    Processes are spawned, never forked from a process that touched the GPU;
    BLAS threads are pinned to one per process."""

    def __init__(self, w, procs: int):
        import multiprocessing as mp
        self.w, self.procs = w, procs
        p, self.c0 = oracle_setup(w)                      # rho once, in the parent
        self.n = p.n                                      # variables of the sampled instance
        ctx = mp.get_context("spawn")
        self.barrier = ctx.Barrier(procs, timeout=600)
        self.results = ctx.Queue()
        self.jobs = [ctx.Queue() for _ in range(procs)]
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.ps = [ctx.Process(target=_crew_member, args=(w["name"], w.get("method", "bsb"), self.c0, s,
                                                               self.barrier, self.jobs[s], self.results))
                       for s in range(procs)]
            for p in self.ps:
                p.start()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, R_s: int, K_s: int) -> tuple:
        for q in self.jobs:
            q.put((R_s, K_s))
        got = [self.results.get(timeout=1800) for _ in self.ps]
        bad = [r for _, r in got if not isinstance(r, float)]
        if bad:
            raise RuntimeError(f"oracle sample failed: {bad[0]}")
        wall = max(r for _, r in got)
        return self.n * R_s * K_s * self.procs / wall, wall

    def close(self):
        for q in self.jobs:
            q.put(None)
        for p in self.ps:
            p.join(timeout=60)


def oracle_parallel_rate(w, R_s: int, K_s: int, procs: int) -> tuple:
    """One replica-parallel round (see OracleCrew): (rate, seconds, processes)."""
    if procs <= 1:
        rate, dt, _ = oracle_sample_rate(w, R_s, K_s)
        return rate, dt, 1
    crew = OracleCrew(w, procs)
    try:
        rate, wall = crew.run(R_s, K_s)
    finally:
        crew.close()
    return rate, wall, procs


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="veloxq_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, gpu_index: int = 0) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    if int(parts[0]) != gpu_index:
                        continue
                    sms.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


# ----------------------------------------------------------------------------- our arm
class Runner:
    """One workload on the library: a context (or a batch of them) and a solve."""

    def __init__(self, B, w, stream, method: int = 0):
        self.B, self.w = B, w
        self.batch = w["kind"] == "batch"
        made = create(B, w)
        self.ctxs = made if self.batch else [made]
        for c in self.ctxs:
            B.veloxq_set_stream(c, stream.cuda_stream)
        self.grad = w["kind"] == "grad"
        if self.grad:
            self.sched = B.make_schedule(readout_every=0, dt=w["dt"], knots=w["knots"])
        else:
            self.sched = B.make_schedule(readout_every=w["readout_every"], prec=w.get("prec", 0), method=method)
        self.n_total = sum(c.info.n for c in self.ctxs)
        self.nnz_field = sum(c.info.nnz_field for c in self.ctxs)
        self.regular = False
        self.int8_couplings = False
        if "sp" in w:
            deg = np.diff(np.asarray(w["sp"].rowptr))
            self.regular = bool(deg.size > 0 and np.all(deg == deg[0]))
            v = np.asarray(w["sp"].val)
            # integer Ising couplings J map to 2 Qs = J: kept as int8 when |J| <= 127
            self.int8_couplings = bool(np.issubdtype(v.dtype, np.integer) and (v.size == 0 or np.abs(v).max() <= 127))

    def solve(self, seed, want_x=False):
        if self.grad:
            self.last_grad = self.B.veloxq_grad(self.ctxs[0], self.w["R"], self.w["K"], self.sched, seed,
                                                self.w["ckpt"])
            return self.last_grad["loss"]
        if self.batch:
            out = self.B.veloxq_solve_batch(self.ctxs, self.w["R"], self.w["K"], self.sched, seed=seed, want_x=want_x)
            self.last_batch_E = out["E"]
            return float(np.min(out["E"]))
        out = self.B.veloxq_solve(self.ctxs[0], self.w["R"], self.w["K"], self.sched, seed=seed, want_x=want_x)
        if want_x:
            self.last_x = out["x"]
        return out["E"]

    def timing(self):
        return self.B.veloxq_last_timing(self.ctxs[0])

    def destroy(self):
        for c in self.ctxs:
            c.destroy()


def roofline(B, w, runner, path, main_ms, main_launches):
    peaks, src = _peaks()
    n, R, K = runner.n_total, w["R"], w["K"]
    if runner.batch:
        # Q streamed per step (BF16 2 B, E4M3 1 B per entry) + state r/w (16 B) + the next operand
        # (2 B BF16, 1 B per E4M3 term) per variable-replica
        fp8 = w.get("prec", 1) != 1
        terms = 2 if w.get("prec", 1) == 2 and w.get("method", "bsb") != "pa" else 1
        qbytes = sum((1 if fp8 else 2) * int(m) * int(m) for m in w["sizes"])
        hbm = K * (qbytes + (16 + (terms if fp8 else 2)) * n * R)
        ach = hbm / (main_ms / 1e3) / 1e9
        return {"kernel": "k_batch", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": f"{src} hbm_gbs",
                "algorithmic_bytes_per_launch": hbm, "ms_per_launch": main_ms}
    if runner.grad:
        # one reverse step: k_adj_a reads s_k, y_k, lam_s, lam_y and writes the local g_s and lam_y (24 B per
        # variable-replica); k_adj_b reads the local g_s and the new lam_y (gathered, from L2 after one DRAM
        # read; g_phi = dt c0 lam_y is formed on the fly) and writes lam_s (12 B); each gathers through the
        # int8 couplings and columns once
        hbm_bytes = 36 * n * R + 2 * 5 * runner.nnz_field
        per = main_ms / K
        ach = hbm_bytes / (per / 1e3) / 1e9
        return {"kernel": "k_adj_a+k_adj_b", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": f"{src} hbm_gbs",
                "algorithmic_bytes_per_launch": hbm_bytes, "ms_per_launch": per,
                "launch": "one reverse step (k_adj_a, k_adj_b and the 1-block k_adj_reduce)"}
    if path == B.VELOXQ_PATH_RESIDENT:
        smem_bytes = (runner.nnz_field + 2 * n) * 4 * R * K
        sms = num_sms()
        peak = SMEM_BYTES_PER_CLK_PER_SM * sms * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9
        ach = smem_bytes / (main_ms / 1e3) / 1e9
        return {"kernel": "k_resident", "bound": "smem", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": f"derived: {SMEM_BYTES_PER_CLK_PER_SM} B/clk/SM x {sms} SMs x "
                               f"{peaks.get('sm_max_mhz', 2070.0)} MHz ({src} max clock)",
                "algorithmic_bytes_per_launch": smem_bytes, "ms_per_launch": main_ms}
    if path == B.VELOXQ_PATH_DENSE and w.get("prec", 0) in (1, 2, 3):
        return tc_roofline(w["prec"], w.get("method", "bsb"), n, R, main_ms / K)
    if path == B.VELOXQ_PATH_DENSE:
        return sgemm_roofline(n, R, main_ms / K)
    # state r/w + couplings (int8 2Qs or float Qs) and int32 columns, per step; the row
    # pointers are read only when rows differ in length (rows of equal length start at i * degree)
    per_nnz = 5 if runner.int8_couplings else 8
    hbm_bytes = 16 * n * R + per_nnz * runner.nnz_field + (0 if runner.regular else 8 * (n + 1))
    per = main_ms / max(1, main_launches)
    ach = hbm_bytes / (per / 1e3) / 1e9
    return {"kernel": "k_stream_step", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": f"{src} hbm_gbs",
            "algorithmic_bytes_per_launch": hbm_bytes, "ms_per_launch": per}


def tc_roofline(prec, method, n, R, per_ms):
    """Roofline of one tensor-core step (k_tc_step) on an n x n dense field
    with R replicas. BF16 and one-term FP8 run one GEMM of 2 n^2 R FLOP; FP8
    with S in two E4M3 terms runs two (Qop hi + Qop lo), 4 n^2 R FLOP against
    the FP8 peak, the same fraction as 2 n^2 R against the BF16 peak.
    Parallel Annealing's operand is exact in one term."""
    peaks, src = _peaks()
    terms = 2 if prec == 2 and method != "pa" else 1
    flops = 2.0 * n * n * R * terms
    peak = peaks["bf16_tflops"] * (2.0 if prec in (2, 3) else 1.0)
    ach = flops / (per_ms / 1e3) / 1e12
    return {"kernel": "k_tc_step", "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None,
            "peak_source": f"{src} bf16_tflops" + (" x 2 (FP8/BF16 nominal ratio)" if prec in (2, 3) else ""),
            "algorithmic_flops_per_launch": flops,
            "flops_per_launch_note": ("two E4M3 GEMMs per step (S as hi + lo terms): 2 x 2 n^2 R" if terms == 2
                                      else "one GEMM per step: 2 n^2 R"),
            "ms_per_launch": per_ms}


def sgemm_roofline(n, R, per_ms):
    """Roofline of one FP32 CUDA-core step (k_dense_step, plus k_dense_finish
    when the k-loop is split): 2 n^2 R FLOP against the FP32 FMA peak derived
    from the lane count and the maximum clock."""
    peaks, src = _peaks()
    sms = num_sms()
    flops = 2.0 * n * n * R
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ach = flops / (per_ms / 1e3) / 1e12
    return {"kernel": "k_dense_step", "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": ach / fp32_peak, "traffic": None,
            "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x {src} max clock",
            "algorithmic_flops_per_launch": flops, "ms_per_launch": per_ms}


def field_errors(B, stream, Q, R=1024, rows=96, seed=7):
    """Normwise error of the field F = Qoff S of each precision against an
    FP64 product, on `rows` sampled rows of a dense instance, S uniform in
    [-1, 1] (seeded). Returns {precision name: error}."""
    import torch
    n = Q.shape[0]
    ctx = B.veloxq_create_dense(Q, np.zeros(n))
    B.veloxq_set_stream(ctx, stream.cuda_stream)
    S = I.uniform_state(R, n, seed=seed)
    idx = np.sort(np.random.default_rng(1).choice(n, size=rows, replace=False))
    Qd = np.asarray(Q, dtype=np.float64)
    Qr = 0.5 * (Qd[idx, :] + Qd[:, idx].T)
    Qr[np.arange(rows), idx] = 0.0
    ref = S.astype(np.float64) @ Qr.T                                      # [R][rows]
    out = {}
    with torch.cuda.stream(stream):
        St = torch.as_tensor(S, device="cuda")
        F = torch.empty(R, n, device="cuda")
        ti = torch.as_tensor(idx, device="cuda")
        for prec, name in PREC_NAMES.items():
            B.veloxq_field_dev(ctx, R, prec, St, F)
            Fg = F[:, ti].cpu().numpy().astype(np.float64)
            out[name] = float(np.linalg.norm(Fg - ref) / np.linalg.norm(ref))
    ctx.destroy()
    return out


TTT_GRID = (10, 20, 30, 40, 50, 60, 80, 100, 120, 140, 160, 180, 200, 250, 300, 400)


def time_to_target(B, stream, seeds=32, n=8192, R=1024, K=200, method=0):
    """Time-to-target of the mixed-precision forms against the plain FP32
    form on the dense SK instance (n = 8192, 1024 replicas), for one
    integrator. The target E* is the median over `seeds` of the FP32 form's
    best energy after K steps (its success rate at K is about 0.5 by
    construction); a form reaches it at the smallest K' of TTT_GRID where at
    least half of the seeds end at or below E*. Times are CUDA-event times of
    whole solves (median over the seeds). The FP32 form's step is also given
    as its own roofline fraction (the SGEMM against the FP32 FMA peak), so
    that the ratios can be read against the quality of the baseline kernel."""
    import torch
    Q, c = I.sk_qubo(n, seed=0)
    ctx = B.veloxq_create_dense(Q, c)
    B.veloxq_set_stream(ctx, stream.cuda_stream)

    def solve(prec, steps, seed):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E = B.veloxq_solve(ctx, R, steps, B.make_schedule(prec=prec, readout_every=0, method=method), seed=seed,
                           want_x=False, want_per_replica=False)["E"]
        e1.record(stream)
        torch.cuda.synchronize()
        return E, e0.elapsed_time(e1)

    mname = {0: "bsb", 1: "asb", 2: "pa"}[method]
    out = {"workload": f"sk n={n}, {R} replicas, final readout only", "seeds": seeds, "method": mname,
           "grid": list(TTT_GRID)}
    with torch.cuda.stream(stream):
        solve(0, 4, 0)
        fp32, steps_ms = [], []
        for s in range(seeds):
            fp32.append(solve(0, K, 100 + s))
            steps_ms.append(B.veloxq_last_timing(ctx).ms_main)
        E_star = float(np.median([e for e, _ in fp32]))
        t32 = float(np.median([t for _, t in fp32]))
        out["E_star"] = E_star
        sg = sgemm_roofline(n, R, float(np.median(steps_ms)) / K)
        out["fp32"] = {"steps": K, "ms": t32, "success": float(np.mean([e <= E_star for e, _ in fp32])),
                       "step_ms": sg["ms_per_launch"], "step_tflops": sg["achieved"],
                       "step_frac_of_fp32_peak": sg["frac"], "step_peak_source": sg["peak_source"]}
        # Parallel Annealing's operand is exact in one E4M3 term: FP8 and FP8_ONE_TERM are the same run
        arms = [("bf16", 1), ("fp8", 2)] + ([] if method == 2 else [("fp8_one_term", 3)])
        for name, prec in arms:
            solve(prec, 4, 0)
            best = None
            for k2 in TTT_GRID:
                runs = [solve(prec, k2, 100 + s) for s in range(seeds)]
                p = float(np.mean([e <= E_star for e, _ in runs]))
                if p >= 0.5:
                    best = {"steps": k2, "ms": float(np.median([t for _, t in runs])), "success": p}
                    break
            out[name] = best
            out[f"speedup_{name}"] = (t32 / best["ms"]) if best else None
    ctx.destroy()
    return out


def time_to_target_batch(B, stream, seeds=4, K=1000, R=64):
    """Time-to-target of the batched forms (one persistent BF16 or FP8 launch
    for the 512 Wishart instances) against the plain FP32 form (each instance solved
    in turn with the library's own path choice: the resident kernel up to
    n = 512, the split-k SGEMM step above). Per instance, the target is the median
    over `seeds` of the FP32 form's best energy after K steps; a form's
    success is the fraction of (instance, seed) pairs at or below their
    target, and it reaches the targets at the smallest K' of a grid with
    success >= 0.5 (the FP32 form's own success is about 0.5 by
    construction). Times are CUDA-event times of the whole batch."""
    import torch
    w = workload("wishart_b512")
    ctxs = [B.veloxq_create_ising_dense(J, None) for J in batch_instances(w)]
    for cx in ctxs:
        B.veloxq_set_stream(cx, stream.cuda_stream)

    def run(prec, steps, seed):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sched = B.make_schedule(prec=prec, readout_every=0)     # the library's own path choice
        e0.record(stream)
        E = B.veloxq_solve_batch(ctxs, R, steps, sched, seed=seed, want_x=False)["E"]
        e1.record(stream)
        torch.cuda.synchronize()
        return np.asarray(E), e0.elapsed_time(e1)

    out = {"workload": f"Wishart batch of {len(ctxs)} instances, {R} replicas, final readout only", "seeds": seeds,
           "note": "one batched BF16 or FP8 launch against the FP32 form solving the instances one by one: "
                   "each ratio combines batching and precision"}
    with torch.cuda.stream(stream):
        fp32 = [run(0, K, 300 + s) for s in range(seeds)]
        E32 = np.stack([e for e, _ in fp32])                     # [seeds][instances]
        E_star = np.median(E32, axis=0)
        t32 = float(np.median([t for _, t in fp32]))
        out["fp32"] = {"steps": K, "ms": t32, "success": float(np.mean(E32 <= E_star[None, :]))}
        for name, prec in (("bf16", 1), ("fp8", 2)):
            run(prec, 4, 0)
            best = None
            for k2 in (100, 250, 500, K, 2 * K):
                runs = [run(prec, k2, 300 + s) for s in range(seeds)]
                Eb = np.stack([e for e, _ in runs])
                p = float(np.mean(Eb <= E_star[None, :]))
                if p >= 0.5:
                    best = {"steps": k2, "ms": float(np.median([t for _, t in runs])), "success": p}
                    break
            out[f"batched_{name}"] = best
            out[f"speedup_{name}"] = (t32 / best["ms"]) if best else None
    for cx in ctxs:
        cx.destroy()
    return out


def _tts99(t_ms: float, p: float):
    """Time to solution with 99% confidence from one run's time and its
    success probability: t ln(0.01) / ln(1 - p) (t itself once p >= 0.99)."""
    if p <= 0.0:
        return None
    if p >= 0.99:
        return t_ms
    return t_ms * math.log(0.01) / math.log(1.0 - p)


def tts_study(B, run, w, stream, seeds):
    """TTS99 against the known ground energy: the dense n = 20 instance
    (enumerated, tests/golden/dense_n20_ground.txt) over `seeds` solves, or
    each Wishart instance's planted energy over `seeds` batch solves."""
    import torch
    times, finals = [], []
    with torch.cuda.stream(stream):
        for i in range(seeds):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E = run.solve(5000 + i)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            finals.append(list(run.last_batch_E) if run.batch else E)
    t = float(np.median(times))
    if not run.batch:
        with open(os.path.join(ROOT, "tests", "golden", "dense_n20_ground.txt")) as f:
            E_min = [int(line.split()[1]) for line in f if line.startswith("E_min")][0]
        p = float(np.mean([E == E_min for E in finals]))
        return {"target": "ground energy by enumeration", "E_target": E_min, "runs": seeds, "p_success": p,
                "ms_per_run": t, "tts99_ms": _tts99(t, p)}
    hits = np.zeros(len(run.ctxs))
    for Es in finals:
        for m, (E, c, e0) in enumerate(zip(Es, run.ctxs, w["E0"])):
            hits[m] += (2 * E + c.info.ising_offset - e0) <= 1e-9 * abs(e0)
    p = hits / seeds
    tts = [_tts99(t, float(q)) for q in p if q > 0]
    return {"target": "planted energy of each instance", "runs": seeds, "ms_per_batch_run": t,
            "instances": len(p), "instances_solved": int(np.sum(p > 0)),
            "tts99_ms_median_over_solved": float(np.median(tts)) if tts else None}


def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2501_19221_gb300 import binding as B
    from paper_2501_19221_gb300 import replicas as RP

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    w = workload(args.workload)
    w["method"] = args.method
    R, K = w["R"], w["K"]
    method = {"bsb": 0, "asb": 1, "pa": 2}[args.method]
    stream = torch.cuda.Stream()
    run = Runner(B, w, stream, method)
    n = run.n_total
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    seed0 = RP.rank_seed(0, rank)
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            run.solve(seed0 + i)
        torch.cuda.synchronize()
        clocks = ClockSampler()
        if rank == 0:
            clocks.start()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        mains, launches, results = [], 0, []
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.add_(1.0)                                # write > L2 between timed steps (not timed)
            ev[i][0].record(stream)
            results.append(run.solve(seed0 + args.warmup + i, want_x=(i == args.steps - 1)))
            ev[i][1].record(stream)
            t = run.timing()
            mains.append(t.ms_main)
            launches += t.launches
            main_launches, path = t.main_launches, t.path
            gather = (t.stream_gather, t.stream_chunk) if hasattr(t, "stream_gather") else (0, 0)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if dist is not None:
            dist.barrier()
        clk = clocks.stop(0) if rank == 0 else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = RP.max_over_ranks(total_ms, dist, device="cuda")
    best_ranks = None
    if not run.batch and not run.grad:
        E_all, _, r_all = RP.best_over_ranks(results[-1], run.last_x, dist, device="cuda")
        best_ranks = {"E": E_all, "rank": r_all}
    value = world * n * R * K * args.steps / (total_ms / 1e3)

    # ---- end to end through the public API from pinned host buffers ----
    e2e_iters = max(1, min(args.steps, 3 if run.batch else 5))
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in input_arrays(w)]
    h2d = int(sum(a.nbytes for a in pinned))
    if w["kind"] in ("ising_csr", "grad", "hubo", "qubo_csr"):
        pw = dict(w)
        pw["sp"] = I.SparseCoupling(n, pinned[0], pinned[1], pinned[2], pinned[3])
    elif w["kind"] == "batch":
        pw = dict(w, inst=pinned, E0=w["E0"])
    else:
        pw = dict(w, Q=pinned[0], c=pinned[1])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_create = t_solve = 0.0
    for i in range(e2e_iters):
        ta = time.perf_counter()
        r2 = Runner(B, pw, stream, method)
        tb = time.perf_counter()
        r2.solve(seed0 + 77 + i, want_x=True)
        tc = time.perf_counter()
        r2.destroy()
        t_create += tb - ta
        t_solve += tc - tb
    e2e_s = (time.perf_counter() - t0) / e2e_iters
    nctx = len(run.ctxs)
    if run.grad:
        d2h = 8 * (2 + w["K"] + 8 + len(w["knots"]))             # loss, d_dt, d_c0, per-step and knot sums
    else:
        d2h = n + (0 if run.batch else 8 * R + 8 * R) + 32 * nctx   # best x, per-replica energies, argmin records
    e2e = {"value": world * n * R * K / e2e_s, "unit": "spin-updates/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
           "create_ms": t_create / e2e_iters * 1e3, "solve_call_ms": t_solve / e2e_iters * 1e3,
           "includes": "context creation (H2D copy, device ingest, spectral-radius estimate) + "
                       + ("gradient (forward, recompute, reverse)" if run.grad else "solve") + " + D2H of results"}

    roof = roofline(B, w, run, path, statistics.mean(mains), main_launches)
    roof["traffic"] = NCU_TRAFFIC.get((roof["kernel"], w["name"]))
    ferr = None
    if rank == 0 and w["kind"] == "dense" and w["n"] >= 1024:
        ferr = field_errors(B, stream, w["Q"], R=R)
        ferr = {"normwise_vs_fp64": ferr, "bar": 3e-2,
                "meets_bar": {k: bool(v <= 3e-2) for k, v in ferr.items()},
                "sample": f"96 sampled rows x {R} replicas, S uniform in [-1, 1] (seed 7), FP64 product of the "
                          "same rows as reference"}
    ttt = None
    if args.ttt and rank == 0:
        ttt = time_to_target(B, stream, seeds=args.ttt_seeds)
        ttt_pa = time_to_target(B, stream, seeds=args.ttt_seeds, method=2)
        ttt = {"bsb": ttt, "pa": ttt_pa}
    if args.ttt_batch and rank == 0:
        ttt_batch = time_to_target_batch(B, stream, seeds=4)
    else:
        ttt_batch = None
    tts = None
    if rank == 0 and w["name"] in ("dense_n20", "wishart_b512"):
        tts = tts_study(B, run, w, stream, seeds=32 if w["name"] == "dense_n20" else 4)

    # ---- CPU baseline: the oracle, single thread, bounded sample ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not run.batch:
        # calibrate on a short run, then time about 12 s of oracle work
        R_s, K_s2 = oracle_plan(w, 12.0, 4 if run.grad else 64)
        rate1, dt1, n_s = oracle_sample_rate(w, R_s, K_s2)
        # each process holds its own copy of the instance: fewer of them when memory is short
        procs = oracle_procs(w, R_s)
        rate, dt, used = oracle_parallel_rate(w, R_s, K_s2, procs)
        what = "reverse-mode gradient over" if run.grad else "solve of"
        inst = ("the same instance" if "oracle_chain" not in w and "oracle_graph_m" not in w else
                f"a chain of {w['oracle_chain']:.0e} spins by the same recipe (n = {n_s} after reduction)"
                if "oracle_chain" in w else
                f"the Zephyr graph Z_{w['oracle_graph_m']} by the same recipe (n = {n_s})")
        cpu = {"value": rate, "unit": "spin-updates/s", "cores": used, "kind": "oracle",
               "sample": f"{what} {R_s} replicas x first {K_s2} of {K} steps of {inst}, FP64, "
                         f"{used} independent processes at once (replica-parallel, {dt:.1f} s wall)",
               "single_thread": {"value": rate1, "sample_s": dt1}}

    if rank == 0:
        prec_name = {0: "f32", 1: "bf16", 2: "fp8e4m3", 3: "fp8e4m3"}[w.get("prec", 0)]
        line = {
            "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec_name,
            "data": "synthetic",
            "config": {"workload": w["name"], "instance": w["desc"], "n": n, "nnz_field": run.nnz_field,
                       "replicas": R, "integration_steps": K, "readout_every": w["readout_every"],
                       "path": {1: "resident", 2: "stream", 3: "dense"}.get(path, str(path)),
                       **({"stream_gather": gather[0], "stream_chunk_replicas": gather[1]} if path == 2 else {}),
                       "method": args.method, "field_operand": PREC_NAMES[w.get("prec", 0)],
                       "state": "f32", "l2": "flushed by a 256 MiB write before each timed step",
                       "parallelism": f"replicas-only x{world}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "field_error": ferr,
            "time_to_target": ttt,
            "time_to_target_batch": ttt_batch,
            "tts99": tts,
            "clocks": clk,
            "quality": {"best_energy_last_step": results[-1]},
            "wall_s_timed_region": wall,
        }
        if run.grad:
            g = run.last_grad
            line["quality"] = {"loss": g["loss"], "d_dt": g["d_dt"], "d_kappa": g["d_kappa"],
                               "d_knots": [float(v) for v in g["d_knots"]]}
            line["config"]["checkpoint_every"] = w["ckpt"]
            line["config"]["counts"] = ("forward steps: one gradient = forward, checkpointed recompute and "
                                        "reverse sweep over K steps")
        elif not run.batch:
            off = run.ctxs[0].info.ising_offset
            line["quality"]["best_ising_energy_last_step"] = 2 * results[-1] + off
            if "E0_ising" in w:
                e0 = w["E0_ising"]
                line["quality"]["planted_energy"] = e0
                line["quality"]["gap_to_planted"] = (2 * results[-1] + off - e0) / abs(e0)
            if w["kind"] == "hubo":
                # the third-order cost of the original spins is at most the reduced cost
                line["quality"]["hubo_energy_upper_bound"] = 2 * results[-1] + off + w["hubo_offset"]
                if "E0_hubo" in w:
                    e0 = w["E0_hubo"]
                    line["quality"]["planted_energy"] = e0
                    line["quality"]["gap_to_planted"] = (line["quality"]["hubo_energy_upper_bound"] - e0) / abs(e0)
            line["quality"]["best_over_ranks"] = best_ranks
        else:
            gaps = [(2 * E + c.info.ising_offset - e0) / abs(e0)
                    for E, c, e0 in zip(run.last_batch_E, run.ctxs, w["E0"])]
            line["quality"] = {"mean_gap_to_planted": float(np.mean(gaps)), "max_gap_to_planted": float(np.max(gaps)),
                               "instances_at_planted_energy": int(np.sum(np.array(gaps) <= 1e-9))}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.workload)
    w["method"] = args.method
    # each step about 2 s of oracle work: up to 32 replicas (4 for the gradient) x the first K_s steps
    R_s, K_s = oracle_plan(w, 2.0, 4 if w["kind"] == "grad" else 32)
    K_s = min(K_s, 1000)
    procs = oracle_procs(w, R_s)
    crew = OracleCrew(w, procs)
    try:
        for _ in range(args.warmup):
            crew.run(R_s, min(K_s, 20))
        times = []
        for _ in range(args.steps):
            _, dt = crew.run(R_s, K_s)
            times.append(dt)
    finally:
        crew.close()
    used = procs
    total = sum(times)
    value = crew.n * R_s * K_s * used * args.steps / total
    what = "reverse-mode gradient, " if w["kind"] == "grad" else ""
    sample = (f"{what}{R_s} replicas x first {K_s} of {w['K']} steps per step in each of {used} independent "
              f"processes at once, FP64 oracle")
    line = {"impl": "reference", "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "instance": w["desc"], "method": args.method, "n": w["n"], "replicas": w["R"],
                       "integration_steps": w["K"], "readout_every": w["readout_every"]},
            "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sk_n8192_fp8")
    ap.add_argument("--method", default="bsb", choices=["bsb", "asb", "pa"],
                    help="integrator (App. B): ballistic SB (default), adiabatic SB, Parallel Annealing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ttt", dest="ttt", action="store_true", default=True,
                    help="measure time-to-target of BF16/FP8 against FP32 on the dense SK instance (default on)")
    ap.add_argument("--no-ttt", dest="ttt", action="store_false")
    ap.add_argument("--ttt-seeds", type=int, default=32)
    ap.add_argument("--ttt-batch", action="store_true",
                    help="time-to-target of the batched BF16 form against the plain FP32 form on the Wishart batch")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        world = max(world, 1)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
