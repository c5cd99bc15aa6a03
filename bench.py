"""Benchmark: noisy-circuit shots/s of the tensor-network PTSBE hot path on GB300.

Workload (one "step"): the 30-qubit 1D brickwork circuit of depth 12 with
depolarizing (p = 0.005) then amplitude damping (gamma = 0.002) after every
gate; 4096 pre-sampled trajectories; 10^6 shots allocated in proportion to
trajectory weight; sampling in blocks of 10 qubits through conditional
marginals over the distinct prefixes.  A step = pre-sampling + UPV merge +
batched contraction + NBS sampling of all blocks (path planning is done once,
outside the timed region, as the paper's throughput definition excludes it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank runs the full workload on its own
trajectory seeds (weak scaling, no collective on the data path); value is the
shots of all ranks over the slowest rank's time.

Timing: the headline steps run uninstrumented except for CUDA events around
the launches of the dominant kernel class (found by a fully instrumented pass
of two steps before the timed region), which give its live average launch
duration for the roofline line.  Tensor-core peaks of the formats the
contraction uses (TF32, FP16) are measured here the same way as the BF16 peak
of MEASURED_PEAKS.json (torch.matmul 8192^3: best of 10, and back to back for
4 s).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "noisy-circuit shots/sec on 1 GB300, batched vs plain path, at stated error vs FP64"
# precision mode -> (library code, measured max norm-wise marginal error vs the complex128 oracle, where)
PRECISIONS = {
    "fp32": (0, "1.5e-5 on networks of the 30-qubit plan searched with 100 restarts, every block "
                "(tests/test_gpu_precision.py), 8.4e-6 on the 16-qubit grid slice; the benchmarked plan "
                "(1000 restarts) agreed with that plan to 6.1e-6 (FP16x3, 64 networks per block)"),
    "bf16x3": (1, "2.0e-5 on networks of the 30-qubit plan searched with 100 restarts "
                  "(tests/test_gpu_precision.py), 1.5e-5 on the 16-qubit grid slice; the benchmarked plan "
                  "(1000 restarts) agreed with that plan to 6.1e-6 (FP16x3, 64 networks per block)"),
    "fp16x3": (2, "1.4e-5 on networks of the 30-qubit plan searched with 100 restarts, every block "
                  "(tests/test_gpu_precision.py), 5.6e-6 on the 16-qubit grid slice; the benchmarked plan "
                  "(1000 restarts) agreed with that plan to 6.1e-6 on 64 networks per block, so within "
                  "2.0e-5 of FP64 there"),
}
# tensor-core steps run three MMAs per real product (hi*hi + hi*lo + lo*hi)
SPLIT_TERMS = 3
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes (read + write) over algorithmic bytes, measured by ncu on the
# 64-trajectory case of this workload (profiles/k_gemm_c2_64traj.md,
# profiles/k_pack_c2_64traj.md: two GEMM and two pack launches of the middle
# block); a class's roofline traffic per launch is this ratio times its
# algorithmic bytes per launch in the timed run.  Classes without a capture
# of the current kernel report null: both kernels changed after those captures
# (the GEMM epilogue's instance map for cached steps, the pack's outer-product
# operands), so the ratios are kept for reference only.
TRAFFIC_RATIO_CAPTURED = {"contract_gemm": (14.089 + 6.385) / (12.10 + 6.44),
                          "gemm_pack": (6.792 + 12.834) / (6.84 + 12.88)}
TRAFFIC_RATIO = {}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def c2_config():
    return W.config_c2()


# ----------------------------------------------------------- CPU oracle ----

def oracle_sample_run(cfg, n_traj_sample, shots_per_traj, seed_offset=0):
    """The oracle's pipeline (exact MPS contraction + NBS replay) for a bounded
    sample of trajectories of the workload; returns (shots, seconds)."""
    from oracle import mps, pts, sampling
    circ = cfg["circuit"]
    blocks = []
    s = 0
    for b in cfg["block_sizes"]:
        blocks.append((s, b))
        s += b
    t0 = time.perf_counter()
    kraus, _ = pts.presample(circ, n_traj_sample, cfg["seed"] + seed_offset)
    states = [mps.trajectory_mps(circ, kraus[i]) for i in range(n_traj_sample)]
    renv = {}

    def marg(j, traj, prefix):
        start, b = blocks[j]
        rows = []
        for t, p in zip(traj, prefix):
            key = (int(t), start + b)
            if key not in renv:
                renv[key] = states[int(t)].right_env(start + b)
            rows.append(states[int(t)].block_marginal(start, b, int(p), renv=renv[key]))
        return np.array(rows)

    tr, bits, cnt, levels, m = sampling.nbs_proportional(marg, blocks, cfg["seed"], n_traj_sample,
                                                         shots=[shots_per_traj] * n_traj_sample)
    return int(cnt.sum()), time.perf_counter() - t0


def _oracle_task(args):
    """One trajectory of the oracle pipeline (run in a worker process)."""
    k, shots_per_traj = args
    return oracle_sample_run(W.config_c2(), 1, shots_per_traj, seed_offset=k)


class OraclePool:
    """Worker processes for the CPU oracle, started with 'spawn' before any
    CUDA call, each with one BLAS thread, so that `cores` trajectories run at
    once on `cores` host cores."""

    def __init__(self, cores):
        import multiprocessing as mp
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.cores = cores

    def run(self, n_traj, shots_per_traj, seed0):
        """Wall time of n_traj oracle trajectories spread over the workers."""
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_task, [(seed0 + i, shots_per_traj) for i in range(n_traj)], chunksize=1)
        return sum(o[0] for o in out), time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(pool, cfg, shots_per_traj):
    """The oracle on a bounded sample: `pool.cores` trajectories per round on
    all worker processes (2 rounds), and one trajectory on one process."""
    pool.run(pool.cores, shots_per_traj, 50_000)          # warm-up (imports in the workers)
    n = 2 * pool.cores
    shots, sec = pool.run(n, shots_per_traj, 60_000)
    s1, t1 = pool.pool.apply(_oracle_task, ((70_000, shots_per_traj),))
    return {"value": shots / sec, "unit": "shots/s", "cores": pool.cores, "kind": "oracle",
            "sample": f"{n} trajectories x {shots_per_traj} shots of the workload on {pool.cores} worker "
                      f"processes (one BLAS thread each): exact MPS contraction + NBS replay, complex128",
            "single_thread": {"value": s1 / t1, "unit": "shots/s", "cores": 1,
                              "sample": f"1 trajectory x {shots_per_traj} shots on one process"}}


def run_reference(args, rank):
    """--impl reference: the CPU oracle as it stands, on bounded samples of the
    workload, trajectories spread over worker processes on the host cores."""
    if rank != 0:
        return
    cfg = c2_config()
    shots_per_traj = cfg["total_shots"] // cfg["n_traj"]
    pool = OraclePool(min(host_cores(), 32))
    n_sample = pool.cores
    try:
        for w in range(args.warmup):
            pool.run(n_sample, shots_per_traj, 1000 + 100 * w)
        times, shots = [], 0
        for k in range(args.steps):
            s_k, t_k = pool.run(n_sample, shots_per_traj, 10_000 + 100 * k)
            times.append(t_k)
            shots += s_k
    finally:
        pool.close()
    value = shots / sum(times)
    sample = (f"{n_sample} trajectories x {shots_per_traj} shots per step on {pool.cores} worker processes "
              f"(one BLAS thread each), exact MPS + NBS replay, complex128")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": {"workload": "c2_brickwork30_d12 (30 qubits, depth 12, dep 0.005 + AD 0.002, blocks 10/10/10)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": "shots/s", "cores": pool.cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def measure_tc_peaks(torch, sustain_s=4.0):
    """Dense TF32 and FP16 tensor-core throughput of this GPU, measured like the
    BF16 figures of MEASURED_PEAKS.json: torch.matmul 8192^3 (2 N^3 flops),
    best of 10 (burst) and back to back for a few seconds (sustained)."""
    N = 8192
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        for name, dt in (("tf32", torch.float32), ("fp16", torch.float16)):
            a = torch.randn(N, N, device="cuda", dtype=dt)
            b = torch.randn(N, N, device="cuda", dtype=dt)
            for _ in range(3):
                torch.matmul(a, b)
            best = 1e9
            for _ in range(10):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            torch.cuda.synchronize()
            n_it, t0 = 0, time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            while time.perf_counter() - t0 < sustain_s:
                for _ in range(20):
                    torch.matmul(a, b)
                n_it += 20
                torch.cuda.synchronize()
            e1.record()
            torch.cuda.synchronize()
            out[f"{name}_tflops"] = 2.0 * N ** 3 / best / 1e12
            out[f"{name}_tflops_sustained"] = 2.0 * N ** 3 * n_it / (e0.elapsed_time(e1) / 1e3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------- our arm ----

def run_nonprop(ptn, shard, torch, rank, n_traj, hypersamples, n=50, n_gates=200, steps=3, warmup=1):
    """Non-proportional NBS (Sec. III-B) on the paper's own circuit family
    (Sec. IV-B): an n-qubit random circuit of n_gates gates, blocks of 10 with
    one shot per prefix and a final block of up to 28 qubits harvested
    exhaustively (p(x | prefix) >= 1e-6), FP16x3.  Metric: unique labelled
    bitstrings (distinct (trajectory, bitstring) records) per second."""
    cfg = W.config_paper(n, n_gates)
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=hypersamples, est_traj=n_traj,
                             est_shots=n_traj)
    stream = torch.cuda.current_stream()
    times, recs, nets = [], 0, None
    for k in range(warmup + steps):
        tr = ptn.ptn_presample_trajectories(plan, shard.rank_seed(cfg["seed"], rank, 500 + k), n_traj)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        res = ptn.ptn_sample_nonprop(plan, tr, 77 + k, mode="exhaustive", threshold=1e-6,
                                     precision=ptn.PTN_PREC_FP16X3)
        b.record(stream)
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(a.elapsed_time(b) / 1e3)
            recs += res.n
            nets = res.nets_per_block
        del tr, res
    t = float(np.sum(times))
    return {"workload": f"{cfg['name']}: paper's random family (H X Y Z T Rx, 20% CX CY CZ CH CRx nearest "
                        f"neighbour, Pauli / two-qubit depolarizing noise p ~ U[0.02, 0.2]), {n_traj} trajectories, "
                        f"blocks {cfg['block_sizes']}, one shot per prefix, exhaustive final block "
                        "p(x | prefix) >= 1e-6, fp16x3",
            "value": recs / t, "unit": "unique bitstrings/s", "ms_per_step": 1e3 * t / len(times),
            "steps": len(times), "records_per_step": recs // len(times), "nets_per_block": nets,
            "contractions_per_s": float(sum(nets or [0])) * len(times) / t}


PRECISION_IDS = {"fp32": "PTN_PREC_FP32", "fp16x3": "PTN_PREC_FP16X3", "bf16x3": "PTN_PREC_BF16X3"}


def run_block_contraction(ptn, torch, hypersamples, b, batches, precisions, n=100, n_gates=600, reps=5):
    """Contraction time of one block of b qubits (the paper's contraction time
    per batch, Sec. V-B) on its 100-qubit, 600-gate family: every block of b
    qubits of a plan with uniform blocks of b (the remainder last) contracted for
    `batch` networks of distinct trajectories with random prefixes; mean
    CUDA-event time per block over the plan's full-size blocks.  Metric:
    contracted qubits per second, b / (time per network).  A block of more
    than 14 qubits can only be the final one (the conditional sampling of a
    non-final block holds 2^b entries in shared memory), so such a b is timed
    as the final block behind blocks of 10."""
    circ = W.config_paper(n, n_gates)["circuit"]
    rng = np.random.default_rng(n_gates)
    if b <= 14:
        bs = [b] * (n // b) + ([n % b] if n % b else [])
    else:   # blocks of more than 14 qubits are sampled only as the final block
        bs = [10] * ((n - b) // 10) + ([(n - b) % 10] if (n - b) % 10 else []) + [b]
    plan = ptn.ptn_plan_path(circ, bs, hypersamples=hypersamples, est_traj=max(batches), est_shots=max(batches))
    nw = ptn.words_of(n)
    stream = torch.cuda.current_stream()
    out = []
    for batch in batches:
        tr = ptn.ptn_presample_trajectories(plan, 4242, batch)
        nt = torch.arange(batch, dtype=torch.int32, device="cuda")
        marg = torch.empty((batch, 1 << b), dtype=torch.float32, device="cuda")
        Z = torch.empty(batch, dtype=torch.float64, device="cuda")
        for prec in precisions:
            pid = getattr(ptn, PRECISION_IDS[prec])
            per_block = []
            for j, (start, bj) in enumerate(plan.blocks):
                if bj != b:
                    continue
                pre = [int.from_bytes(rng.bytes(8 * nw), "little") & ((1 << start) - 1) for _ in range(batch)]
                npre = torch.from_numpy(ptn.int_to_words(pre, nw).copy()).cuda()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(reps + 2)]
                torch.cuda.synchronize()
                for a, e in ev:
                    a.record(stream)
                    ptn.ptn_contract_batch(plan, tr, j, nt, npre, marg, Z, precision=pid)
                    e.record(stream)
                torch.cuda.synchronize()
                per_block.append(float(np.mean([a.elapsed_time(e) for a, e in ev[2:]])))
            ms = float(np.mean(per_block))
            out.append({"b": b, "networks": batch, "precision": prec, "ms_per_block": ms,
                        "ms_per_block_min_max": [min(per_block), max(per_block)], "blocks_timed": len(per_block),
                        "us_per_network": 1e3 * ms / batch, "value": b * batch / (ms / 1e3),
                        "unit": "contracted qubits/s"})
        del tr, marg, Z
    return {"workload": f"paper_n{n}_g{n_gates}: paper's random family, blocks {bs}, each block contracted for "
                        "a batch of networks (distinct trajectories, random prefixes), CUDA events, "
                        f"{reps} timed of {reps + 2} calls per block",
            "lines": out}


MIXED_MAX_EST_S = 15.0   # per-circuit time budget of the mixed batch (modelled seconds)
REPLAN_FACTOR = 10       # circuits within this factor of the budget are planned again with this many times
                         # the restarts


def run_mixed_batch(ptn, shard, torch, dist, rank, world, hypersamples, workers, replan=False):
    """Plans (untimed), pre-samples (untimed) and runs the mixed batch through
    ptn_sample_shots_batch, once with one circuit in flight and once with
    `workers`; circuits beyond the planner's limits or the memory cap count as
    failed (TOO_LARGE), as do those whose modelled contraction time exceeds
    MIXED_MAX_EST_S seconds (the 6x5 grids: 20 s to 5e7 s modelled).  With
    several ranks, the circuits are shared out by modelled cost (longest
    first, no collective on the data path)."""
    cfgs = W.config_c3()
    plans, status = {}, {}
    t0 = time.perf_counter()
    for c in cfgs:
        try:
            plans[c["name"]] = ptn.ptn_plan_path(c["circuit"], c["block_sizes"], hypersamples=hypersamples,
                                                 est_traj=c["n_traj"], est_shots=c["total_shots"])
        except ptn.PtnError as e:
            status[c["name"]] = f"plan: {ptn.STATUS_NAMES.get(e.status, e.status)}"
    # replan: a circuit whose modelled time is over the budget but within
    # REPLAN_FACTOR of it is planned again with REPLAN_FACTOR times the greedy
    # restarts (the randomised search keeps finding cheaper paths for the 6x5 grids)
    replanned = {}
    for c in cfgs:
        if c["name"] not in plans:
            continue
        est = sum(b["est_time"] for b in plans[c["name"]].describe()["blocks"])
        if replan and MIXED_MAX_EST_S < est <= REPLAN_FACTOR * MIXED_MAX_EST_S:
            p2 = ptn.ptn_plan_path(c["circuit"], c["block_sizes"], hypersamples=REPLAN_FACTOR * hypersamples,
                                   est_traj=c["n_traj"], est_shots=c["total_shots"])
            est2 = sum(b["est_time"] for b in p2.describe()["blocks"])
            replanned[c["name"]] = [round(est, 2), round(est2, 2)]
            if est2 < est:
                plans[c["name"]] = p2
    planned = [c for c in cfgs if c["name"] in plans]
    costs = [sum(b["est_time"] for b in plans[c["name"]].describe()["blocks"]) for c in planned]
    mine = [planned[i] for i in shard.shard_items(costs, world)[rank]]
    items, names = [], []
    for c in mine:
        p = plans[c["name"]]
        tr = ptn.ptn_presample_trajectories(p, c["seed"], c["n_traj"], dedup=True, circuit_id=c["circuit_id"])
        items.append(dict(plan=p, traj=tr, seed=c["seed"], total_shots=c["total_shots"], circuit_id=c["circuit_id"]))
        names.append(c["name"])
    t_plan = time.perf_counter() - t0
    runs, first_error = {}, ""
    for nw in sorted({1, workers}):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ptn.ptn_sample_shots_batch(items, n_workers=nw, max_est_seconds=MIXED_MAX_EST_S)
        torch.cuda.synchronize()
        dt = shard.max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
        ok = [it for it, (st, _) in zip(items, out) if st == 0]
        shots = shard.sum_over_ranks(sum(it["total_shots"] for it in ok), dist, device="cuda")
        done = shard.sum_over_ranks(len(ok), dist, device="cuda")
        runs[nw] = {"seconds": dt, "completed": int(done), "shots": int(shots), "value": shots / dt}
        if nw == workers:
            for nm, (st, _) in zip(names, out):
                status[nm] = "ok" if st == 0 else f"run: {ptn.STATUS_NAMES.get(st, st)}"
            first_error = ptn.last_batch_error
        del out
    best = runs[workers]
    return {"workload": "64 circuits: 20-40-qubit 1D brickwork or 6x5 grid, depth 8-16, depolarizing 0.001-0.02, "
                        "16-8192 trajectories, 1e3-1e6 shots each",
            "value": best["value"], "unit": "shots/s", "workers": workers, "completed": best["completed"],
            "completed_fraction": best["completed"] / len(cfgs), "shots": best["shots"], "seconds": best["seconds"],
            "serial_seconds": runs[1]["seconds"], "plan_and_presample_seconds": t_plan,
            "replanned_modelled_s": replanned, "first_error_rank0": first_error,
            "status_rank0": {nm: status.get(nm, "other rank") for nm in (c["name"] for c in cfgs)}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--hypersamples", type=int, default=100,
                    help="greedy restarts of the path search for the sub-line workloads")
    ap.add_argument("--plan-hypersamples", type=int, default=1000,
                    help="greedy restarts of the path search for the 30-qubit workload (planning is untimed; "
                         "1000 restarts find a path with a 4x shallower dominant contraction than 100)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-traj", type=int, default=64,
                    help="trajectories timed on the plain per-trajectory path")
    ap.add_argument("--profile-range", action="store_true",
                    help="open a CUDA profiler range around the timed steps (for ncu --profile-from-start off)")
    ap.add_argument("--grad-calls", type=int, default=3,
                    help="timed ptn_expval_grad calls on the 16-qubit ansatz (0: skip)")
    ap.add_argument("--mixed-batch", type=int, default=4, metavar="WORKERS",
                    help="also run the 64-circuit mixed batch with this many concurrent circuits (0: skip)")
    ap.add_argument("--cache", type=int, default=1, choices=[0, 1],
                    help="intermediate caching across error sets (ptn_plan_opts.cache_intermediates)")
    ap.add_argument("--replan", type=int, default=0, choices=[0, 1],
                    help="mixed batch: plan circuits modelled within 10x of the time budget again with 10x the "
                         "restarts")
    ap.add_argument("--keep-products", type=int, default=0, choices=[0, 1],
                    help="1: materialise outer-product steps instead of forming them in the operand pack")
    ap.add_argument("--nonprop-traj", type=int, default=256,
                    help="trajectories of the non-proportional sub-lines on the paper's family (0: skip)")
    ap.add_argument("--nonprop-sizes", default="50x200,100x600,200x1000",
                    help="qubits x gates of the non-proportional sub-lines")
    ap.add_argument("--block-b", default="10,24",
                    help="block sizes of the per-block contraction sub-line at 100 qubits, 600 gates ('': skip)")
    ap.add_argument("--no-precision-lines", action="store_true",
                    help="skip the timed steps of the other tensor-core operand splits")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip measuring the TF32 / FP16 tensor-core peaks (the roofline then uses the "
                         "BF16 peak x the nominal format ratio)")
    ap.add_argument("--n-traj", type=int, default=0,
                    help="trajectories per step (default: the workload's 4096; smaller values are for profiling)")
    ap.add_argument("--total-shots", type=int, default=0,
                    help="shots per step (default: the workload's 1e6; smaller values are for profiling)")
    ap.add_argument("--mem-cap-gb", type=float, default=0.0,
                    help="device workspace cap (default: 40%% of free memory; small caps are for profiling)")
    ap.add_argument("--precision", default="fp16x3", choices=list(PRECISIONS),
                    help="tensor-core operand split (fp32: TF32 hi/lo; bf16x3 / fp16x3: 16-bit hi/lo)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    # the oracle's worker processes are spawned before the first CUDA call
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = OraclePool(min(host_cores(), 32))

    import torch
    torch.cuda.set_device(local)
    tc_peaks = {} if args.no_peaks else measure_tc_peaks(torch)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2604_08467_gb300 import ptn, shard

    cfg = c2_config()
    E = args.n_traj or cfg["n_traj"]
    M = args.total_shots or cfg["total_shots"]
    t_plan = time.perf_counter()
    plan = ptn.ptn_plan_path(cfg["circuit"], cfg["block_sizes"], hypersamples=args.plan_hypersamples,
                             est_traj=cfg["n_traj"], est_shots=cfg["total_shots"], mem_cap_bytes=args.mem_cap_gb * 1e9,
                             cache_intermediates=bool(args.cache), keep_products=bool(args.keep_products))
    t_plan = time.perf_counter() - t_plan
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    prec = PRECISIONS[args.precision][0]

    def step(k):
        tr = ptn.ptn_presample_trajectories(plan, shard.rank_seed(cfg["seed"], rank, k), E)
        res = ptn.ptn_sample_shots(plan, tr, cfg["seed"] + k, total_shots=M, precision=prec)
        return tr, res

    for w in range(args.warmup):
        tr, res = step(10_000 + w)
        del tr, res
    torch.cuda.synchronize()

    # ---- instrumented pass (every launch bracketed by events): the per-kernel
    # breakdown and the dominant kernel class; not part of the headline
    n_instr = 2
    ptn.ptn_stats_reset()
    ptn.ptn_stats_enable(True)
    instr_times = []
    for k in range(n_instr):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tr, res = step(20_000 + k)
        b.record(stream)
        torch.cuda.synchronize()
        instr_times.append(a.elapsed_time(b) / 1e3)
        del tr, res
    ptn.ptn_stats_enable(False)
    stats = ptn.ptn_stats_read()
    dominant = max(stats, key=lambda k: stats[k]["ms"])

    # ---- timed region: only the dominant class's launches carry events
    nets = None
    n_records = 0
    times = []
    ptn.ptn_stats_reset()
    ptn.ptn_stats_enable_only(dominant)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if args.profile_range:
            torch.cuda.profiler.start()
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tr, res = step(k)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
            nets = res.nets_per_block
            n_records = res.n
            del tr, res
        if args.profile_range:
            torch.cuda.profiler.stop()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
    ptn.ptn_stats_enable(False)
    live = ptn.ptn_stats_read()
    free_b, total_b = torch.cuda.mem_get_info()
    clocks = clk.summary()
    t_step = shard.max_over_ranks(float(np.mean(times)), dist, device="cuda")
    value = M * world / t_step

    # ---- the other tensor-core operand splits, same workload, uninstrumented
    other_prec = {}
    if not args.no_precision_lines:
        for pname, (pcode, perr) in PRECISIONS.items():
            if pname == args.precision:
                continue
            pt = []
            for k in range(max(2, min(args.steps, 4))):
                flush.zero_()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                tr = ptn.ptn_presample_trajectories(plan, shard.rank_seed(cfg["seed"], rank, 30_000 + k), E)
                res = ptn.ptn_sample_shots(plan, tr, cfg["seed"] + k, total_shots=M, precision=pcode)
                b.record(stream)
                torch.cuda.synchronize()
                pt.append(a.elapsed_time(b) / 1e3)
                del tr, res
            tp = shard.max_over_ranks(float(np.mean(pt)), dist, device="cuda")
            other_prec[pname] = {"value": M * world / tp, "unit": "shots/s", "ms_per_step": tp * 1e3,
                                 "steps": len(pt), "error_vs_fp64": perr}

    # ---- end to end through the public API, result copied to pinned host memory
    e2e_times = []
    d2h = 0
    h2d = 0
    for k in range(max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr, res = step(100 + k)
        t, bits, cnt = res.to_torch()
        ht = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
        hb = torch.empty(bits.shape, dtype=bits.dtype, pin_memory=True)
        hc = torch.empty(cnt.shape, dtype=cnt.dtype, pin_memory=True)
        ht.copy_(t, non_blocking=True)
        hb.copy_(bits, non_blocking=True)
        hc.copy_(cnt, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        if int(hc.sum()) != M:
            raise RuntimeError(f"step produced {int(hc.sum())} shots, expected {M}")
        d2h = t.numel() * 4 + bits.numel() * 8 + cnt.numel() * 8
        # host->device per step: the chunk index tables the runtime uploads per block
        h2d = 8 * E + sum(4 * n for n in res.nets_per_block) + 4 * E
        del tr, res
    e2e = {"value": M * world / float(np.mean(e2e_times)), "unit": "shots/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    # ---- plain per-trajectory path on a subset (same kernels, one trajectory per launch)
    plain = None
    if args.plain_traj > 0:
        tr = ptn.ptn_presample_trajectories(plan, shard.rank_seed(cfg["seed"], rank, 999_999), args.plain_traj)
        m_pt = M // E
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ptn.ptn_sample_shots(plan, tr, cfg["seed"], shots_per_traj=m_pt, max_traj_per_chunk=1,
                                   precision=ptn.PTN_PREC_FP32)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        plain = {"value": args.plain_traj * m_pt / tp, "unit": "shots/s",
                 "sample": f"{args.plain_traj} trajectories x {m_pt} shots, one trajectory per chunk"}
        del tr, res

    # ---- adjoint gradients: 16-qubit, 6-layer hardware-efficient ansatz, 192
    # angles, depolarizing 0.01, 1024 trajectories, O = mean_q Z_q Z_{q+1}
    grad = None
    if args.grad_calls > 0:
        c5 = W.config_c5()
        gplan = ptn.ptn_plan_path(c5["circuit"], c5["block_sizes"], hypersamples=args.hypersamples,
                                  est_traj=c5["n_traj"], grad_checkpoint=True)
        gtr = ptn.ptn_presample_trajectories(gplan, c5["seed"], c5["n_traj"], dedup=True)
        nq = c5["circuit"].n_qubits
        terms = [(1.0 / nq, (1 << q) | (1 << ((q + 1) % nq))) for q in range(nq)]
        th = c5["thetas"]
        gv = torch.empty(1, dtype=torch.float64, device="cuda")
        gg = torch.empty(th.size, dtype=torch.float64, device="cuda")
        ptn.ptn_expval_grad(gplan, gtr, terms, th, gv, gg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.grad_calls):
            ptn.ptn_expval_grad(gplan, gtr, terms, th + 1e-3 * k, gv, gg)
        torch.cuda.synchronize()
        tg = (time.perf_counter() - t0) / args.grad_calls
        grad = {"workload": "c5_hea16_l6: 16-qubit ansatz, 6 layers RY RZ + CZ ring, 192 angles, depolarizing 0.01, "
                            f"{c5['n_traj']} trajectories ({gtr.n_unique} distinct), O = mean Z_q Z_q+1, "
                            "checkpointed intermediates",
                "value": c5["n_traj"] / tg, "unit": "trajectory gradients/s", "ms_per_call": tg * 1e3,
                "expval": float(gv.item())}
        del gplan, gtr

    # ---- mixed-circuit batch: 64 circuits of 20-40 qubits, 1D or 6x5 grid,
    # depth 8-16, 16-8192 trajectories, 1e3-1e6 shots (the batching workload)
    nonprop = None
    if args.nonprop_traj > 0:
        nonprop = [run_nonprop(ptn, shard, torch, rank, args.nonprop_traj, args.hypersamples, n=int(a), n_gates=int(g))
                   for a, g in (x.split("x") for x in args.nonprop_sizes.split(",") if x)]
    block_contraction = None
    if args.block_b:
        block_contraction = [run_block_contraction(ptn, torch, args.hypersamples, int(b),
                                                   [1, 256] if int(b) <= 16 else [1],
                                                   ["fp32", "fp16x3"] if int(b) <= 16 else ["fp32"])
                             for b in args.block_b.split(",") if b]

    mixed = None
    if args.mixed_batch > 0:
        del plan          # frees the brickwork workspace so the batch gets the device memory
        mixed = run_mixed_batch(ptn, shard, torch, dist, rank, world, args.hypersamples, args.mixed_batch, replan=bool(args.replan))

    # ---- rooflines.  Tensor-core GEMMs are charged their algorithmic complex
    # flops (8 per complex multiply-add) against the dense peak of their input
    # format measured above (sustained: the kernel runs inside a long step),
    # divided by the three MMAs of the hi/lo split; every other kernel class is
    # charged algorithmic bytes against the measured HBM copy bandwidth.  The
    # headline is the dominant class, timed live inside the timed region; the
    # per-class breakdown comes from the instrumented pass.
    peaks, peak_src = load_peaks()
    fmt = {"fp32": "tf32", "fp16x3": "fp16", "bf16x3": "bf16"}[args.precision]
    if fmt == "bf16":
        tc_base, tc_note = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]), f"bf16 sustained ({peak_src})"
    elif f"{fmt}_tflops_sustained" in tc_peaks:
        tc_base, tc_note = tc_peaks[f"{fmt}_tflops_sustained"], f"{fmt} sustained (measured in this run)"
    else:
        ratio = 0.5 if fmt == "tf32" else 1.0
        tc_base = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * ratio
        tc_note = f"bf16 sustained x {ratio} nominal {fmt} ratio ({peak_src})"
    tc_peak = tc_base / SPLIT_TERMS

    def roof_of(name, s, steps, step_seconds):
        sec = s["ms"] / 1e3
        if name == "contract_gemm":
            ach = s["alg_flops"] / sec / 1e12 if sec > 0 else 0.0
            r = {"kernel": name, "bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s",
                 "peak_note": f"{tc_note} / {SPLIT_TERMS} split terms"}
        else:
            ach = s["alg_bytes"] / sec / 1e9 if sec > 0 else 0.0
            r = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "peak_note": f"hbm copy ({peak_src})"}
        tr = TRAFFIC_RATIO.get(name)
        old = TRAFFIC_RATIO_CAPTURED.get(name)
        r.update({"frac": r["achieved"] / r["peak"],
                  "traffic": tr * s["alg_bytes"] / max(s["timed_launches"], 1) if tr else None,
                  "traffic_unit": "bytes per launch (ncu DRAM/algorithmic ratio x algorithmic bytes)" if tr else None,
                  "traffic_note": (f"null: the kernel changed after its last ncu DRAM capture (DRAM/algorithmic "
                                   f"ratio then {old:.2f})") if (old and not tr) else None,
                  "launches_per_step": s["timed_launches"] / max(steps, 1),
                  "ms_per_step": s["ms"] / max(steps, 1),
                  "share_of_step": sec / max(step_seconds, 1e-12)})
        return r

    roofs = {k: roof_of(k, v, n_instr, sum(instr_times)) for k, v in stats.items() if v["ms"] > 0}
    roof = roof_of(dominant, live[dominant], args.steps, sum(times))
    roof["timing"] = "CUDA events around this class's launches inside the timed region"
    launches = sum(v["launches"] for v in live.values())

    cpu = None
    if pool is not None:
        cpu = cpu_baseline(pool, cfg, M // E)
        pool.close()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64" if args.precision == "fp32" else f"c64/{args.precision}",
                "data": "synthetic",
                "config": {"workload": "c2_brickwork30_d12: 30-qubit 1D brickwork depth 12, Haar U(2) + CZ, "
                                       "depolarizing 0.005 + amplitude damping 0.002 after every gate, "
                                       f"{E} trajectories, {M} shots proportional, blocks 10/10/10",
                           "device_mem_used_gb": (total_b - free_b) / 1e9,
                           "parallelism": f"replicas{world}", "l2": "flushed between steps (256 MB write)",
                           "nets_per_block": nets, "plan_seconds": t_plan, "plan_hypersamples": args.plan_hypersamples,
                           "cache_intermediates": bool(args.cache), "keep_products": bool(args.keep_products),
                           "precision": f"{args.precision}: complex64 storage, tensor-core operands split hi/lo "
                                        f"({args.precision}), fp64 CDF / log-probabilities",
                           "error_vs_fp64": PRECISIONS[args.precision][1]},
                "e2e": e2e, "plain_path": plain, "other_precisions": other_prec, "expval_grad": grad,
                "mixed_batch": mixed, "nonprop": nonprop, "block_contraction": block_contraction, "roofline": roof, "cpu_baseline": cpu,
                "contractions_per_s": float(sum(nets or [0])) * world / t_step,
                "distinct_records_per_s": float(n_records) * world / t_step,
                "gpu_launches": int(launches), "clocks": clocks, "tc_peaks_measured": tc_peaks,
                "kernels_instrumented": {
                    "note": f"{n_instr} extra steps with events around every launch "
                            f"({1e3 * float(np.mean(instr_times)):.1f} ms per step there)",
                    **{k: {"launches_per_step": r["launches_per_step"], "ms_per_step": r["ms_per_step"],
                           "share": r["share_of_step"], "achieved": r["achieved"], "unit": r["unit"],
                           "frac": r["frac"]} for k, r in roofs.items()}}}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
