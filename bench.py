#!/usr/bin/env python
"""Throughput of the batched Kaczmarz-type RZF precoders on one or more GB300s.

Workload (one step): the uneven batch of 512 near-field channels, Nt in
{1024, 2048, 4096}, K in U{32..256}, VR lengths round(U[0.1, 0.4] Nt), 16 QPSK
right-hand sides each (8192 precoders), solved by VR-OAHK in one persistent
launch (CUDA-graph replay of the queue reset + kernel), complex64 / FP32.
The same batch is also solved by plain GRK (paper's greedy rule) for the
"VR-OAHK vs GRK" comparison.  Every column of every channel is verified
afterwards against the FP64 oracle's closed-form RZF.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle (literal VR-OAHK, whole channels in parallel over the host cores) on
bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "converged precoders/s at rel.err 1e-5: VR-OAHK vs plain GRK; % HBM roofline"
N_INST = 512
NRHS = 16
TOL = 1e-6          # residual tolerance; every sampled column must verify at rel.err <= 1e-5
MAX_ITER = 1000
GRK_MAX_ITER = 100000
ERR_BAR = 1e-5

# DRAM traffic of one solver launch on this workload per launch configuration
# (ncu, one pass: dram__bytes_read.sum + dram__bytes_write.sum; the profiles/
# summary of this workload), valid only for the kernel sources it was measured
# on (their SHA-256 prefix).
TRAFFIC = {"sources_sha256": "27a80334db26c63f",
           # one J = 8 launch per step over the whole batch (read + write)
           "bytes_per_launch": {("tc", 8, 512): 1.02e9 + 0.16e9}}
KERNEL_SOURCES = ("paper_2501_10689_gb300/csrc/kz_ahk.cu", "paper_2501_10689_gb300/csrc/kz_device.cuh",
                  "paper_2501_10689_gb300/csrc/kz_internal.h")


def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def workload_desc():
    return ("batched VR-OAHK, one persistent launch: 512 near-field channels, Nt in {1024,2048,4096}, "
            "K in U{32..256}, VR round(U[0.1,0.4]*Nt), 16 QPSK RHS each, SNR 10 dB (xi = K/10), complex64")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=N_INST)
    ap.add_argument("--verify", type=int, default=N_INST, help="instances checked against the oracle")
    ap.add_argument("--rhs-per-cta", type=int, default=0, help="fix the launch instead of autotuning")
    ap.add_argument("--kernel", default="resident", choices=["resident", "tc"],
                    help="kernel used with --rhs-per-cta")
    ap.add_argument("--threads", type=int, default=512, help="threads per CTA used with --rhs-per-cta")
    ap.add_argument("--no-grk", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=6.0, help="seconds per CPU-baseline leg")
    ap.add_argument("--configs", action="store_true",
                    help="measure the other workloads (configs 1, 2, 4, 5) instead of the benchmark line")
    ap.add_argument("--only", default="config1,config2,config4,config5",
                    help="with --configs: comma-separated subset of config1, config2, config4, config5")
    ap.add_argument("--sweep", action="store_true",
                    help="fixed-T (T = 15) sum rates on the paper's scenario versus SNR and Nt (Figs. 3-4)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="kz_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
            p = [c.strip() for c in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle timing
def host_cores():
    """Cores this process may run on (the GPU machine's host cores)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_job(job):
    """One bounded piece of oracle work in a worker process: ``(index, method,
    columns)``.  Returns (columns solved, seconds).  The oracle runs as it
    stands; each worker is one single-threaded process."""
    import kzgen
    import oracle
    idx, method, cols = job
    inst = kzgen.config3_instance(idx)
    S = inst.S[:, :cols]
    t0 = time.perf_counter()
    if method == "vr_oahk":
        oracle.kaczmarz.solve(inst, S, "vr_oahk", tol=TOL, max_iter=MAX_ITER)
    elif method == "grk":
        oracle.kaczmarz.solve(inst, S, "grk", rule="paper", tol=TOL, max_iter=GRK_MAX_ITER)
    elif method == "rzf":
        oracle.rzf.rzf(inst.dense(), inst.xi, S)
    else:
        raise ValueError(method)
    return S.shape[1], time.perf_counter() - t0


class OraclePool:
    """Worker processes for the oracle, started with ``spawn`` (never forked
    from a process that has touched CUDA), each pinned to one BLAS thread."""

    def __init__(self, n):
        self.n = n
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = multiprocessing.get_context("spawn").Pool(n)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, jobs):
        """Wall seconds and columns of ``jobs`` spread over the workers."""
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_job, jobs, chunksize=1)
        return time.perf_counter() - t0, sum(c for c, _ in out)

    def close(self):
        self.pool.close()
        self.pool.join()


def serial_rate(method, seconds, start=0, cols=NRHS):
    """Single-core rate of one oracle method over whole instances (or ``cols``
    columns of each) until ``seconds`` have elapsed: (precoders/s, description)."""
    t0 = time.perf_counter()
    done = n = 0
    while True:
        c, _ = _oracle_job((start + n, method, cols))
        done += c
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done / el, f"{n} instances x {cols} columns ({done} precoders) from index {start}, {el:.1f} s"


def cpu_baselines(seconds, pool):
    """The oracle timed on the host cores: literal FP64 VR-OAHK on one core and
    on every core (whole channels in parallel), the closed-form Cholesky RZF and
    literal GRK (paper rule) on one core.  Each leg runs for about ``seconds``."""
    one, one_s = serial_rate("vr_oahk", seconds)
    n_jobs = max(pool.n, int(round(seconds * one * pool.n / NRHS)))
    wall, cols = pool.run([(k, "vr_oahk", NRHS) for k in range(n_jobs)])
    rzf, rzf_s = serial_rate("rzf", seconds / 2)
    grk, grk_s = serial_rate("grk", seconds / 2, cols=1)
    allc = cols / wall
    return {"value": allc, "unit": "precoders/s", "cores": pool.n, "kind": "oracle",
            "sample": f"literal FP64 VR-OAHK, {n_jobs} whole instances ({cols} precoders) of the batch over "
                      f"{pool.n} single-threaded processes, {wall:.1f} s wall",
            "single_core": {"value": one, "sample": one_s},
            "rzf_cholesky_single_core": {"value": rzf, "sample": rzf_s},
            "grk_single_core": {"value": grk, "sample": grk_s, "rule": "paper (p_i = |r_i|^2/||r||^2)"}}


def shard(rank, n):
    """Instance numbers solved by ``rank``: n per rank, disjoint across ranks
    (weak scaling; channels are independent, so no data-path collective)."""
    return list(range(rank * n, rank * n + n))


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (every rank calls this after the timed region)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, world, ms_per_step):
    """Precoders of all ranks per second of the slowest rank's step."""
    return n_per_rank * NRHS * world / (ms_per_step / 1000.0)


def batch_l2_note(insts):
    return "inputs larger than L2 (packed H of the batch is %.0f MB)" % (
        sum(int(i.vr_len.sum()) for i in insts) * 8 / 1e6)


def bench_config(args, insts):
    """The ``config`` of both arms: the workload and its solve parameters."""
    return {"workload": workload_desc(), "instances_per_gpu": args.instances, "nrhs": NRHS, "tol": TOL,
            "max_iter": MAX_ITER, "l2": batch_l2_note(insts)}


def run_reference(args):
    """The oracle as it stands on the host cores: each step solves a bounded
    sample of the batch's channels (literal FP64 VR-OAHK, whole channels, one
    single-threaded process per core) and is timed on the wall clock."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import kzgen
    cores = host_cores()
    pool = OraclePool(cores)
    per_step = 4 * cores  # channels per step: about four per core (evens out uneven channel sizes)
    nxt = 0
    for w in range(args.warmup):
        pool.run([(nxt + k, "vr_oahk", NRHS) for k in range(cores)])
        nxt += cores
    walls, cols = [], []
    for s in range(args.steps):
        wall, c = pool.run([(nxt + k, "vr_oahk", NRHS) for k in range(per_step)])
        nxt += per_step
        walls.append(wall)
        cols.append(c)
    pool.close()
    value = sum(cols) / sum(walls)
    insts = kzgen.config3(args.instances)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "precoders/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sum(walls) / args.steps,
            "ms_per_step_note": (f"measured wall time of one step; a step is a sample of {per_step} whole channels "
                                 f"({per_step * NRHS} precoders) of the batch, not the whole batch"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, insts),
            "cpu_baseline": {"value": value, "unit": "precoders/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: {per_step} whole channels of the batch (indices {args.warmup * cores}"
                                       f"..{nxt - 1} over the steps), literal FP64 VR-OAHK, {cores} single-threaded "
                                       "processes"},
            "e2e": {"value": value, "unit": "precoders/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU
def run_ours(args):
    import torch

    import __graft_entry__
    import kzgen
    import oracle
    from paper_2501_10689_gb300 import kzprecode as kp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()

    # CPU baseline first (before heavy GPU work; worker processes are spawned)
    gen_t0 = time.perf_counter()
    insts = [kzgen.config3_instance(i) for i in shard(rank, args.instances)]
    gen_s = time.perf_counter() - gen_t0
    cpu = None
    if rank == 0:
        pool = OraclePool(host_cores())
        cpu = cpu_baselines(args.cpu_seconds, pool)
        pool.close()

    # the batch's right-hand sides and outputs live in four contiguous device
    # buffers (each item a view), so the end-to-end leg moves them with one
    # copy per direction and buffer
    plans, items = [], []
    n_s = sum(NRHS * inst.K for inst in insts)
    n_x = sum(NRHS * inst.Nt for inst in insts)
    S_all = torch.empty(n_s, dtype=torch.complex64, device=dev)
    X_all = torch.empty(n_x, dtype=torch.complex64, device=dev)
    V_all = torch.empty(n_s, dtype=torch.complex64, device=dev)
    IT_all = torch.empty(len(insts) * NRHS, dtype=torch.int32, device=dev)
    R_all = torch.empty(len(insts) * NRHS, dtype=torch.float64, device=dev)
    os_, ox = 0, 0
    for b, inst in enumerate(insts):
        p = kp.plan_from_instance(inst, device=dev)
        plans.append(p)
        S = S_all[os_:os_ + NRHS * inst.K].view(NRHS, inst.K)
        S.copy_(kp.rhs_tensor(inst.S, device=dev))
        items.append(dict(plan=p, s=S, x=X_all[ox:ox + NRHS * inst.Nt].view(NRHS, inst.Nt),
                          v=V_all[os_:os_ + NRHS * inst.K].view(NRHS, inst.K),
                          iters=IT_all[b * NRHS:(b + 1) * NRHS], resid=R_all[b * NRHS:(b + 1) * NRHS], xi=inst.xi))
        os_ += NRHS * inst.K
        ox += NRHS * inst.Nt
    batch = kp.kz_batch_prepare(items, NRHS, "vr_oahk",
                                rhs_per_cta=args.rhs_per_cta if args.kernel == "resident" else 0)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    tuned = None
    if args.rhs_per_cta == 0:
        with torch.cuda.stream(stream):
            tuned = kp.kz_batch_tune(batch, "paper", TOL, MAX_ITER, 0)
    else:
        kp.kz_batch_set_launch(batch, args.kernel, args.rhs_per_cta, args.threads)

    def launch():
        kp.kz_precode_batched(batch, "paper", TOL, MAX_ITER, 0, status=status)

    # warm-up (also the CUDA graph capture)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            launch()
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        launch()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            a.record(stream)
            graph.replay()
            b.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(args.instances, world, ms_per_step)

    # ---- results of the last replay: iterations and verification
    st = int(status.item())
    iters = np.concatenate([it["iters"].cpu().numpy() for it in items])
    resid = np.concatenate([it["resid"].cpu().numpy() for it in items])
    verify_idx = list(range(0, args.instances, max(1, args.instances // max(args.verify, 1))))[: args.verify]
    max_err = max_err_v = 0.0
    rzf_ref = {}
    for k in verify_idx:  # every column of every checked channel, x and v
        inst = insts[k]
        rzf_ref[k] = V, X = oracle.rzf.rzf(inst.dense(), inst.xi, inst.S)
        x = items[k]["x"].cpu().numpy().T
        v = items[k]["v"].cpu().numpy().T
        max_err = max(max_err, float(np.max(oracle.rzf.rel_err(x, X))))
        max_err_v = max(max_err_v, float(np.max(oracle.rzf.rel_err(v, V))))

    # ---- roofline of the solver kernel (one launch per step)
    launch_now = (tuned if tuned else (args.kernel, args.rhs_per_cta, args.threads))
    tc = launch_now[0] == "tc"
    sumL = np.array([p.sum_len for p in plans], dtype=np.float64)
    # the orthogonal set's share (read in complex64 by every kernel)
    sumLF = np.array([float(np.sum(insts[b].vr_len[kp.kz_plan_query(p)[0]])) for b, p in enumerate(plans)])
    Nt = np.array([i.Nt for i in insts], dtype=np.float64)
    col_iters = iters.reshape(args.instances, NRHS).astype(np.float64)
    # per column-iteration (the workload's formula, complex64 H): H read twice
    # per iteration (the orthogonal rows' dot and update, the other rows'
    # residual and aggregate), shared by the 16 columns, plus the iterate
    # column read twice and written twice
    h_unit = 2.0 * sumL * 8.0 / NRHS
    unit_bytes = h_unit + 4.0 * Nt * 8.0
    alg_bytes = float(np.sum(col_iters * unit_bytes[:, None]))
    # the same count with H in the width the kernel reads it (the tensor-core
    # kernel: the V rows from the FP16 copy, 4 bytes an entry; the orthogonal
    # rows in complex64)
    h_unit_read = 2.0 * (sumLF * 8.0 + (sumL - sumLF) * (4.0 if tc else 8.0)) / NRHS
    read_bytes = float(np.sum(col_iters * (h_unit_read + 4.0 * Nt * 8.0)[:, None]))
    unit_flops = 16.0 * sumL  # residual + aggregate, 8 real flops per complex MAC
    alg_flops = float(np.sum(col_iters * unit_flops[:, None]))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        hbm_peak, peak_src = 6800.0, "fallback"
    achieved_gbs = alg_bytes / (ms_per_step / 1000.0) / 1e9
    h_bytes = float(np.sum(col_iters * h_unit[:, None]))
    h_gbs = h_bytes / (ms_per_step / 1000.0) / 1e9
    achieved_tflops = alg_flops / (ms_per_step / 1000.0) / 1e12
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA lanes x clock under load
    launches_per_step = kp.kz_batch_query(batch)["launches"]
    traffic = None
    if kernel_sources_sha() == TRAFFIC["sources_sha256"] and args.instances == N_INST:
        traffic = TRAFFIC["bytes_per_launch"].get(tuple(launch_now))
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                "traffic_note": "DRAM bytes per launch from ncu (one pass) on this workload and kernel build; "
                                "null when the kernel sources or launch differ",
                "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy)",
                "kernel": (f"kz_ahk_kernel<J = {launch_now[1]}, {launch_now[2] // 32} warps, tensor-core mode> "
                           f"(batched VR-OAHK; {launches_per_step} launch(es) per step: a second, concurrent "
                           "J = 4 launch only for channels whose J iterate columns do not fit)" if tc
                           else "kz_ahk_kernel (batched VR-OAHK)"),
                "alu_view": {"achieved_tflops": achieved_tflops, "fp32_fma_peak_tflops": alu_peak,
                             "frac": achieved_tflops / alu_peak},
                # the channel's bytes alone (the H term of the bytes above; the
                # iterate term stays in shared memory)
                "h_bytes_view": {"achieved": h_gbs, "unit": "GB/s", "frac": h_gbs / hbm_peak},
                # H counted in the width the kernel reads it
                "read_width_view": {"achieved": read_bytes / (ms_per_step / 1000.0) / 1e9, "unit": "GB/s",
                                    "frac": read_bytes / (ms_per_step / 1000.0) / 1e9 / hbm_peak,
                                    "note": "the V rows at 4 bytes an entry (FP16 copy) in the tensor-core kernel"},
                # what DRAM actually moved per launch (ncu), over the step time
                "dram_view": ({"achieved": traffic / (ms_per_step / 1000.0) / 1e9, "unit": "GB/s",
                               "frac": traffic / (ms_per_step / 1000.0) / 1e9 / hbm_peak} if traffic else None)}
    if tc and "bf16_tflops" in peaks:
        f16_peak = float(peaks["bf16_tflops"])  # dense FP16 runs at the BF16 rate
        roofline["tensor_view"] = {"achieved_tflops": achieved_tflops, "fp16_peak_tflops": f16_peak,
                                   "peak_source": "measured bf16_tflops (burst); dense FP16 runs at the BF16 rate",
                                   "frac": achieved_tflops / f16_peak}

    # ---- GRK on the same batch (comparison arm)
    grk = None
    if not args.no_grk:
        gitems = [dict(it, x=torch.empty_like(it["x"]), v=torch.empty_like(it["v"]),
                       iters=torch.empty_like(it["iters"]), resid=torch.empty_like(it["resid"])) for it in items]
        gbatch = kp.kz_batch_prepare(gitems, NRHS, "grk", rhs_per_cta=args.rhs_per_cta)
        gstatus = torch.zeros(1, dtype=torch.int32, device=dev)
        with torch.cuda.stream(stream):
            kp.kz_precode_batched(gbatch, "paper", TOL, GRK_MAX_ITER, 0, status=gstatus)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kp.kz_precode_batched(gbatch, "paper", TOL, GRK_MAX_ITER, 0, status=gstatus)
            b.record(stream)
        torch.cuda.synchronize(dev)
        gms = a.elapsed_time(b)
        gerr = 0.0
        for k in verify_idx:
            V, X = rzf_ref[k]
            gerr = max(gerr, float(np.max(oracle.rzf.rel_err(gitems[k]["x"].cpu().numpy().T, X))))
        gi = np.concatenate([it["iters"].cpu().numpy() for it in gitems])
        grk = {"value": args.instances * NRHS / (gms / 1000.0), "unit": "precoders/s", "ms_per_step": gms,
               "rule": "paper (p_i = |r_i|^2/||r||^2)", "mean_row_steps": float(gi.mean()),
               "max_rel_err_vs_fp64_rzf": gerr, "instances_checked": len(verify_idx), "status": int(gstatus.item()),
               "vroahk_speedup": (args.instances * NRHS / (ms_per_step / 1000.0)) / (args.instances * NRHS / (gms / 1000.0))}
        del gbatch

    # ---- end to end through the C-ABI with host buffers.  Every step copies
    # each channel's packed H in from pinned host memory and re-runs the
    # per-channel set-up on it (kz_plan_update: packing, row norms, inner
    # products of overlapping rows -- step A0), copies the right-hand sides in,
    # solves, and copies x, iterations and residuals out (one copy per buffer).
    # The same loop without the channel upload and set-up is reported beside it.
    H_pin = torch.from_numpy(np.concatenate([inst.H_packed for inst in insts])).pin_memory()
    H_dev = torch.empty(H_pin.shape, dtype=H_pin.dtype, device=dev)
    h_off = np.concatenate([[0], np.cumsum([p.sum_len for p in plans])]).astype(np.int64)
    S_pin = S_all.cpu().pin_memory()
    X_pin = torch.empty(X_all.shape, dtype=X_all.dtype).pin_memory()
    IT_pin = torch.empty(IT_all.shape, dtype=IT_all.dtype).pin_memory()
    R_pin = torch.empty(R_all.shape, dtype=R_all.dtype).pin_memory()
    d2h = X_pin.numel() * 8 + IT_pin.numel() * 4 + R_pin.numel() * 8

    # the channel upload in four item ranges of about equal size on a copy
    # stream, each range's set-up (kz_batch_update_items) starting once its
    # channels have arrived, while the next range uploads
    copy_stream = torch.cuda.Stream(device=dev)
    cum = np.concatenate([[0], np.cumsum([p.sum_len for p in plans])]).astype(np.int64)
    bounds = [0] + [int(np.searchsorted(cum, cum[-1] * q / 4.0)) for q in (1, 2, 3)] + [len(plans)]
    ranges = [(f, l - f) for f, l in zip(bounds[:-1], bounds[1:]) if l > f]

    def upload_and_update(pipelined):
        if not pipelined:
            H_dev.copy_(H_pin, non_blocking=True)
            update_plans(H_dev)
            return
        copy_stream.wait_stream(stream)  # the previous step's set-up has read H_dev
        for first, count in ranges:
            a_, b_ = int(cum[first]), int(cum[first + count])
            with torch.cuda.stream(copy_stream):
                H_dev[a_:b_].copy_(H_pin[a_:b_], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            stream.wait_event(ev)
            kp.kz_batch_update_items(batch, H_dev, first, count, stream=stream)

    def e2e_loop(new_channel, pipelined=True):
        ts = []
        with torch.cuda.stream(stream):
            for rep in range(2 + min(args.steps, 3)):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                if new_channel:
                    upload_and_update(pipelined)
                S_all.copy_(S_pin, non_blocking=True)
                launch()
                X_pin.copy_(X_all, non_blocking=True)
                IT_pin.copy_(IT_all, non_blocking=True)
                R_pin.copy_(R_all, non_blocking=True)
                b.record(stream)
                b.synchronize()
                if rep >= 2:
                    ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def update_plans(H):  # every channel's set-up in four launches
        kp.kz_batch_update(batch, H)

    ms_new = e2e_loop(True)
    ms_new_serial = e2e_loop(True, pipelined=False)
    ms_same = e2e_loop(False)
    # the set-up alone (channel already resident), for the breakdown
    with torch.cuda.stream(stream):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        update_plans(H_dev)
        b.record(stream)
        b.synchronize()
    ms_setup = a.elapsed_time(b)
    n_prec = args.instances * NRHS * world
    e2e = {"value": n_prec / (ms_new / 1000.0), "unit": "precoders/s",
           "h2d_bytes_per_step": H_pin.numel() * 8 + S_pin.numel() * 8, "d2h_bytes_per_step": d2h,
           "ms_per_step": ms_new,
           "note": "a new channel every step: H upload, per-channel set-up of every channel (kz_batch_update_items "
                   "over four item ranges, each starting once its channels have arrived while the next range uploads; "
                   "step A0), right-hand sides in, solve, x / iterations / residuals out",
           "setup_ms": ms_setup,
           "serial_upload_ms_per_step": ms_new_serial,
           "same_channel": {"value": n_prec / (ms_same / 1000.0), "unit": "precoders/s", "ms_per_step": ms_same,
                            "h2d_bytes_per_step": S_pin.numel() * 8, "d2h_bytes_per_step": d2h,
                            "note": "channel and set-up kept across steps: right-hand sides in, solve, results out"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "precoders/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f16" if tc else "f32", "data": "synthetic",
                "precision": ("complex64 storage; inside the correction-form iteration FP16 tensor-core "
                              "products with FP32 sums, from an FP16 copy of H (each row scaled by a power of "
                              "two at or above its norm), the correction held in FP16 scaled per column and "
                              "phi scaled per column; orthogonal half-step in FP32 on complex64 H; refresh "
                              "b = s - H H^H q through the overlap-pattern Gram matrix, true residual and "
                              "stopping test with compensated FP32 sums" if tc else
                              "complex64 storage, FP32 arithmetic; true residual with compensated sums"),
                "config": bench_config(args, insts),
                "launch": ({"kernel": tuned[0], "rhs_per_cta": tuned[1], "threads": tuned[2],
                            "chosen_by": "kz_batch_tune"}
                           if tuned else {"kernel": args.kernel, "rhs_per_cta": args.rhs_per_cta,
                                          "threads": args.threads, "chosen_by": "command line"}),
                "graph": "CUDA graph replay of queue reset + persistent kernel",
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * launches_per_step,
                "clocks": clocks, "grk": grk,
                "verify": {"instances_checked": len(verify_idx), "columns_checked": len(verify_idx) * NRHS,
                           "max_rel_err_vs_fp64_rzf": max_err, "max_rel_err_v_vs_fp64": max_err_v,
                           "bar": ERR_BAR, "ok": bool(max(max_err, max_err_v) <= ERR_BAR), "status_word": st,
                           "mean_iters": float(iters.mean()), "max_iters": int(iters.max()),
                           "max_resid": float(resid.max())},
                "gen_seconds": gen_s, "step_ms": step_ms}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- other workloads
def _time_ms(fn, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def run_configs(args):
    """One JSON line per (workload, method): time per solve, throughput and the
    error against the FP64 oracle.  Not the benchmark line."""
    import torch

    import __graft_entry__
    import kzgen
    import oracle
    from paper_2501_10689_gb300 import kzprecode as kp
    __graft_entry__.build()
    dev = torch.device("cuda", 0)

    def emit(d):
        print(json.dumps(d), flush=True)

    def solve(plan, S, xi, algo, tol, max_iter, kernel="auto", sel="paper"):
        return kp.precode(plan, S, xi, algo=algo, sel=sel, tol=tol, max_iter=max_iter, kernel=kernel, sync=False)

    only = set(args.only.split(","))

    # config 1: single column, latency.  us_per_iter_device is the slope of the
    # solve time between two fixed iteration counts (tol = 0), free of the
    # per-solve launch and set-up time
    inst = kzgen.config1()
    V, X = oracle.rzf.rzf(inst.dense(), inst.xi, inst.S)
    plan = kp.plan_from_instance(inst, device=dev)
    S = kp.rhs_tensor(inst.S, device=dev)
    for algo in (("rk_energy", "grk", "vr_ogrk", "gk", "ahk", "vr_oahk") if "config1" in only else ()):
        T1, T2 = (1000, 5000) if algo == "rk_energy" else (50, 250)
        for kernel in ("resident", "small"):  # auto picks the small-channel kernel here
            max_iter = 100000 if algo == "rk_energy" else 4000
            out = kp.precode(plan, S, inst.xi, algo=algo, tol=1e-6, max_iter=max_iter, kernel=kernel)
            err = float(oracle.rzf.rel_err(out["x"].cpu().numpy().T, X)[0])
            ms = _time_ms(lambda: solve(plan, S, inst.xi, algo, 1e-6, max_iter, kernel), reps=20)
            t1 = _time_ms(lambda: solve(plan, S, inst.xi, algo, 0.0, T1, kernel), reps=20)
            t2 = _time_ms(lambda: solve(plan, S, inst.xi, algo, 0.0, T2, kernel), reps=20)
            it = int(out["iters"][0].item())
            emit({"workload": "config1 Nt=256 K=16 1 column SNR 10 dB", "algo": algo, "kernel": kernel, "tol": 1e-6,
                  "us_per_solve": 1000 * ms, "iters": it, "us_per_iter": 1000 * ms / max(it, 1),
                  "us_per_iter_device": 1000 * (t2 - t1) / (T2 - T1), "rel_err": err})

    # config 2: 256 columns sharing one channel, every method, three SNRs
    for snr in ((0.0, 10.0, 20.0) if "config2" in only else ()):
        inst = kzgen.config2(snr)
        V, X = oracle.rzf.rzf(inst.dense(), inst.xi, inst.S)
        plan = kp.plan_from_instance(inst, device=dev)
        S = kp.rhs_tensor(inst.S, device=dev)
        for algo, kernel in (("rk_energy", "auto"), ("grk", "auto"), ("vr_ogrk", "auto"), ("ahk", "auto"),
                             ("ahk", "tc"), ("vr_oahk", "resident"), ("vr_oahk", "tc"), ("vr_oahk", "group")):
            max_iter = 400000 if algo.startswith("rk") else (40000 if "grk" in algo else 4000)
            for tol in (1e-5, 3e-6, 1e-6):
                out = kp.precode(plan, S, inst.xi, algo=algo, tol=tol, max_iter=max_iter, kernel=kernel)
                err = float(np.max(oracle.rzf.rel_err(out["x"].cpu().numpy().T, X)))
                if err <= ERR_BAR:
                    break
            ms = _time_ms(lambda: solve(plan, S, inst.xi, algo, tol, max_iter, kernel), reps=3)
            emit({"workload": f"config2 Nt=1024 K=64 256 columns SNR {snr:g} dB", "algo": algo, "kernel": kernel,
                  "tol": tol, "ms_per_solve": ms, "precoders_per_s": 256 / (ms / 1000.0),
                  "mean_iters": float(out["iters"].float().mean().item()), "max_rel_err": err})

    # config 4: large array, BF16-mixed vs complex64
    for inst in ([kzgen.config4()] if "config4" in only else []):
        V, X = oracle.rzf.rzf(inst.dense(), inst.xi, inst.S)
        S = kp.rhs_tensor(inst.S, device=dev)
        for prec, kernel in (("bf16", "resident"), ("c64", "resident"), ("c64", "tc"), ("c64", "group"), ("bf16", "group")):
            plan = kp.plan_from_instance(inst, prec=prec, device=dev)
            try:
                out = kp.precode(plan, S, inst.xi, algo="vr_oahk", tol=1e-6, max_iter=3000, kernel=kernel)
            except kp.KzError as e:  # e.g. the tensor-core kernel's iterate does not fit shared memory
                emit({"workload": "config4 Nt=16384 K=512 VR 1024-4096 64 columns", "algo": "vr_oahk", "prec": prec,
                      "kernel": kernel, "unsupported": str(e)})
                continue
            err = float(np.max(oracle.rzf.rel_err(out["x"].cpu().numpy().T, X)))
            ms = _time_ms(lambda: solve(plan, S, inst.xi, "vr_oahk", 1e-6, 3000, kernel), reps=3)
            emit({"workload": "config4 Nt=16384 K=512 VR 1024-4096 64 columns", "algo": "vr_oahk", "prec": prec,
                  "kernel": kernel, "tol": 1e-6, "ms_per_solve": ms, "precoders_per_s": 64 / (ms / 1000.0),
                  "mean_iters": float(out["iters"].float().mean().item()), "max_rel_err_vs_fp64": err})
    if "config5" not in only:
        return

    # config 5: forward + adjoint of the sum-rate loss over 64 channels
    from oracle import adjoint as oadj
    from paper_2501_10689_gb300 import autograd as kad
    chans = [kzgen.config5_instance(i) for i in range(64)]
    snr_lin = 10.0
    Hps = [torch.tensor(c.H_packed, device=dev) for c in chans]
    Ss = [kp.rhs_tensor(c.S, device=dev) for c in chans]

    def grad_all():
        total = 0.0
        for c, Hp0, S0 in zip(chans, Hps, Ss):
            Hp = Hp0.clone().requires_grad_(True)
            xi = torch.tensor(c.xi, dtype=torch.float32, device=dev, requires_grad=True)
            X5, V5 = kad.precode(Hp, xi, S0, c.vr_offset, c.vr_len, c.Nt, tol=1e-6)
            L = kad.sum_rate_loss(kad.dense_from_packed(Hp, c.vr_offset, c.vr_len, c.Nt), X5, snr_lin)
            L.backward()
            total += float(L.item())
        return total

    grad_all()
    t0 = time.perf_counter()
    grad_all()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    c = chans[0]
    L_ref, gH_ref, gxi_ref = oadj.reference_gradient(c, snr_lin)
    Hp = Hps[0].clone().requires_grad_(True)
    xi = torch.tensor(c.xi, dtype=torch.float32, device=dev, requires_grad=True)
    X5, V5 = kad.precode(Hp, xi, Ss[0], c.vr_offset, c.vr_len, c.Nt, tol=1e-6)
    kad.sum_rate_loss(kad.dense_from_packed(Hp, c.vr_offset, c.vr_len, c.Nt), X5, snr_lin).backward()
    gH = Hp.grad.cpu().numpy().astype(np.complex128)
    emit({"workload": "config5 64 channels Nt=2048 K=128 VR 256-1024 identity symbols, forward + adjoint",
          "mode": "per-channel", "grad_evals_per_s": 64 / dt, "seconds_per_batch": dt,
          "grad_H_rel_err_vs_fp64_autograd": float(np.linalg.norm(gH - gH_ref) / np.linalg.norm(gH_ref)),
          "grad_xi_rel_err": float(abs(xi.grad.item() - gxi_ref) / abs(gxi_ref)),
          "note": "per-channel autograd calls (plan set-up, forward solve, adjoint solve, loss in torch) timed "
                  "end to end on the host clock"})

    # per-user SINR and sum rate of the 64 precoders in one launch
    from oracle import sinr as osinr
    sr_items = []
    for c, Hp0, S0 in zip(chans, Hps, Ss):
        p = kp.kz_plan_create(c.K, c.Nt, c.vr_offset, c.vr_len, Hp0)
        sr_items.append(dict(plan=p, s=S0, x=torch.empty((c.K, c.Nt), dtype=torch.complex64, device=dev), v=None,
                             iters=torch.empty(c.K, dtype=torch.int32, device=dev),
                             resid=torch.empty(c.K, dtype=torch.float64, device=dev), xi=c.xi))
    srb = kp.kz_batch_prepare(sr_items, 128, "vr_oahk")
    kp.kz_precode_batched(srb, "paper", 1e-6, 2000, 0)
    sinr_all = torch.empty((64, 128), dtype=torch.float64, device=dev)
    rate_all = torch.empty(64, dtype=torch.float64, device=dev)
    ms = _time_ms(lambda: kp.kz_sum_rate_batched(srb, snr_lin, sinr_all, rate_all), reps=5)
    x0 = sr_items[0]["x"].cpu().numpy().T.astype(np.complex128)
    ref0 = osinr.sinr(chans[0].dense(), x0, snr_lin)
    emit({"workload": "config5 64 channels Nt=2048 K=128: per-user SINR and sum rate of the precoders (eq. (rate))",
          "ms_per_batch": ms, "channels_per_s": 64 / (ms / 1000.0),
          "max_rel_err_sinr_vs_fp64_oracle_same_precoder": float(np.max(np.abs(sinr_all[0].cpu().numpy() - ref0) / ref0)),
          "sum_rate_channel0_bits": float(rate_all[0].item())})

    # the precoder matrix of channel 0 by the subarray form (eq. (precoding2))
    # from its V, against the dense product H^H V (a cuBLAS complex GEMM), with
    # Table I's FLOP counts for the plan
    c0, p0 = chans[0], sr_items[0]["plan"]
    V0 = kp.precode(p0, Ss[0], c0.xi, algo="vr_oahk", tol=1e-6, max_iter=2000)["v"]
    Hd0 = torch.tensor(c0.dense().astype(np.complex64), device=dev)
    F_ref = torch.matmul(V0, Hd0.conj())
    ms_dense = _time_ms(lambda: torch.matmul(V0, Hd0.conj()), reps=20)
    Fm = torch.empty((c0.K, c0.Nt), dtype=torch.complex64, device=dev)
    for S_sub in (16, 64):
        ms_sub = _time_ms(lambda: kp.kz_precoder_matrix(p0, V0, S_sub, Fm), reps=20)
        err = float(torch.linalg.norm(Fm - F_ref) / torch.linalg.norm(F_ref))
        emit({"workload": "config5 channel 0 Nt=2048 K=128: precoder matrix F = [H_s]_{Q_s}^H [V]_{Q_s} (eq. (precoding2))",
              "subarrays": S_sub, "us_subarray_form": 1000 * ms_sub, "us_dense_cublas_HhV": 1000 * ms_dense,
              "rel_diff_vs_dense": err,
              "table1_flops_vr_oahk_T15": kp.kz_plan_flops(p0, "vr_oahk", S_sub, 15.0),
              "table1_flops_rzf": kp.kz_plan_flops(p0, "rzf", S_sub, 0.0)})

    # the same gradients through one batched forward and one batched adjoint
    pre = kad.BatchedPrecoder([(c.vr_offset, c.vr_len, c.Nt) for c in chans], 128, tol=1e-6, max_iter=2000)
    H_cat = torch.cat(Hps)
    S_cat = torch.cat([s.reshape(-1) for s in Ss])
    xi_cat = torch.tensor([c.xi for c in chans], dtype=torch.float32, device=dev)

    def grad_batched():
        H = H_cat.clone().requires_grad_(True)
        xb = xi_cat.clone().requires_grad_(True)
        X5, _ = pre(H, xb, S_cat)
        L = kad.sum_rate_loss_batched(pre.dense(H), X5.view(64, 128, 2048), snr_lin)
        L.backward()
        return H, xb

    grad_batched()
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        H, xb = grad_batched()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    gH = H.grad[:int(pre.h_off[1])].cpu().numpy().astype(np.complex128)
    emit({"workload": "config5 64 channels Nt=2048 K=128 VR 256-1024 identity symbols, forward + adjoint",
          "mode": "batched", "grad_evals_per_s": 64 / dt, "seconds_per_batch": dt,
          "grad_H_rel_err_vs_fp64_autograd": float(np.linalg.norm(gH - gH_ref) / np.linalg.norm(gH_ref)),
          "grad_xi_rel_err": float(abs(xb.grad[0].item() - gxi_ref) / abs(gxi_ref)),
          "launch": list(pre._launch),
          "note": "BatchedPrecoder: plan re-pack, one batched forward solve, loss in torch, one batched adjoint "
                  "(right-hand sides, solve, contractions), host clock, mean of 5"})


def run_sweep(args, T=15, seeds=4):
    """Sum rate (bits/s/Hz, eq. (rate)) of each method's precoder after T
    iterations on the paper's scenario (multipath, Bernoulli subarray VRs,
    K = 30, S = 20), versus SNR at Nt = 2000 and versus Nt at 10 dB; the RZF
    curve is the library's converged VR-OAHK (tol 1e-7).  Mean over `seeds`
    channels.  One JSON line per point."""
    import torch

    import __graft_entry__
    import kzgen
    from paper_2501_10689_gb300 import kzprecode as kp
    __graft_entry__.build()
    methods = (("vr_oahk", "paper"), ("vr_ogrk", "paper"), ("gk", "paper"), ("rk_swor", "paper"),
               ("rk_uniform", "paper"))

    def point(Nt, snr_db):
        acc = {}
        for seed in range(seeds):
            inst = kzgen.paper_scenario(500 + seed, Nt=Nt, snr_db=snr_db)
            plan = kp.plan_from_instance(inst)
            S = kp.rhs_tensor(inst.S)
            snr = 1.0 / inst.xi
            runs = [("rzf", "vr_oahk", "paper", 1e-7, 5000)] + [(a, a, s_, 0.0, T) for a, s_ in methods]
            for name, algo, sel, tol, it in runs:
                out = kp.precode(plan, S, inst.xi, algo=algo, sel=sel, tol=tol, max_iter=it, seed=seed)
                r = torch.empty(1, dtype=torch.float64, device="cuda")
                kp.kz_sum_rate(plan, out["x"], snr, rate=r)
                torch.cuda.synchronize()
                acc[name] = acc.get(name, 0.0) + float(r.item()) / seeds
        return acc

    for snr_db in (-10.0, 0.0, 10.0, 20.0, 30.0):
        print(json.dumps({"sweep": "snr", "Nt": 2000, "K": 30, "snr_db": snr_db, "T": T, "seeds": seeds,
                          "sum_rate": point(2000, snr_db)}), flush=True)
    for Nt in (1000, 2000, 4000, 8000):
        print(json.dumps({"sweep": "Nt", "Nt": Nt, "K": 30, "snr_db": 10.0, "T": T, "seeds": seeds,
                          "sum_rate": point(Nt, 10.0)}), flush=True)


def main():
    args = parse()
    if args.configs:
        run_configs(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
