#!/usr/bin/env python
"""HOTRG (beta, Delta) points/s at D_cut = 64 on B300.

Workload: distinct (beta, Delta) points of the q = 2 generalized XY model,
beta ~ U[0.5, 2.0], Delta ~ U[0, 1] (seed 20536, drawn one point at a time),
n_max = 4 (D0 = 9), D_cut = 64, 25 coarse-graining steps per point (2^25
sites), run through the C-ABI library (hotrg_run_batch on worker streams) in
the split-BF16 precision form with block-sparse (per U(1) charge block)
contractions.  One bench step = one pass of the whole hot path (initial
tensor, 25 HOTRG steps, closing trace) over `--points` points per GPU.
Several GPUs run independent replicas on distinct points (no collective on
the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--points P] [--impl ours|reference]

Besides the timed line: the plain FP64 form (block-sparse, FP64 FMA per
charge block) runs every timed point in full, which gives both the FP64-form
throughput and |d ln Z/N| of every timed point; the dense split and dense FP64
forms run one full point each; the timed form is compared with the stored
oracle results at D_cut = 64 (tests/golden); the FP64 CPU oracle is timed on a
bounded sample.  `--impl reference` times that oracle sample as the reference
arm (the oracle is test infrastructure; these are its only uses here).
"""

import argparse
import ctypes
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HOTRG (beta,Delta) points/s at D_cut=64, mixed vs FP64 GPU, |d lnZ/N|<=1e-9"
UNIT = "points/s"
D_CUT, N_MAX, N_STEPS = 64, 4, 25
WORKLOAD = ("gXY q=2 HOTRG points, beta~U[0.5,2.0], Delta~U[0,1] (seed 20536), n_max=4 (D0=9), "
            "D_cut=64, 25 one-axis steps per point (2^25 sites), split-BF16 tensor-core form")
WORKLOAD_BS = ", contractions per U(1) charge block"
# ncu DRAM traffic of the grouped coarse-contraction kernel (s1, s2, s3 of one full-size
# step), keyed by the hash of the kernel sources it was captured on: bytes per launch and
# the algorithmic bytes of the same launches (profiles/traffic_umma_grouped_dcut64.md)
KNOWN_TRAFFIC = {
    "9cc54c89a97f07b1": {"dram_to_algorithmic": 1.4138, "dram_bytes_per_full_step_launch": 0.9685e9,
                         "algorithmic_bytes_per_full_step_launch": 0.6850e9,
                         "source": "profiles/traffic_umma_grouped_dcut64.md (ncu dram__bytes_read/write.sum, "
                                   "the three coarse launches of a full-size D_cut=64 step)"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--points", type=int, default=6, help="points per bench step per GPU")
    ap.add_argument("--nstreams", type=int, default=0,
                    help="worker streams of the batch runner (0: autotuned over 1..min(max-streams, points) before "
                         "the warm-up; 1: points one after another on one stream)")
    ap.add_argument("--max-streams", type=int, default=6, help="largest worker-stream count the autotuner tries")
    ap.add_argument("--tiles", default="auto", choices=["auto", "128", "64"],
                    help="tile width of the tensor-core products (auto: hotrg_autotune_tiles on the first points)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    ap.add_argument("--block-sparse", type=int, default=1, choices=[0, 1],
                    help="1: contractions per U(1) charge block (the default form); 0: dense")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-form, dense-form, accuracy and CPU legs")
    ap.add_argument("--no-dense-fp64", action="store_true", help="skip the one dense FP64 point (~4 min)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d["bf16_tflops"], d["bf16_tflops_sustained"], d.get("hbm_gbs", 6465.2), "measured"
    return 1800.0, 1400.0, 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash():
    h = hashlib.sha256()
    for f in ["hotrg_umma.cu", "hotrg_blocks.cu", "internal.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2609_20536_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# Algorithmic (dense) work of a point, the unit of the CPU oracle's samples
# ---------------------------------------------------------------------------
def step_sizes(d0=2 * N_MAX + 1, d_cut=D_CUT, n_steps=N_STEPS):
    h = v = d0
    out = []
    for _ in range(n_steps):
        dp = min(d_cut, h * h)
        out.append((h, v, dp))
        h, v = v, dp
    return out


def step_flops(Dh, Dv, Dp):
    """Dense flops of one step as the oracle computes it: both environments (A, B, E,
    Eq. 2.12 regrouped) and the coarse contraction s1, s2, s3 (Eq. 2.16)."""
    env = 2 * (2 * 2 * Dh ** 3 * Dv ** 3 + 2 * Dh ** 4 * Dv ** 2)
    coarse = 2 * Dp * Dh ** 3 * Dv ** 2 + 2 * Dp * Dh ** 3 * Dv ** 3 + 2 * Dp ** 2 * Dh ** 2 * Dv ** 2
    return float(env), float(coarse)


def point_flops():
    return sum(sum(step_flops(*s)) for s in step_sizes())


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(beta, delta, nx=4):
    """One bounded sample of a point's work on the FP64 oracle, timed in full.

    Steps 1 and 2 run in full.  Step 3 (the first at full size, D_h = D_v =
    D' = 64, like every later step) runs its two environments and
    truncations in full and its coarse contraction on nx of the D' output
    columns x, then the norm.  Returns (seconds, units, detail): units is the
    sample's share of a whole point's algorithmic flops (the flop model of
    step_flops, the eigensolves not counted), so units / seconds is the
    oracle's throughput in points/s.
    """
    import numpy as np
    from oracle import gxy
    from oracle import hotrg as OH

    t_all = time.perf_counter()
    T = gxy.site_tensor(beta, delta, N_MAX)
    T = T / np.linalg.norm(T)
    q = gxy.leg_charges(N_MAX, "u1")
    qh, qv = q.copy(), q.copy()
    for _ in range(2):
        T, qh, qv, _, _ = OH.hotrg_step(T, qh, qv, D_CUT, "u1")
    Dh, Dv = T.shape[0], T.shape[2]
    Dp = min(D_CUT, Dh * Dh)
    qf = OH.fused_charges(qh, "u1")
    t0 = time.perf_counter()
    EL = OH.environment_left(T)
    ER = OH.environment_right(T)
    P, _, _, _ = OH.truncation(EL, qf, Dp)
    OH.truncation(ER, qf, Dp)
    t_env = time.perf_counter() - t0
    P3 = P.reshape(Dh, Dh, Dp)
    t0 = time.perf_counter()
    Tn = OH.coarse(np.ascontiguousarray(P3[:, :, :nx]), T, T)  # nx of the D' left output columns
    float(np.linalg.norm(Tn))
    t_coarse = time.perf_counter() - t0
    sec = time.perf_counter() - t_all
    sizes = step_sizes()
    work = sum(sum(step_flops(*s)) for s in sizes[:2])
    env3, coarse3 = step_flops(*sizes[2])
    work += env3 + coarse3 * nx / Dp
    units = work / point_flops()
    return sec, units, {"step3_env_trunc_s": t_env, "step3_coarse_s": t_coarse, "x_columns": nx,
                        "units_per_sample": units}


def blas_threads():
    """Threads of the BLAS pool: from threadpoolctl when it is importable, else from the
    thread-count variables the pool reads at start-up, else every host core."""
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var, "")
        if v.isdigit() and int(v) > 0:
            return int(v)
    return os.cpu_count()


def oracle_sample_one_thread(beta, delta):
    """The oracle sample with 1 of 64 coarse columns, timed in a child process whose BLAS and
    OpenMP pools are one thread wide (the variables are set before numpy loads, so no
    thread-control module is needed).  Returns (seconds, units, threads) or None."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, {root!r}); import bench; "
            "s, u, _ = bench.oracle_sample({b!r}, {d!r}, nx=1); "
            "print(json.dumps([s, u, bench.blas_threads()]))").format(root=ROOT, b=float(beta), d=float(delta))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=900)
        lines = [x for x in r.stdout.splitlines() if x.startswith("[")]
        if r.returncode != 0 or not lines:
            return None
        s1, u1, threads = json.loads(lines[-1])
        return float(s1), float(u1), int(threads)
    except Exception:  # a reported extra: its failure must not cost the bench line
        return None


SAMPLE_TEXT = ("each sample: one point's steps 1-2 in full, then step 3 (full size, D=64) with both environments "
               "and truncations in full and the coarse contraction on {nx} of 64 output columns; units = the "
               "sample's share of a point's algorithmic flops (dense flop model of the oracle's contractions, "
               "eigensolves uncounted)")


def run_reference(args):
    from paper_2609_20536_b300.workloads import headline_points
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pts = headline_points(args.warmup + args.steps, d_cut=D_CUT, n_max=N_MAX, n_steps=N_STEPS)
    for p in pts[: args.warmup]:
        oracle_sample(p.beta, p.delta)
    secs, units = 0.0, 0.0
    detail = None
    for p in pts[args.warmup:]:
        s, u, detail = oracle_sample(p.beta, p.delta)
        secs += s
        units += u
    value = units / secs
    cores = blas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("split-BF16 tensor-core form", "FP64 CPU oracle (numpy)"),
                       "samples_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": SAMPLE_TEXT.format(nx=4), "detail": detail},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2609_20536_b300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2609_20536_b300 import hotrg as H
    from paper_2609_20536_b300.workloads import headline_points

    prec = {"split": H.SPLIT_BF16, "fast": H.SPLIT_BF16_FAST, "fp64": H.FP64}[args.prec]
    stream = torch.cuda.current_stream()
    ctx = H.Context(stream=stream.cuda_stream)
    P = args.points
    n_total = (args.warmup + args.steps) * P * world
    pts = headline_points(n_total, d_cut=D_CUT, n_max=N_MAX, n_steps=N_STEPS)

    def batch_pts(step):
        base = (step * world + rank) * P
        return pts[base:base + P]

    def batch(step, pr=prec, bs=args.block_sparse):
        return [H.params(p.beta, p.delta, p.n_max, p.d_cut, p.n_steps, prec=pr, block_sparse=bs)
                for p in batch_pts(step)]

    tuned = None
    if args.nstreams == 0:
        # autotune the worker-stream count on one bench step's worth of points (untimed); more
        # streams than points per step would only idle
        best, secs = ctx.autotune_batch(batch(0), max_streams=max(1, min(args.max_streams, P)))
        tuned = {"chosen": best, "seconds_per_count": secs, "points": P}
        args.nstreams = best

    tiles = None
    if args.block_sparse and prec != H.FP64:
        if args.tiles == "auto":
            (te, tc), tsecs = ctx.autotune_tiles(batch(0), nstreams=args.nstreams)
            tiles = {"chosen_env_coarse": [te, tc], "seconds_128_128_128_64_64_128_64_64": tsecs}
        else:
            ctx.set_tiles(int(args.tiles), int(args.tiles))
            tiles = {"chosen_env_coarse": [int(args.tiles)] * 2}

    def run(plist):
        if args.nstreams > 1:
            return ctx.run_batch(plist, nstreams=args.nstreams)
        return ctx.run(plist)

    for s in range(args.warmup):
        run(batch(s))
    # the timed region runs as a user runs it: graph replay on the worker streams, no per-kernel
    # events (profiling replays no graphs); the counters are reset to count its launches
    H.hotrg_profile_enable(ctx.handle, False)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    results = []
    for s in range(args.warmup, args.warmup + args.steps):
        results += run(batch(s))  # host params in, host results out (synchronous C-ABI call)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    dev_ms = ev0.elapsed_time(ev1)
    launches = int(H.hotrg_profile_read(ctx.handle).launches)
    # the same points again with per-kernel-class CUDA events on the worker streams: the
    # breakdown and the roofline entries (kernel durations; this pass is not the timed value)
    H.hotrg_profile_enable(ctx.handle, True)
    tp = time.perf_counter()
    for s in range(args.warmup, args.warmup + args.steps):
        run(batch(s))
    profiled_s = time.perf_counter() - tp
    prof = H.hotrg_profile_read(ctx.handle)
    H.hotrg_profile_enable(ctx.handle, False)
    t = torch.tensor([dev_ms, wall], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_ms, wall = t[0].item(), t[1].item()
    points = args.steps * P * world
    value = points / (dev_ms / 1e3)
    e2e = points / wall
    bad = [r.status for r in results if r.status != 0]
    if bad:
        raise SystemExit(f"hotrg_run returned status {bad[0]}")

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    timed = [p for s in range(args.warmup, args.warmup + args.steps) for p in batch_pts(s)]
    roof, breakdown = roofline(H, prof, prec, args.block_sparse)
    breakdown["profiled_pass_s"] = profiled_s
    breakdown["note"] = ("CUDA-event time per region class summed over worker streams (regions overlap in time), "
                         "from a second pass over the timed points with profiling on (no graph replay)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec != H.FP64 else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + (WORKLOAD_BS if args.block_sparse else ""), "points_per_step": P,
                       "worker_streams": args.nstreams, "autotune": tuned, "tiles": tiles,
                       "d_cut": D_CUT, "n_max": N_MAX,
                       "n_steps": N_STEPS, "prec": args.prec, "block_sparse": args.block_sparse,
                       "parallelism": f"replicas x{world}",
                       "l2": "working set above L2: D^5 intermediates (8.6 GB dense arrays) every HOTRG step"},
            "roofline": roof, "breakdown": breakdown, "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": ctypes.sizeof(H.Params) * P * world,
                    "d2h_bytes_per_step": ctypes.sizeof(H.Result) * P * world,
                    "note": "host wall clock around the synchronous hotrg_run_batch / hotrg_run C-ABI call: "
                            "params in, results out"}}
    if not args.no_extras and world == 1:
        line.update(extras(H, ctx, timed, results, prec, args, value))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def roofline(H, prof, prec, bs):
    """Roofline entry of the coarse-contraction GEMM plus per-kernel-class fractions."""
    burst, sustained, hbm, src = peaks()
    ns_coarse = 5 if prec == H.SPLIT_BF16 else (3 if prec == H.SPLIT_BF16_FAST else 1)
    ns_env = 4 if prec == H.SPLIT_BF16 else (3 if prec == H.SPLIT_BF16_FAST else 1)
    prods = lambda ns: ns * (ns + 1) // 2 if prec != H.FP64 else 1  # noqa: E731  BF16 slice products
    coarse_ms, env_ms = prof.gemm_ms[1], prof.gemm_ms[0]
    fp64_equiv = prof.gemm_flops[1] / (coarse_ms / 1e3) / 1e12 if coarse_ms > 0 else 0.0
    achieved = fp64_equiv * prods(ns_coarse)
    kname = ("umma_grouped_kernel<5> (block-sparse coarse contraction s1/s2/s3)" if bs
             else "umma_gemm_kernel<5> (coarse contraction s1/s2/s3)")
    traffic = KNOWN_TRAFFIC.get(source_hash())
    calls = max(1, prof.gemm_calls[1])
    # algorithmic bytes of one coarse launch: the BF16 slices of every operand element once,
    # the output once (W, Z as FP32 pairs, T' in FP64: 8 bytes either way)
    alg_bytes = (prof.operand_elems[1] * 2 * ns_coarse + prof.output_elems[1] * 8) / calls
    roof = {"bound": "tensor", "kernel": kname,
            "achieved": achieved, "peak": sustained, "unit": "TFLOP/s", "frac": achieved / sustained,
            "peak_source": f"bf16 sustained, {src}",
            "achieved_is": (f"{prods(ns_coarse)} BF16 slice products x 2MNK per contraction (per charge block, "
                            "summed over blocks, when block-sparse) / CUDA-event time on its stream, in a profiled "
                            "pass over the timed points"),
            "slice_products": prods(ns_coarse), "fp64_equivalent_tflops": fp64_equiv,
            "kernel_share_of_steps": coarse_ms / prof.step_ms if prof.step_ms else None,
            "algorithmic_bytes_per_launch": alg_bytes if bs else None,
            # the ncu ratio of DRAM to algorithmic bytes at a full-size step, applied to this run's
            # algorithmic bytes per coarse launch (traffic grows with the block elements processed)
            "traffic": traffic["dram_to_algorithmic"] * alg_bytes if (traffic and bs) else None,
            "traffic_source": traffic["source"] if traffic else "no ncu capture of this kernel build"}
    kernels = {}
    if env_ms > 0:
        env_tf = prof.gemm_flops[0] / (env_ms / 1e3) / 1e12 * prods(ns_env)
        kernels["env_grouped_gemm"] = {"bound": "tensor", "achieved_tflops": env_tf, "frac": env_tf / sustained,
                                       "slice_products": prods(ns_env),
                                       "share_of_steps": env_ms / prof.step_ms if prof.step_ms else None}
    if prof.slice_ms > 0 and bs and prec != H.FP64:
        # each operand element is read once (8 bytes: FP64 or an FP32 pair) and written as NS BF16 slices
        sb = prof.operand_elems[0] * (8 + 2 * ns_env) + prof.operand_elems[1] * (8 + 2 * ns_coarse)
        gbs = sb / (prof.slice_ms / 1e3) / 1e9
        kernels["slicers"] = {"bound": "hbm", "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                              "algorithmic_bytes": sb, "share_of_steps": prof.slice_ms / prof.step_ms}
    if prof.steps:
        kernels["eigensolve"] = {"bound": "latency", "ms_per_step": prof.eig_ms / prof.steps,
                                 "share_of_steps": prof.eig_ms / prof.step_ms if prof.step_ms else None}
    roof["kernels"] = kernels
    breakdown = {"coarse_gemm_ms": coarse_ms, "env_gemm_ms": env_ms, "slice_ms": prof.slice_ms,
                 "eig_ms": prof.eig_ms, "eig_parts_ms": {"jacobi_small": prof.eig_part_ms[0],
                                                          "subspace_fp32": prof.eig_part_ms[1],
                                                          "rayleigh_ritz": prof.eig_part_ms[2],
                                                          "select_projector": prof.eig_part_ms[3]},
                 "steps_ms": prof.step_ms, "hotrg_steps": prof.steps,
                 "coarse_block_flops": prof.gemm_flops[1], "env_block_flops": prof.gemm_flops[0],
                 "note": "CUDA-event time per region class summed over worker streams (regions overlap in time)"}
    return roof, breakdown


def extras(H, ctx, timed, results, prec, args, value):
    """FP64 form and accuracy on every timed point, dense forms on one point each, the oracle
    goldens, the CPU oracle baseline."""
    import torch
    out = {}
    bs, ns = args.block_sparse, args.nstreams
    # the plain FP64 form (per charge block when the timed form is) on every timed point, in full,
    # through the same batch runner and stream count
    fp = [H.params(p.beta, p.delta, p.n_max, p.d_cut, p.n_steps, prec=H.FP64, block_sparse=bs) for p in timed]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rf = ctx.run_batch(fp, nstreams=ns) if ns > 1 else ctx.run(fp)
    tf = time.perf_counter() - t0
    fp_value = len(fp) / tf
    out["fp64_form"] = {"value": fp_value, "unit": UNIT, "points": len(fp), "n_steps": N_STEPS,
                        "block_sparse": bs, "worker_streams": ns, "s_per_point": tf / len(fp),
                        "mixed_vs_fp64": value / fp_value,
                        "note": "plain FP64 form (FP64 FMA contractions, FP64 Jacobi on every block) on the same "
                                "points as the timed form, full length, host wall clock around the synchronous "
                                "call"}
    d = [r.lnz_per_site - f.lnz_per_site for r, f in zip(results, rf)]
    acc = {"vs_fp64_form": {"max_abs_dlnz": max(abs(x) for x in d), "points": len(d), "d_cut": D_CUT,
                            "n_steps": N_STEPS, "over_1e-9": sum(abs(x) > 1e-9 for x in d),
                            "per_point": [float("%.3g" % x) for x in d]}}
    # the stored oracle results (tests/golden, written by the FP64 CPU oracle alone)
    gold = []
    for f in sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "oracle_*.json"))):
        g = json.load(open(f))
        r = ctx.run([H.params(g["beta"], g["delta"], g["n_max"], g["d_cut"], g["n_steps"], prec=prec,
                              block_sparse=bs)])[0]
        gold.append({"case": g["case"], "d_cut": g["d_cut"], "n_steps": g["n_steps"],
                     "dlnz": r.lnz_per_site - g["lnz_per_site"]})
    if gold:
        acc["vs_oracle"] = {"max_abs_dlnz": max(abs(x["dlnz"]) for x in gold), "cases": gold}
    out["accuracy"] = acc
    # dense forms (every contraction over all elements), one full point each
    q = timed[0]
    dense = {}
    t0 = time.perf_counter()
    rd = ctx.run([H.params(q.beta, q.delta, q.n_max, q.d_cut, q.n_steps, prec=prec)])[0]
    td = time.perf_counter() - t0
    dense["split"] = {"value": 1.0 / td, "dlnz_vs_block_form": rd.lnz_per_site - results[0].lnz_per_site}
    if not args.no_dense_fp64:
        t0 = time.perf_counter()
        rdf = ctx.run([H.params(q.beta, q.delta, q.n_max, q.d_cut, q.n_steps, prec=H.FP64)])[0]
        tdf = time.perf_counter() - t0
        dense["fp64"] = {"value": 1.0 / tdf, "dlnz_vs_dense_split": rd.lnz_per_site - rdf.lnz_per_site}
        dense["dense_split_vs_dense_fp64"] = tdf / td
    dense["note"] = "one full point each, host wall clock around the synchronous call"
    out["dense_form"] = dense
    # CPU oracle baseline (bounded samples, all host cores and one)
    s, u, detail = oracle_sample(timed[0].beta, timed[0].delta)
    cpu = {"value": u / s, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
           "sample": SAMPLE_TEXT.format(nx=4), "sample_wall_s": s, "detail": detail}
    one = oracle_sample_one_thread(timed[0].beta, timed[0].delta)
    if one is not None:
        s1, u1, threads = one
        cpu["single_core"] = {"value": u1 / s1, "unit": UNIT, "cores": threads, "sample": SAMPLE_TEXT.format(nx=1),
                              "sample_wall_s": s1}
    out["cpu_baseline"] = cpu
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    main()
