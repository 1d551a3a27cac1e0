#!/usr/bin/env python
"""HOTRG (beta, Delta) points/s at D_cut = 64 on B300.

Workload: distinct (beta, Delta) points of the q = 2 generalized XY model,
beta ~ U[0.5, 2.0], Delta ~ U[0, 1] (seed 20536), n_max = 4 (D0 = 9),
D_cut = 64, 25 coarse-graining steps per point (2^25 sites), run through the
C-ABI library (hotrg_run_batch on worker streams) in the split-BF16
precision form with block-sparse (per U(1) charge block) contractions.  One bench step =
one pass of the whole hot path (initial tensor, 25 HOTRG steps, closing
trace) over `--points` points per GPU.  Several GPUs run independent
replicas on distinct points (no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--points P] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the oracle is test infrastructure; this is its only use here).
"""

import argparse
import ctypes
import hashlib
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

METRIC = "HOTRG (beta,Delta) points/s at D_cut=64, mixed vs FP64 GPU, |d lnZ/N|<=1e-9"
UNIT = "points/s"
D_CUT, N_MAX, N_STEPS = 64, 4, 25
WORKLOAD = ("gXY q=2 HOTRG points, beta~U[0.5,2.0], Delta~U[0,1] (seed 20536), n_max=4 (D0=9), "
            "D_cut=64, 25 one-axis steps per point (2^25 sites), split-BF16 tensor-core form")
WORKLOAD_BS = ", contractions per U(1) charge block"
# ncu DRAM traffic of the coarse-contraction kernel, keyed by the source hash it was captured on
KNOWN_TRAFFIC = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--points", type=int, default=2, help="points per bench step per GPU")
    ap.add_argument("--nstreams", type=int, default=0,
                    help="worker streams of the batch runner (0: autotuned over 1..min(3, points) before the warm-up; "
                         "1: points one after another on one stream)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    ap.add_argument("--block-sparse", type=int, default=1, choices=[0, 1],
                    help="1: coarse contraction per U(1) charge block (the default form); 0: dense")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-form, accuracy and CPU legs")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d["bf16_tflops"], d["bf16_tflops_sustained"], "measured"
    return 1800.0, 1400.0, "fallback"


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
    for f in ["hotrg_umma.cu", "internal.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2609_20536_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_point_seconds(beta, delta, nx=4):
    """Seconds per point of the FP64 oracle, from a bounded sample.

    Steps 1 and 2 run in full.  Step 3 is the first step at full size
    (D_h = D_v = D' = 64) and every later step has the same size: its
    environments and truncations are timed in full, its coarse contraction on
    nx of the D' output columns x (the contraction is linear in that count),
    scaled by D'/nx.  Per point = t1 + t2 + (n_steps - 2) x t3.
    """
    import numpy as np
    from oracle import gxy
    from oracle import hotrg as OH

    T = gxy.site_tensor(beta, delta, N_MAX)
    T = T / np.linalg.norm(T)
    q = gxy.leg_charges(N_MAX, "u1")
    qh, qv = q.copy(), q.copy()
    t_steps = []
    for _ in range(2):
        t0 = time.perf_counter()
        T, qh, qv, _, _ = OH.hotrg_step(T, qh, qv, D_CUT, "u1")
        t_steps.append(time.perf_counter() - t0)
    Dh = T.shape[0]
    Dp = min(D_CUT, Dh * Dh)
    qf = OH.fused_charges(qh, "u1")
    t0 = time.perf_counter()
    EL = OH.environment_left(T)
    ER = OH.environment_right(T)
    P, _, eps_l, _ = OH.truncation(EL, qf, Dp)
    OH.truncation(ER, qf, Dp)
    t_env = time.perf_counter() - t0
    P3 = P.reshape(Dh, Dh, Dp)
    t0 = time.perf_counter()
    Tn = OH.coarse(np.ascontiguousarray(P3[:, :, :nx]), T, T)  # nx of the D' left output columns
    t_coarse = (time.perf_counter() - t0) * Dp / nx
    t0 = time.perf_counter()
    float(np.linalg.norm(Tn))
    t_norm = (time.perf_counter() - t0) * Dp / nx
    t3 = t_env + t_coarse + t_norm
    return t_steps[0] + t_steps[1] + (N_STEPS - 2) * t3, {"t_step1": t_steps[0], "t_step2": t_steps[1],
                                                          "t_step3_est": t3, "x_columns": nx}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else os.cpu_count()
    except Exception:
        return os.cpu_count()


def run_reference(args):
    from paper_2609_20536_b300.workloads import headline_points
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pts = headline_points(args.warmup + args.steps, d_cut=D_CUT, n_max=N_MAX, n_steps=N_STEPS)
    for p in pts[: args.warmup]:
        oracle_point_seconds(p.beta, p.delta)
    per_point = []
    detail = None
    for p in pts[args.warmup:]:
        s, detail = oracle_point_seconds(p.beta, p.delta)
        per_point.append(s)
    sec = statistics.mean(per_point)
    value = 1.0 / sec
    sample = ("per point: steps 1-2 in full, step 3 environments/truncation in full and its coarse "
              "contraction on 4 of 64 output columns scaled x16, steps 3-25 taken equal (extrapolated)")
    cores = blas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("split-BF16 tensor-core form", "FP64 CPU oracle (numpy)"),
                       "points_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "detail": detail},
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

    def batch(step):
        base = (step * world + rank) * P
        return [H.params(p.beta, p.delta, p.n_max, p.d_cut, p.n_steps, prec=prec, block_sparse=args.block_sparse)
                for p in pts[base:base + P]]

    tuned = None
    if args.nstreams == 0:
        # autotune the worker-stream count on one bench step's worth of points (untimed); more
        # streams than points per step would only idle
        best, secs = ctx.autotune_batch(batch(0), max_streams=max(1, min(3, P)))
        tuned = {"chosen": best, "seconds_per_count": secs, "points": P}
        args.nstreams = best

    def run(plist):
        if args.nstreams > 1:
            return ctx.run_batch(plist, nstreams=args.nstreams)
        return ctx.run(plist)

    for s in range(args.warmup):
        run(batch(s))
    H.hotrg_profile_enable(ctx.handle, True)
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
    prof = H.hotrg_profile_read(ctx.handle)
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
    burst, sustained, src = peaks()
    coarse_ms = prof.gemm_ms[1]
    fp64_equiv = prof.gemm_flops[1] / (coarse_ms / 1e3) / 1e12 if coarse_ms > 0 else 0.0
    slices = 15 if prec == H.SPLIT_BF16 else (6 if prec == H.SPLIT_BF16_FAST else 1)
    # a split form is bounded by the BF16 tensor pipe: every slice product is 2MNK of BF16 work
    achieved = fp64_equiv * slices
    kname = ("umma_grouped_kernel<5> (block-sparse coarse contraction s1/s2/s3)" if args.block_sparse
             else "umma_gemm_kernel<5> (coarse contraction s1/s2/s3)")
    roof = {"bound": "tensor", "kernel": kname,
            "achieved": achieved, "peak": sustained, "unit": "TFLOP/s", "frac": achieved / sustained,
            "peak_source": f"bf16 sustained, {src}",
            "achieved_is": (f"{slices} BF16 slice products x 2MNK per contraction (per charge block, summed over "
                            "blocks, when block-sparse) / CUDA-event time on its stream"),
            "slice_products": slices, "fp64_equivalent_tflops": fp64_equiv,
            "kernel_share_of_steps": coarse_ms / prof.step_ms if prof.step_ms else None,
            "traffic": KNOWN_TRAFFIC.get(source_hash())}
    breakdown = {"coarse_gemm_ms": coarse_ms, "env_gemm_ms": prof.gemm_ms[0], "slice_ms": prof.slice_ms,
                 "eig_ms": prof.eig_ms, "eig_parts_ms": {"jacobi_small": prof.eig_part_ms[0],
                                                          "subspace_fp32": prof.eig_part_ms[1],
                                                          "rayleigh_ritz": prof.eig_part_ms[2],
                                                          "select_projector": prof.eig_part_ms[3]},
                 "steps_ms": prof.step_ms, "hotrg_steps": prof.steps,
                 "note": "CUDA-event time per region class summed over worker streams (regions overlap in time)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec != H.FP64 else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + (WORKLOAD_BS if args.block_sparse else ""), "points_per_step": P,
                       "worker_streams": args.nstreams, "autotune": tuned,
                       "d_cut": D_CUT, "n_max": N_MAX,
                       "n_steps": N_STEPS, "prec": args.prec, "parallelism": f"replicas x{world}",
                       "l2": "working set above L2: 8.6 GB D^5 intermediates per HOTRG step"},
            "roofline": roof, "breakdown": breakdown, "clocks": clk, "gpu_launches": int(prof.launches),
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": ctypes.sizeof(H.Params) * P * world,
                    "d2h_bytes_per_step": ctypes.sizeof(H.Result) * P * world,
                    "note": "host wall clock around the synchronous hotrg_run_batch / hotrg_run C-ABI call: "
                            "params in, results out"}}
    if not args.no_extras and world == 1:
        line.update(extras(H, ctx, pts, prec, args.block_sparse))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extras(H, ctx, pts, prec, bs):
    """FP64-form and dense-form timing at the same D_cut, accuracy against the oracle, CPU oracle baseline."""
    out = {}
    import torch
    # FP64 form: first 3 steps of one point (step 3 is the first at full size)
    p = pts[0]
    t0 = time.perf_counter()
    r2 = ctx.run([H.params(p.beta, p.delta, p.n_max, p.d_cut, 2, prec=H.FP64)])[0]
    t2 = time.perf_counter() - t0
    t0 = time.perf_counter()
    r3 = ctx.run([H.params(p.beta, p.delta, p.n_max, p.d_cut, 3, prec=H.FP64)])[0]
    t3 = time.perf_counter() - t0 - t2
    fp64_point_s = t2 + (N_STEPS - 2) * t3
    split3 = ctx.run([H.params(p.beta, p.delta, p.n_max, p.d_cut, 3, prec=prec, block_sparse=bs)])[0]
    out["fp64_form"] = {"value": 1.0 / fp64_point_s, "unit": UNIT, "s_per_full_step": t3,
                        "note": "FP64 SIMT form at the same workload, 3 steps timed, steps 3-25 taken equal",
                        "dlnz_split_vs_fp64_after_3_steps": split3.lnz_per_site - r3.lnz_per_site}
    if bs:
        # the dense split form (every contraction over all elements) on one point, for comparison
        q = pts[1]
        t0 = time.perf_counter()
        rd = ctx.run([H.params(q.beta, q.delta, q.n_max, q.d_cut, q.n_steps, prec=prec)])[0]
        td = time.perf_counter() - t0
        rb = ctx.run([H.params(q.beta, q.delta, q.n_max, q.d_cut, q.n_steps, prec=prec, block_sparse=1)])[0]
        out["dense_form"] = {"value": 1.0 / td, "unit": UNIT, "note": "split-BF16 form with dense contractions, "
                             "one point, host wall clock", "dlnz_block_vs_dense": rb.lnz_per_site - rd.lnz_per_site}
    # accuracy of the timed form against the FP64 oracle on smaller points of the same family
    from oracle import hotrg as OH
    errs = []
    for q in pts[:3]:
        ref = OH.run_gxy(q.beta, q.delta, q.n_max, 16, 20).lnz_per_site
        got = ctx.run([H.params(q.beta, q.delta, q.n_max, 16, 20, prec=prec, block_sparse=bs)])[0].lnz_per_site
        errs.append(abs(got - ref))
    out["accuracy"] = {"max_abs_dlnz_vs_oracle": max(errs), "points": 3, "d_cut": 16, "n_steps": 20,
                       "note": "same (beta, Delta) points at D_cut=16 (oracle at D_cut=64 takes ~30 min/point)"}
    # CPU oracle baseline (bounded sample)
    t0 = time.perf_counter()
    sec, detail = oracle_point_seconds(p.beta, p.delta)
    out["cpu_baseline"] = {"value": 1.0 / sec, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                           "sample": ("one point: steps 1-2 in full, step 3 environments/truncation in full and "
                                      "its coarse contraction on 4 of 64 output columns scaled x16, steps 3-25 "
                                      "taken equal (extrapolated)"),
                           "sample_wall_s": time.perf_counter() - t0, "detail": detail}
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    main()
