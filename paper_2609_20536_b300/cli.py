"""Command-line entry points of the library.

  python -m paper_2609_20536_b300.cli run --beta 1.1 --delta 0.5 --n-max 4 --d-cut 64 --steps 25 [--prec split] [--block-sparse 1]
  python -m paper_2609_20536_b300.cli contract --M 65536 --N 4096 --K 4096 [--prec split] [--repeat 1]
  python -m paper_2609_20536_b300.cli grid --n 64 [--nstreams 0]

`run` prints ln Z/N and the per-step scalars of one point; `grid` times a
sample of the 64 x 64 (beta, Delta) grid with D_cut drawn from {24, 32, 48,
64} through the batch runner; `contract` times one C = A B^T of the given
shape through the contraction engine (random FP64 operands generated on the
device).
"""

import argparse
import json
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser(prog="paper_2609_20536_b300.cli")
    sub = ap.add_subparsers(dest="cmd", required=True)
    r = sub.add_parser("run")
    r.add_argument("--beta", type=float, required=True)
    r.add_argument("--delta", type=float, required=True)
    r.add_argument("--n-max", type=int, default=4)
    r.add_argument("--d-cut", type=int, default=64)
    r.add_argument("--steps", type=int, default=25)
    r.add_argument("--h", type=float, default=0.0)
    r.add_argument("--h1", type=float, default=0.0)
    r.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    r.add_argument("--block-sparse", type=int, default=1, choices=[0, 1])
    g = sub.add_parser("grid")
    g.add_argument("--n", type=int, default=64, help="first n points of the 64 x 64 (beta, Delta) grid")
    g.add_argument("--stride", type=int, default=61, help="take every stride-th grid point (spreads beta, Delta)")
    g.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    g.add_argument("--block-sparse", type=int, default=1, choices=[0, 1])
    g.add_argument("--nstreams", type=int, default=0, help="0: autotune 1..4 worker streams on 8 points first")
    c = sub.add_parser("contract")
    c.add_argument("--M", type=int, required=True)
    c.add_argument("--N", type=int, required=True)
    c.add_argument("--K", type=int, required=True)
    c.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    c.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)

    import torch
    from . import hotrg as H

    prec = {"split": H.SPLIT_BF16, "fast": H.SPLIT_BF16_FAST, "fp64": H.FP64}[a.prec]
    ctx = H.Context(stream=torch.cuda.current_stream().cuda_stream)
    if a.cmd == "run":
        p = H.params(a.beta, a.delta, a.n_max, a.d_cut, a.steps, h=a.h, h1=a.h1, prec=prec,
                     block_sparse=a.block_sparse if prec != H.FP64 else 0)
        t0 = time.perf_counter()
        res = ctx.run([p])[0]
        dt = time.perf_counter() - t0
        print(json.dumps({"lnz_per_site": res.lnz_per_site, "seconds": dt,
                          "ln_c": [res.step[k].ln_c for k in range(a.steps)],
                          "side": [res.step[k].side for k in range(a.steps)]}))
    elif a.cmd == "grid":
        from .workloads import grid_points
        allp = grid_points()
        sel = [allp[(i * a.stride) % len(allp)] for i in range(a.n)]
        bs = a.block_sparse if prec != H.FP64 else 0
        plist = [H.params(p.beta, p.delta, p.n_max, p.d_cut, p.n_steps, prec=prec, block_sparse=bs) for p in sel]
        tuned = None
        if a.nstreams == 0:
            best, secs = ctx.autotune_batch(plist[:8], max_streams=4)
            tuned = {"chosen": best, "seconds_per_count": secs}
        ctx.run_batch(plist[:4], nstreams=a.nstreams)  # workspaces and graphs of the classes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.run_batch(plist, nstreams=a.nstreams)
        dt = time.perf_counter() - t0
        counts = {}
        for p in sel:
            counts[p.d_cut] = counts.get(p.d_cut, 0) + 1
        print(json.dumps({"points": a.n, "seconds": dt, "points_per_s": a.n / dt, "d_cut_counts": counts,
                          "autotune": tuned, "status": sorted(set(r.status for r in res))}))
    else:
        g = torch.Generator(device="cuda").manual_seed(0)
        A = torch.randn(a.M, a.K, dtype=torch.float64, device="cuda", generator=g)
        B = torch.randn(a.N, a.K, dtype=torch.float64, device="cuda", generator=g)
        C = torch.empty(a.M, a.N, dtype=torch.float64, device="cuda")
        times = []
        for _ in range(a.repeat):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H.hotrg_contract(ctx.handle, prec, a.M, a.N, a.K, A.data_ptr(), a.K, B.data_ptr(), a.K, C.data_ptr(), a.N)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        best = min(times)
        print(json.dumps({"M": a.M, "N": a.N, "K": a.K, "prec": a.prec, "seconds": best,
                          "algorithmic_tflops": 2.0 * a.M * a.N * a.K / best / 1e12}))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
