"""Command-line entry points of the library.

  python -m paper_2609_20536_b300.cli run --beta 1.1 --delta 0.5 --n-max 4 --d-cut 64 --steps 25 [--prec split] [--block-sparse 1]
  python -m paper_2609_20536_b300.cli contract --M 65536 --N 4096 --K 4096 [--prec split] [--repeat 1]
  python -m paper_2609_20536_b300.cli grid --n 64 [--nstreams 0]
  python -m paper_2609_20536_b300.cli surrogate [--nb 12 --nd 8 --d-cut 12 --steps 16]
  python -m paper_2609_20536_b300.cli phase --delta 0.32 [--t-lo 0.5 --t-hi 1.2 --n-t 36 --hbar 0.005,0.01,0.02,0.04]
  python -m paper_2609_20536_b300.cli peaks
  python -m paper_2609_20536_b300.cli sweep --delta 0.3 [--b-lo 0.8 --b-hi 1.6 --b-step 0.01 --n-max 6 --d-cut 96 --steps 30]

`run` prints ln Z/N and the per-step scalars of one point; `grid` times a
sample of the 64 x 64 (beta, Delta) grid with D_cut drawn from {24, 32, 48,
64} through the batch runner; `surrogate` builds a training grid of
observables, trains the MLP ensemble, audits it against HOTRG on random
points and refines near the C_V / chi maxima; `phase` scans one Delta in
temperature and prints the C_V peaks, the chi peak at each central field and
the zero-field T_c of the fit T_p = a + b hbar^c (a row of Table 3.1 at this
bond dimension); `sweep` runs a beta sweep at one Delta with C_V by FP64
central differences of ln Z/N and the impurity observables m, chi (cos theta,
h != 0: no conserved label) and m1, chi1 (cos 2 theta, h1 != 0: Z2 blocks),
each family at its own D_cut; `peaks` measures cuBLAS's dense GEMM rates (torch.matmul)
in FP64, FP32, TF32 and BF16, the denominators of the FP64-form rooflines;
`contract` times one C = A B^T of the given
shape through the contraction engine (random FP64 operands generated on the
device).
"""

import argparse
import json
import sys
import time


def phase_summary(H, delta, d_cut, temps, hbars, res, seconds, cv_prominence=0.0):
    """JSON-ready summary of one hotrg_phase_scan: every C_V peak (with its height, its
    prominence and whether a neighbouring sample has C_V < 0), the chi peak per central
    field and the zero-field fit.  At small D_cut a change of the kept set between
    beta - hb and beta + hb puts isolated spikes or dips into C_V's difference quotient;
    a peak next to a negative C_V is such an artefact, not a transition."""
    import numpy as np
    temps = np.asarray(temps, dtype=np.float64)
    cv = res["cv"]
    cv_out = []
    if cv is not None:
        peaks, _ = H.hotrg_find_peaks(temps, cv, cv_prominence, len(temps))
        for x, y, p in peaks:
            k = int(np.argmin(np.abs(temps - x)))
            neg = bool(np.any(cv[max(0, k - 1):k + 2] < 0))
            cv_out.append({"T": x, "cv": y, "prominence": p, "next_to_negative_cv": neg})
    f = res["fit"]
    return {"delta": delta, "field": {H.T_IMP_M: "h", H.T_IMP_M1: "h1"}.get(res["field"], None), "d_cut": d_cut,
            "seconds": seconds, "cv_peaks": cv_out, "hbar": list(hbars),
            "T_chi_peak": [None if np.isnan(v) else float(v) for v in res["t_peak"]],
            "T_c_zero_field": None if f.n == 0 else f.a,
            "fit": None if f.n == 0 else {"a": f.a, "b": f.b, "c": f.c, "a_err": f.a_err, "b_err": f.b_err,
                                          "c_err": f.c_err, "n": f.n, "at_bound": f.at_bound},
            "status": res["status"]}


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
    r.add_argument("--profile", action="store_true", help="also print the library's per-class profile counters")
    g = sub.add_parser("grid")
    g.add_argument("--n", type=int, default=64, help="first n points of the 64 x 64 (beta, Delta) grid")
    g.add_argument("--stride", type=int, default=61, help="take every stride-th grid point (spreads beta, Delta)")
    g.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    g.add_argument("--block-sparse", type=int, default=1, choices=[0, 1])
    g.add_argument("--nstreams", type=int, default=0, help="0: autotune 1..4 worker streams on 8 points first")
    g.add_argument("--check", type=int, default=0,
                   help="re-run this many of the points (spread over the sample) in the FP64 block form and "
                        "report |d lnZ/N| against it")
    g.add_argument("--out", default="", help="write every point's (beta, Delta, D_cut, lnZ/N, status) as JSON here")
    sg = sub.add_parser("surrogate")
    sg.add_argument("--nb", type=int, default=12, help="training grid: nb betas in [b-lo, b-hi]")
    sg.add_argument("--nd", type=int, default=8, help="training grid: nd Deltas in [d-lo, d-hi]")
    sg.add_argument("--b-lo", type=float, default=0.6)
    sg.add_argument("--b-hi", type=float, default=1.6)
    sg.add_argument("--d-lo", type=float, default=0.1)
    sg.add_argument("--d-hi", type=float, default=0.9)
    sg.add_argument("--per-peak", type=int, default=4, help="refinement points per C_V or chi window and Delta")
    sg.add_argument("--out", default="", help="write the training, audit and refinement tables as JSON here")
    sg.add_argument("--n-max", type=int, default=2)
    sg.add_argument("--d-cut", type=int, default=12)
    sg.add_argument("--steps", type=int, default=16)
    sg.add_argument("--epochs", type=int, default=2000)
    sg.add_argument("--threshold", type=float, default=1e-3)
    sg.add_argument("--audit", type=int, default=64)
    sg.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    ph = sub.add_parser("phase")
    ph.add_argument("--delta", type=float, required=True)
    ph.add_argument("--t-lo", type=float, default=0.5)
    ph.add_argument("--t-hi", type=float, default=1.2)
    ph.add_argument("--n-t", type=int, default=36)
    ph.add_argument("--hbar", default="0.005,0.01,0.02,0.04", help="central fields of chi, comma separated")
    ph.add_argument("--field", default="auto", choices=["auto", "h", "h1"])
    ph.add_argument("--dh", type=float, default=1e-3)
    ph.add_argument("--n-max", type=int, default=4)
    ph.add_argument("--d-cut", type=int, default=24)
    ph.add_argument("--steps", type=int, default=30)
    ph.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    ph.add_argument("--nstreams", type=int, default=0)
    ph.add_argument("--chi-prominence", type=float, default=0.0, help="least prominence of a chi peak")
    ph.add_argument("--cv-prominence", type=float, default=0.0, help="least prominence of a listed C_V peak")
    sw = sub.add_parser("sweep")
    sw.add_argument("--delta", type=float, default=0.3)
    sw.add_argument("--b-lo", type=float, default=0.8)
    sw.add_argument("--b-hi", type=float, default=1.6)
    sw.add_argument("--b-step", type=float, default=0.01)
    sw.add_argument("--n-max", type=int, default=6)
    sw.add_argument("--d-cut", type=int, default=96, help="D_cut of the pure runs (ln Z/N, f, C_V)")
    sw.add_argument("--m-d-cut", type=int, default=0, help="D_cut of the cos theta runs (m, chi); 0: skip them")
    sw.add_argument("--m1-d-cut", type=int, default=0, help="D_cut of the cos 2 theta runs (m1, chi1); 0: skip")
    sw.add_argument("--steps", type=int, default=30)
    sw.add_argument("--hb", type=float, default=1e-3)
    sw.add_argument("--hbar", type=float, default=0.01)
    sw.add_argument("--dh", type=float, default=1e-3)
    sw.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    sw.add_argument("--nstreams", type=int, default=1,
                    help="worker streams (each holds a full workspace: keep 1 at D_cut = 96)")
    sw.add_argument("--out", default="")
    pk = sub.add_parser("peaks")
    pk.add_argument("--repeat", type=int, default=5)
    c = sub.add_parser("contract")
    c.add_argument("--M", type=int, required=True)
    c.add_argument("--N", type=int, required=True)
    c.add_argument("--K", type=int, required=True)
    c.add_argument("--prec", default="split", choices=["split", "fast", "fp64"])
    c.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)

    import torch
    from . import hotrg as H

    if a.cmd == "peaks":
        # dense n^3 matmuls through cuBLAS (torch): 3 warm-ups, best of --repeat, CUDA events
        out = {}
        for name, dt, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192),
                            ("tf32", torch.float32, 8192), ("bf16", torch.bfloat16, 8192)):
            torch.backends.cuda.matmul.allow_tf32 = name == "tf32"
            x = torch.randn(n, n, device="cuda", dtype=dt)
            y = torch.randn(n, n, device="cuda", dtype=dt)
            for _ in range(3):
                torch.matmul(x, y)
            best = 1e30
            for _ in range(a.repeat):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(x, y)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = {"n": n, "tflops": 2.0 * n ** 3 / best / 1e12}
            del x, y
        torch.backends.cuda.matmul.allow_tf32 = False
        out["device"] = torch.cuda.get_device_name()
        print(json.dumps(out))
        return 0
    prec = {"split": H.SPLIT_BF16, "fast": H.SPLIT_BF16_FAST, "fp64": H.FP64}[a.prec]
    ctx = H.Context(stream=torch.cuda.current_stream().cuda_stream)
    if a.cmd == "run":
        p = H.params(a.beta, a.delta, a.n_max, a.d_cut, a.steps, h=a.h, h1=a.h1, prec=prec,
                     block_sparse=a.block_sparse)
        if a.profile:
            H.hotrg_profile_enable(ctx.handle, True)
        t0 = time.perf_counter()
        res = ctx.run([p])[0]
        dt = time.perf_counter() - t0
        out = {"lnz_per_site": res.lnz_per_site, "seconds": dt,
               "ln_c": [res.step[k].ln_c for k in range(a.steps)],
               "side": [res.step[k].side for k in range(a.steps)]}
        if a.profile:
            pr = H.hotrg_profile_read(ctx.handle)
            out["profile"] = {f: (list(getattr(pr, f)) if hasattr(getattr(pr, f), "__len__") else getattr(pr, f))
                              for f, _ in H.Profile._fields_}
        print(json.dumps(out))
    elif a.cmd == "grid":
        import os

        import numpy as np
        from . import replicas
        from .workloads import grid_points
        allp = grid_points()
        everything = [allp[(i * a.stride) % len(allp)] for i in range(a.n)]
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if world > 1:  # replicas: each rank runs its longest-first share, scalars gathered on the host
            import torch.distributed as dist
            dist.init_process_group("gloo")
        mine = replicas.shard(everything, world, rank)
        sel = [everything[i] for i in mine]
        bs = a.block_sparse
        plist = [H.params(p.beta, p.delta, p.n_max, p.d_cut, p.n_steps, prec=prec, block_sparse=bs) for p in sel]
        tuned = None
        if a.nstreams == 0:
            best, secs = ctx.autotune_batch(plist[:8], max_streams=4)
            tuned = {"chosen": best, "seconds_per_count": secs}
        ctx.run_batch(plist[:4], nstreams=a.nstreams)  # workspaces and graphs of the classes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = H.hotrg_run_batch(ctx.handle, plist, nstreams=a.nstreams, check=False)  # failures stay per point
        dt = time.perf_counter() - t0
        counts = {}
        for p in sel:
            counts[p.d_cut] = counts.get(p.d_cut, 0) + 1
        merged = replicas.gather({i: (r.lnz_per_site, r.status) for i, r in zip(mine, res)})
        if world > 1:
            import torch.distributed as dist
            t = [None] * world
            dist.all_gather_object(t, dt)
            dt = max(t)
            dist.destroy_process_group()
        if rank == 0:
            summary = {"points": len(merged), "ranks": world, "seconds": dt, "points_per_s": len(merged) / dt,
                       "d_cut_counts_rank0": counts, "autotune": tuned,
                       "status": sorted(set(v[1] for v in merged.values())),
                       "failed": sum(1 for v in merged.values() if v[1] != 0)}
            if a.check > 0 and world == 1:
                idx = [int(i) for i in np.linspace(0, len(sel) - 1, a.check)]
                chk = [H.params(sel[i].beta, sel[i].delta, sel[i].n_max, sel[i].d_cut, sel[i].n_steps,
                                prec=H.FP64, block_sparse=1) for i in idx]
                rf = ctx.run_batch(chk, nstreams=max(1, a.nstreams))
                dl = [res[i].lnz_per_site - r.lnz_per_site for i, r in zip(idx, rf)]
                summary["check_vs_fp64_block"] = {"points": len(idx), "max_abs_dlnz": max(abs(x) for x in dl),
                                                  "d_cut": [sel[i].d_cut for i in idx],
                                                  "dlnz": [float("%.3g" % x) for x in dl]}
            if a.out:
                with open(a.out, "w") as f:
                    json.dump([{"beta": everything[i].beta, "delta": everything[i].delta,
                                "d_cut": everything[i].d_cut, "lnz_per_site": v[0], "status": v[1]}
                               for i, v in sorted(merged.items())], f)
            print(json.dumps(summary))
    elif a.cmd == "surrogate":
        import numpy as np
        out = {}

        def mk(b, d):
            return H.params(b, d, a.n_max, a.d_cut, a.steps, prec=prec, block_sparse=1)

        betas, deltas = np.linspace(a.b_lo, a.b_hi, a.nb), np.linspace(a.d_lo, a.d_hi, a.nd)
        X = np.array([[b, d] for d in deltas for b in betas])
        t0 = time.perf_counter()
        obs = ctx.observables_batch([mk(b, d) for b, d in X], nstreams=0)
        out["train_points"], out["train_observables_s"] = len(X), time.perf_counter() - t0
        out["hotrg_points_per_s"] = len(X) / out["train_observables_s"]
        Y = np.array([[o.f, o.cv, o.chi, o.chi1] for o in obs])
        sur = H.Surrogate(ensemble=4, seed=20536)
        t0 = time.perf_counter()
        out["final_loss"] = sur.fit(X, Y, epochs=a.epochs, batch=64, lr=2e-3)
        out["fit_s"] = time.perf_counter() - t0
        rng = np.random.default_rng(7)
        Xa = np.column_stack([rng.uniform(a.b_lo, a.b_hi, a.audit), rng.uniform(a.d_lo, a.d_hi, a.audit)])
        pred, sd = sur.predict(Xa)
        Xt = np.column_stack([rng.uniform(a.b_lo, a.b_hi, 65536), rng.uniform(a.d_lo, a.d_hi, 65536)])
        sur.predict(Xt[:1024])
        t0 = time.perf_counter()
        sur.predict(Xt)
        out["predictions_per_s"] = len(Xt) / (time.perf_counter() - t0)
        ref = ctx.observables_batch([mk(b, d) for b, d in Xa], nstreams=0)
        R = np.array([[o.f, o.cv, o.chi, o.chi1] for o in ref])
        err = np.abs(pred - R) / np.array(sur.scaling.y_std[:])
        out["audit_std_err_max"] = err.max(0).tolist()
        out["audit_std_err_rms"] = np.sqrt((err ** 2).mean(0)).tolist()
        out["audit_spread_median"] = float(np.median(sd.max(1)))
        Xr, pk = sur.peaks(deltas, a.b_lo, a.b_hi, 401, a.per_peak, 0.05)
        t0 = time.perf_counter()
        yr, sdr, solved = sur.refine(ctx, mk(1.0, 0.5), Xr, threshold=a.threshold, nstreams=0)
        out["refine_points"], out["refine_resolved"] = len(Xr), int(solved.sum())
        out["refine_s"] = time.perf_counter() - t0
        # the surrogate's own answer on the refinement points, judged by HOTRG where HOTRG re-solved
        ys, _ = sur.predict(Xr)
        if solved.any():
            errs = np.abs(ys[solved] - yr[solved]) / np.array(sur.scaling.y_std[:])
            out["refine_resolved_std_err_rms"] = np.sqrt((errs ** 2).mean(0)).tolist()
        out["refine_kept_surrogate"] = int((~solved).sum())
        if (~solved).any():
            out["refine_kept_spread_max"] = float(sdr[~solved].max())
        out["peak_beta_cv_chi"] = pk.tolist()
        if a.out:
            with open(a.out, "w") as f:
                json.dump({"X": X.tolist(), "Y": Y.tolist(), "Xa": Xa.tolist(), "Ya": R.tolist(), "pred_a": pred.tolist(),
                           "Xr": Xr.tolist(), "yr": yr.tolist(), "solved": solved.tolist()}, f)
        sur.close()
        print(json.dumps(out))
    elif a.cmd == "sweep":
        import numpy as np
        nb = int(round((a.b_hi - a.b_lo) / a.b_step)) + 1
        betas = [a.b_lo + i * a.b_step for i in range(nb)]

        def runs(plist, imp):
            t0 = time.perf_counter()
            if a.nstreams > 1:
                r = H.hotrg_run_batch(ctx.handle, plist, imp_kind=imp, nstreams=a.nstreams, check=False)
            else:
                r = H.hotrg_run(ctx.handle, plist, imp_kind=imp, check=False)
            return r, time.perf_counter() - t0

        def mk(b, dc, h=0.0, h1=0.0):
            return H.params(b, a.delta, a.n_max, dc, a.steps, h=h, h1=h1, prec=prec, block_sparse=1)

        out = {"delta": a.delta, "n_max": a.n_max, "steps": a.steps, "prec": a.prec, "hb": a.hb, "hbar": a.hbar,
               "dh": a.dh, "beta": betas, "d_cut": a.d_cut}
        pure, t = runs([mk(b + o, a.d_cut) for b in betas for o in (-a.hb, 0.0, a.hb)], H.T_PURE)
        lz = np.array([r.lnz_per_site for r in pure]).reshape(nb, 3)
        out["pure_runs"], out["pure_s"] = 3 * nb, t
        out["status_pure"] = sorted(set(r.status for r in pure))
        out["lnz"] = lz[:, 1].tolist()
        out["f"] = (-lz[:, 1] / np.array(betas)).tolist()
        out["cv"] = (np.array(betas) ** 2 * (lz[:, 2] - 2 * lz[:, 1] + lz[:, 0]) / a.hb ** 2).tolist()
        for name, dc, kind in (("m", a.m_d_cut, H.T_IMP_M), ("m1", a.m1_d_cut, H.T_IMP_M1)):
            if dc <= 0:
                continue
            fld = (lambda v: {"h": v}) if name == "m" else (lambda v: {"h1": v})
            rr, t = runs([mk(b, dc, **fld(a.hbar + o)) for b in betas for o in (-a.dh, 0.0, a.dh)], kind)
            m = np.array([r.imp_ratio for r in rr]).reshape(nb, 3)
            out[name] = m[:, 1].tolist()
            out["chi" if name == "m" else "chi1"] = ((m[:, 2] - m[:, 0]) / (2 * a.dh)).tolist()
            out[name + "_d_cut"], out[name + "_runs"], out[name + "_s"] = dc, 3 * nb, t
            out["status_" + name] = sorted(set(r.status for r in rr))
        cvp, _ = H.hotrg_find_peaks(np.array(betas), np.array(out["cv"]), 0.0, 4)
        out["cv_peaks_beta"] = [x for x, _, _ in cvp]
        # C_V < 0 cannot be physical: the kept set changed between beta - hb and beta + hb (a kink of
        # the truncated ln Z); such samples, and peaks next to them, are truncation artefacts
        cv = np.array(out["cv"])
        out["cv_negative_beta"] = [b for b, v in zip(betas, cv) if v < 0]
        for key in ("chi", "chi1"):
            if key in out:
                pk_, _ = H.hotrg_find_peaks(np.array(betas), np.array(out[key]), 0.0, 4)
                out[key + "_peaks_beta"] = [x for x, _, _ in pk_]
        if a.out:
            with open(a.out, "w") as f:
                json.dump(out, f)
        print(json.dumps({k: v for k, v in out.items() if not isinstance(v, list) or len(v) < 8}))
    elif a.cmd == "phase":
        import numpy as np
        temps = np.linspace(a.t_lo, a.t_hi, a.n_t)
        hbars = [float(v) for v in a.hbar.split(",") if v]
        field = {"auto": 0, "h": H.T_IMP_M, "h1": H.T_IMP_M1}[a.field]
        base = H.params(1.0, a.delta, a.n_max, a.d_cut, a.steps, prec=prec, block_sparse=1)
        t0 = time.perf_counter()
        res = ctx.phase_scan(base, temps, hbars, field=field, dh=a.dh, nstreams=a.nstreams,
                             min_prominence=a.chi_prominence, check=False)
        dt = time.perf_counter() - t0
        if res["status"] not in (H.OK, H.ENOCONV):
            print(json.dumps({"status": res["status"], "error": H.hotrg_last_error(ctx.handle)}))
            ctx.close()
            return 1
        print(json.dumps(phase_summary(H, a.delta, a.d_cut, temps, hbars, res, dt, a.cv_prominence)))
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
