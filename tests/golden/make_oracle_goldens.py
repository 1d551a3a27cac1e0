#!/usr/bin/env python
"""Write the oracle's full-length results at the large bond dimensions.

Calls only the FP64 CPU oracle (``oracle/``).  Each case runs the truncated
HOTRG step of §2.4.1 (Eq. 2.11, 2.12, the eps_1 / eps_2 comparison, Eq. 2.15,
2.16) for its full number of steps and stores ln Z / N, ln c_0, the closing
trace and, per step, ln c_k, eps_1, eps_2, the chosen side, D' and the
decision diagnostics (would the strict tie and side widths have kept the same
eigenpairs, and how far each decision was from its threshold).

Cases (one JSON file each, written as soon as the case ends):
  c2_dcut48      beta = 1.1, Delta = 0.5, n_max = 5 (D0 = 11), D_cut = 48, 30 steps
  headline0/1    the first two points of the seeded D_cut = 64 workload
                 (beta ~ U[0.5, 2], Delta ~ U[0, 1], seed 20536, drawn one
                 point at a time), n_max = 4, 25 steps
A case name with the suffix "_strict" reruns that case with the strict widths
(cut cluster 1e-12, bare eps_2 < eps_1 comparison) and writes
strict_<case>.json: what the two widths of the reading change.

Dense FP64 on the host: the D_cut = 64 cases hold two D^5 = 1.07e9-element
intermediates (8.6 GB each) and take about an hour each on eight cores.

    python tests/golden/make_oracle_goldens.py [case ...]
"""

import json
import math
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import hotrg as OH  # noqa: E402

SEED = 20536


def headline(i):
    # the seeded workload's draw, restated here so that this script needs only numpy and oracle/
    rng = np.random.default_rng(SEED)
    bd = rng.uniform((0.5, 0.0), (2.0, 1.0), size=(i + 1, 2))
    return float(bd[i, 0]), float(bd[i, 1]), 4, 64, 25


CASES = {
    "c2_dcut48": (1.1, 0.5, 5, 48, 30),
    "headline0": headline(0),
    "headline1": headline(1),
}


def fnum(x):
    return None if (isinstance(x, float) and math.isnan(x)) else x


def run_case(name):
    strict = name.endswith("_strict")
    base = name[: -len("_strict")] if strict else name
    beta, delta, n_max, d_cut, n_steps = CASES[base]
    widths = ({"tie_rtol": OH.STRICT_TIE_RTOL, "side_rtol": OH.STRICT_SIDE_RTOL} if strict
              else {"tie_rtol": OH.TIE_RTOL, "side_rtol": OH.SIDE_RTOL})
    t_steps = []
    t_last = [time.perf_counter()]

    def on_step(k, rec):
        now = time.perf_counter()
        t_steps.append(now - t_last[0])
        t_last[0] = now
        print(f"  {name} step {k}: ln c = {rec.ln_c:.15f} side {rec.side} D' {rec.Dp} "
              f"strict_same {rec.strict_same} ({t_steps[-1]:.1f} s)", flush=True)

    t0 = time.perf_counter()
    res = OH.run_gxy(beta, delta, n_max, d_cut, n_steps, on_step=on_step, **widths)
    wall = time.perf_counter() - t0
    out = {
        "case": base, "strict": strict,
        "written_by": "tests/golden/make_oracle_goldens.py (FP64 CPU oracle, oracle.hotrg.run_gxy)",
        "passage": "thesis §2.4.1 (Eq. 2.11, 2.12, eps_1/eps_2 rule, Eq. 2.15, 2.16), tensor Eq. 3.4/3.6",
        "beta": beta, "delta": delta, "n_max": n_max, "d_cut": d_cut, "n_steps": n_steps,
        "tie_rtol": widths["tie_rtol"], "side_rtol": widths["side_rtol"],
        "strict_tie_rtol": OH.STRICT_TIE_RTOL, "strict_side_rtol": OH.STRICT_SIDE_RTOL,
        "lnz_per_site": res.lnz_per_site, "ln_c0": res.ln_c0, "ln_trace": res.ln_trace,
        "steps": [{"k": k + 1, "Dh": r.Dh, "Dv": r.Dv, "dprime": r.Dp, "ln_c": r.ln_c,
                   "eps_left": r.eps_left, "eps_right": fnum(r.eps_right), "side": r.side,
                   "strict_same": bool(r.strict_same), "side_margin": fnum(r.side_margin),
                   "cut_gap": r.cut_gap if math.isfinite(r.cut_gap) else None,
                   "kept_min": float(np.min(r.kept)), "kept_max": float(np.max(r.kept))}
                  for k, r in enumerate(res.steps)],
        "wall_s": wall, "step_s": t_steps,
        "host": {"machine": platform.machine(), "cpus": os.cpu_count(), "numpy": np.__version__},
    }
    path = os.path.join(HERE, f"strict_{base}.json" if strict else f"oracle_{name}.json")
    with open(path + ".tmp", "w") as f:
        json.dump(out, f, indent=1)
    os.replace(path + ".tmp", path)
    print(f"{name}: lnZ/N = {res.lnz_per_site!r} in {wall:.0f} s -> {path}", flush=True)


if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        if name.endswith("_strict") and name[: -len("_strict")] not in CASES or (
                not name.endswith("_strict") and name not in CASES):
            raise SystemExit(f"unknown case {name}")
        run_case(name)
