"""Error of the mixed FP32/FP64 step against the FP64 step over a long run.

  python -m paper_1806_05089_gb300.precision_report --workload precision --n 4096 \
      --steps 1000 --every 100

Both forms start from the same fields and advance side by side on one GPU;
every ``--every`` steps the moments are compared on the device and one JSON
line is printed:
  rho: max over nodes of |rho32 - rho64| / rho64
  T:   max over nodes of |T32 - T64| / T64
  u:   max over nodes of |u32 - u64| / max(max|u64|, sqrt(mean T64))
(the velocity scale is the larger of the flow speed and the thermal speed,
since FP32 rounding of the populations moves u by an amount set by the
particle speeds).  Timings of both forms are reported with the errors.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["precision", "supersonic", "tg"], default="precision")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--eps32", type=float, nargs="+", default=[1e-6],
                    help="mixed-form tolerances to compare (eps_abs = eps_rel = value); "
                         "one mixed run per value against the same FP64 run")
    ap.add_argument("--fixed", type=int, default=0, help="fixed pass count for every run")
    a = ap.parse_args()

    import torch

    from . import pond, workloads
    pond.load()
    if a.workload == "precision":
        f = workloads.precision(a.n)
    elif a.workload == "supersonic":
        f = workloads.supersonic(a.n)
    else:
        f = workloads.taylor_green(a.n, a.n, 0.05)
    n = a.n
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    s64 = pond.Sim(n, n, pond.POND_FP64, stream=stream, fixed_iter=a.fixed)
    mixed = [pond.Sim(n, n, pond.POND_FP32_MIXED, stream=stream, use_graph=1, fixed_iter=a.fixed,
                      eps_abs=e, eps_rel=e) for e in a.eps32]
    for s in [s64] + mixed:
        s.set_state(f.rho, f.ux, f.uy, f.T)
    del f
    m64 = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(4)]
    m32 = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(4)]
    done = 0
    t64 = 0.0
    t32 = [0.0] * len(mixed)
    p64 = 0
    p32 = [0] * len(mixed)
    while done < a.steps:
        k = min(a.every, a.steps - done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st64 = s64.step(k)
        t64 += time.perf_counter() - t0
        p64 += st64["passes"]
        sts = []
        for i, s in enumerate(mixed):
            t0 = time.perf_counter()
            st = s.step(k)
            t32[i] += time.perf_counter() - t0
            p32[i] += st["passes"]
            sts.append(st)
        done += k
        pond.pond_moments(s64.ctx, 0, *m64)
        rho64, ux64, uy64, T64 = m64
        uscale = max(float(torch.maximum(ux64.abs().max(), uy64.abs().max())),
                     float(T64.mean().sqrt()))
        for i, s in enumerate(mixed):
            pond.pond_moments(s.ctx, 0, *m32)
            torch.cuda.synchronize()
            rho32, ux32, uy32, T32 = m32
            line = {
                "workload": "%s-%d" % (a.workload, n), "step": done, "eps32": a.eps32[i],
                "fixed": a.fixed,
                "rho": float(((rho32 - rho64).abs() / rho64).max()),
                "u": float(torch.maximum((ux32 - ux64).abs().max(),
                                         (uy32 - uy64).abs().max())) / uscale,
                "T": float(((T32 - T64).abs() / T64).max()),
                "mass_drift": float((rho32.sum() - rho64.sum()) / rho64.sum()),
                "fp64_s": t64, "mixed_s": t32[i],
                "fp64_passes": p64 / (done * n * n), "mixed_passes": p32[i] / (done * n * n),
                "speedup": t64 / t32[i] if t32[i] > 0 else None,
                "nonconverged": [st64["nonconverged"], sts[i]["nonconverged"]],
                "nonphysical": [st64["nonphysical"], sts[i]["nonphysical"]],
            }
            print(json.dumps(line), flush=True)
    for s in [s64] + mixed:
        s.close()


if __name__ == "__main__":
    main()
