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
    s64 = pond.Sim(n, n, pond.POND_FP64, stream=stream)
    s32 = pond.Sim(n, n, pond.POND_FP32_MIXED, stream=stream, use_graph=1)
    for s in (s64, s32):
        s.set_state(f.rho, f.ux, f.uy, f.T)
    del f
    m64 = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(4)]
    m32 = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(4)]
    done = 0
    t64 = t32 = 0.0
    passes64 = passes32 = 0
    while done < a.steps:
        k = min(a.every, a.steps - done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st64 = s64.step(k)
        t1 = time.perf_counter()
        st32 = s32.step(k)
        t2 = time.perf_counter()
        t64 += t1 - t0
        t32 += t2 - t1
        passes64 += st64["passes"]
        passes32 += st32["passes"]
        done += k
        pond.pond_moments(s64.ctx, 0, *m64)
        pond.pond_moments(s32.ctx, 0, *m32)
        torch.cuda.synchronize()
        rho64, ux64, uy64, T64 = m64
        rho32, ux32, uy32, T32 = m32
        uscale = max(float(torch.maximum(ux64.abs().max(), uy64.abs().max())),
                     float(T64.mean().sqrt()))
        line = {
            "workload": "%s-%d" % (a.workload, n), "step": done,
            "rho": float(((rho32 - rho64).abs() / rho64).max()),
            "u": float(torch.maximum((ux32 - ux64).abs().max(), (uy32 - uy64).abs().max())) / uscale,
            "T": float(((T32 - T64).abs() / T64).max()),
            "fp64_s": t64, "mixed_s": t32,
            "fp64_passes": passes64 / (done * n * n), "mixed_passes": passes32 / (done * n * n),
            "speedup": t64 / t32 if t32 > 0 else None,
            "nonconverged": [st64["nonconverged"], st32["nonconverged"]],
            "nonphysical": [st64["nonphysical"], st32["nonphysical"]],
        }
        print(json.dumps(line), flush=True)
    s64.close()
    s32.close()


if __name__ == "__main__":
    main()
