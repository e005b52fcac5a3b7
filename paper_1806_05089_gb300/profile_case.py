"""Run one small PonD case for profiling (e.g. under ncu).

  python -m paper_1806_05089_gb300.profile_case --form fp64 --n 1024 --steps 2 [--kernel direct]
  python -m paper_1806_05089_gb300.profile_case --form mixed --n 2048 --steps 3
  python -m paper_1806_05089_gb300.profile_case --form batched --grids 64 --steps 2
  python -m paper_1806_05089_gb300.profile_case --form adjoint --n 256 --steps 2

fp64 / mixed use the supersonic workload (uniform u = (1.5, 0.5), 8 seeded
sinusoids in rho and T) at n x n; batched uses the first ``--grids`` members
of the 256-grid ensemble; adjoint runs ``--steps`` forward steps and their
adjoint on the Taylor-Green + pulse workload at n x n.  One warm-up step
precedes the measured steps, so ``ncu -s`` can skip it.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--form", choices=["fp64", "mixed", "batched", "adjoint"], default="fp64")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--grids", type=int, default=64)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--tile", type=int, default=0,
                    help="tile kernels: tile rows (4, 8, 16 mixed only; -16 = the direct mixed "
                         "kernel's two nodes per thread)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="adjoint: precision of the rollout and its adjoint")
    ap.add_argument("--npw", type=int, default=0,
                    help="fp64: nodes per warp of the step kernel (1, 2, 3 on d2q9, 32 = one per "
                         "thread; 0 = default)")
    ap.add_argument("--kernel", choices=["staged", "direct"], default="staged",
                    help="fp64 / mixed / batched / adjoint: the reference-gauge staged tile "
                         "kernel (the default) or the direct per-pair kernels")
    ap.add_argument("--lattice", choices=["d2q16", "d2q9"], default="d2q16",
                    help="fp64 / mixed / batched: lattice (d2q9 runs the same flow at "
                         "T_L = 1/3: T/3, u/sqrt 3)")
    a = ap.parse_args()

    import torch

    from . import pond, workloads
    pond.load()
    out = {"form": a.form, "lattice": a.lattice}
    q9 = a.lattice == "d2q9"
    lat = {"lattice": pond.POND_D2Q9, "T_ref": 1.0 / 3.0} if q9 else {}

    def scaled(f):
        if q9:
            f.T = f.T / 3.0
            f.ux = f.ux / 3.0 ** 0.5
            f.uy = f.uy / 3.0 ** 0.5
        return f
    if a.form in ("fp64", "mixed"):
        prec = pond.POND_FP64 if a.form == "fp64" else pond.POND_FP32_MIXED
        f = scaled(workloads.supersonic(a.n))
        cfg = dict(lat)
        cfg["kernel"] = pond.POND_KERNEL_STAGED if a.kernel == "staged" else pond.POND_KERNEL_DIRECT
        if prec == pond.POND_FP32_MIXED or a.kernel == "staged":
            cfg["tile_rows"] = a.tile
        else:
            cfg["nodes_per_warp"] = a.npw
        with pond.Sim(a.n, a.n, prec, **cfg) as s:
            s.set_state(f.rho, f.ux, f.uy, f.T)
            s.step(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = s.step(a.steps)
            sec = time.perf_counter() - t0
            out.update(n=a.n, steps=a.steps, seconds=sec, tile=st["tile_rows"],
                       node_updates_per_s=a.n * a.n * a.steps / sec,
                       passes=st["passes"] / st["node_updates"])
    elif a.form == "batched":
        nxs, nys = workloads.ensemble_sizes(256)
        nxs, nys = nxs[:a.grids], nys[:a.grids]
        kern = pond.POND_KERNEL_STAGED if a.kernel == "staged" else pond.POND_KERNEL_DIRECT
        with pond.Sim(nxs, nys, pond.POND_FP32_MIXED, tile_rows=a.tile, kernel=kern, **lat) as s:
            for i in range(a.grids):
                m = scaled(workloads.ensemble_member(i, nxs[i], nys[i]))
                s.set_state(m.rho, m.ux, m.uy, m.T, grid=i)
            s.step(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = s.step(a.steps)
            sec = time.perf_counter() - t0
            nodes = int(sum(x * y for x, y in zip(nxs, nys)))
            out.update(grids=a.grids, nodes=nodes, steps=a.steps, seconds=sec, tile=st["tile_rows"],
                       node_updates_per_s=nodes * a.steps / sec)
    else:
        from .autograd import pond_rollout
        f, target = workloads.adjoint(a.n)
        dev = torch.device("cuda")
        r = torch.tensor(f.rho, device=dev, requires_grad=True)
        prec = pond.POND_FP64 if a.precision == "fp64" else pond.POND_FP32_MIXED
        kern = pond.POND_KERNEL_STAGED if a.kernel == "staged" else pond.POND_KERNEL_DIRECT
        rho = pond_rollout(r, 0.01, *(torch.tensor(v, device=dev) for v in (f.ux, f.uy, f.T)),
                           a.steps, a.steps, precision=prec, kernel=kern)
        (0.5 * ((rho - torch.tensor(target, device=dev)) ** 2).sum()).backward()
        torch.cuda.synchronize()
        out.update(n=a.n, steps=a.steps, precision=a.precision, kernel=a.kernel,
                   grad_norm=float(r.grad.norm()))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
