"""One ETC solve of the benchmark geometry, for profilers (ncu).

python -m paper_2404_02433_b300.profile_case --n 512 --precision fp64 --dir 2

Builds the seeded random-sphere RVE (radius 8-20 voxels, fraction 0.25,
inclusions 1000, seed 2001) on an n^3 grid (or an nz x ny x nx grid with
--shape nz,ny,nx), then runs one solve to relative residual
1e-8 through the C ABI and prints kappa_eff and the iteration count.  With
--warm a two-iteration solve runs first (it fills the tile autotuner's cache)
and only the measured solve lies inside cudaProfilerStart/Stop, so
``ncu --profile-from-start off`` sees the PCG launches alone.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import numpy as np
    import torch

    from paper_2404_02433_b300 import binding as B
    from paper_2404_02433_b300 import build as BUILD
    from paper_2404_02433_b300 import microstructure as M

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--shape", type=str, default=None, help="nz,ny,nx instead of n^3")
    ap.add_argument("--dir", type=int, default=2)
    ap.add_argument("--precision", choices=["fp64", "mixed", "mixed_f64"], default="fp64")
    ap.add_argument("--contrast", type=float, default=1000.0)
    ap.add_argument("--maxit", type=int, default=5000)
    ap.add_argument("--warm", action="store_true")
    args = ap.parse_args()
    BUILD.build()
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else (args.n,) * 3
    mask, _ = M.random_spheres(shape, (8.0, 20.0), 0.25, 2001, 0.0, 1.0)
    k = torch.from_numpy(np.ascontiguousarray(1.0 + (args.contrast - 1.0) * mask)).cuda()
    rve = B.RVE(k)
    del k
    prec = {"fp64": B.ETC_PREC_FP64, "mixed": B.ETC_PREC_MIXED,
            "mixed_f64": B.ETC_PREC_MIXED_F64}[args.precision]
    if args.warm:
        rve.solve(args.dir, rtol=1e-8, maxit=2, precision=prec)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    kap, info = rve.solve(args.dir, rtol=1e-8, maxit=args.maxit, precision=prec)
    torch.cuda.synchronize()
    if args.warm:
        torch.cuda.profiler.stop()
    print(f"shape={shape} dir={args.dir} {args.precision}: kappa_eff={kap:.10f} "
          f"iters={info['iters']} relres={info['relres']:.3e} "
          f"solve_ms={info['t_solve_ms']:.1f}")
    rve.close()


if __name__ == "__main__":
    main()
