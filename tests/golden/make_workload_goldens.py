#!/usr/bin/env python3
"""Write tests/golden/workloads_oracle.txt: kappa_eff of the benchmark-family
workloads computed by the CPU oracle alone.

Only ``oracle/`` (the FP64 restatement of Algorithms 1-3 and the outflow
formula, Eq. effective formula dis) and the seeded input generators of
``paper_2404_02433_b300/microstructure.py`` (geometry and random numbers, none
of the method's arithmetic) are used; nothing here touches the CUDA library.

One fresh PCG run per (workload, loading direction), x0 = 0, to rtol 1e-12.
The run is observed after every pass (``on_iterate``), so the same iterates
give kappa_eff at the first pass with ||r||/||b|| <= 1e-8, <= 1e-10 and at the
end -- the values a fresh GPU solve stopped at that rtol reproduces up to
rounding (same Algorithm 1, same centred reference parameters of Algorithm 2).
The energy form of kappa_eff (an identity of the discrete system, error
quadratic in the solve error) is recorded at the end as a cross-check of the
converged value.

Workloads (the paper's random-inclusion experiments of Sec. 4, at sizes the
oracle finishes in minutes):
  spheres256_1000  256^3 random spheres, radius U[8, 20] voxels, fraction 0.25,
                   seed 2001, matrix 1, inclusions 1000 (the 512^3 benchmark's
                   generator at 256^3); loads z and x
  ellipsoids256    256^3 three-phase random ellipsoids, semi-axes U[4, 12],
                   phases 2 and 3 at fraction 0.15 each, kappa 1 / 20 / 500,
                   seed 3002; loads x and z
  lognormal128     the [0:128, 0:128, 0:128] crop of the 512^3 lognormal field
                   (exponential covariance, correlation length 16 voxels,
                   sigma 1.5, seed 3001); load x
  slab512_1000     512 x 512 x 16 voxels (x, y, z) of the benchmark's sphere
                   generator (radius U[8, 20], fraction 0.25, seed 2001,
                   1:1000): loads z (length-512 transforms on both axes, 16
                   planes) and x (transforms of lengths 512 and 16, 512 planes)

Usage: python tests/golden/make_workload_goldens.py [case ...]
(all cases by default; results are appended as each solve finishes).
"""
from __future__ import annotations

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import etc_oracle as O  # noqa: E402
from paper_2404_02433_b300 import microstructure as M  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads_oracle.txt")
THRESHOLDS = (1e-8, 1e-10)
RTOL_FINAL = 1e-12
MAXIT = 40000


def workload(name):
    """(kappa array (Nz, Ny, Nx), loading directions) of a named workload."""
    if name == "spheres256_1000":
        k, _ = M.random_spheres((256, 256, 256), (8.0, 20.0), 0.25, 2001, 1.0, 1000.0)
        return k, (2, 0)
    if name == "ellipsoids256":
        k, _ = M.random_ellipsoids((256, 256, 256), (4.0, 12.0), (0.15, 0.15),
                                   (1.0, 20.0, 500.0), 3002)
        return k, (0, 2)
    if name == "lognormal128":
        k = M.lognormal_field((512, 512, 512), 16.0, 1.5, 3001)[:128, :128, :128].copy()
        return k, (0,)
    if name == "slab512_1000":
        k, _ = M.random_spheres((16, 512, 512), (8.0, 20.0), 0.25, 2001, 1.0, 1000.0)
        return k, (2, 0)
    raise ValueError(name)


CASES = ("spheres256_1000", "ellipsoids256", "lognormal128", "slab512_1000")


def solve(k, direction):
    """One observed PCG run; returns the record of the golden file."""
    (k0, k1, k2), lens = O.permute_medium(k, k, k, (1.0, 1.0, 1.0), direction)
    f = O.face_conductances(k0, k1, k2, lens)
    kref = O.reference_parameters(O.group_extrema(f))
    b = O.right_hand_side(f, 1.0, 0.0)
    seen = {}

    def watch(it, p, relres):
        for t in THRESHOLDS:
            if t not in seen and relres <= t:
                seen[t] = (it, O.outflow_etc(f, p, lens, 1.0, 0.0))

    res = O.pcg(f, b, kref, rtol=RTOL_FINAL, maxit=MAXIT, on_iterate=watch)
    kap = O.outflow_etc(f, res.p, lens, 1.0, 0.0)
    ken = O.energy_etc(f, res.p, b, lens, 1.0, 0.0)
    true_rel = float(((b - O.apply_operator(f, res.p)) ** 2).sum() ** 0.5
                     / (b ** 2).sum() ** 0.5)
    return seen, res.iters, res.relres, true_rel, kap, ken


def main(argv):
    cases = argv or list(CASES)
    if not os.path.exists(OUT):
        with open(OUT, "w") as fh:
            fh.write("# kappa_eff of the workloads named in make_workload_goldens.py, written by\n"
                     "# that script from the CPU oracle only (Algorithms 1-3, centred LP optimum,\n"
                     "# x0 = 0, p_in = 1, p_out = 0, unit cube).  One fresh PCG run per row;\n"
                     "# kappa_eff (outflow, Eq. effective formula dis) at the first pass with\n"
                     "# relres <= 1e-8 and <= 1e-10, and at the end of the run (rtol 1e-12);\n"
                     "# kappa_energy is the energy identity at the end (cross-check).\n"
                     "# case dir it_1e-8 kappa_1e-8 it_1e-10 kappa_1e-10 it_end relres_end"
                     " true_relres_end kappa_end kappa_energy_end\n")
    for name in cases:
        t0 = time.time()
        k, dirs = workload(name)
        for d in dirs:
            seen, it, rel, trel, kap, ken = solve(k, d)
            i8, k8 = seen.get(1e-8, (-1, float("nan")))
            i10, k10 = seen.get(1e-10, (-1, float("nan")))
            line = (f"{name} {d} {i8} {k8:.17g} {i10} {k10:.17g} {it} {rel:.3e} {trel:.3e} "
                    f"{kap:.17g} {ken:.17g}\n")
            with open(OUT, "a") as fh:
                fh.write(line)
            print(f"{line.strip()}  ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
