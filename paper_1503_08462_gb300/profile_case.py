"""A short, fixed launch sequence of the hot path for single-kernel profiler captures.

    python -m paper_1503_08462_gb300.profile_case vcycle LEVEL [--width W]
    python -m paper_1503_08462_gb300.profile_case defect LEVEL [--width W]

builds the L-shape workload (domain (-1,1)^2 minus [0,1)x(-1,0], h = 1/512, N = 784,385, seed 2,
Ruge-Stueben hierarchy with a 400-row coarse cap), loads it and runs ONE float32 V-cycle from
LEVEL on a seeded N_LEVEL x W block through the public ``amgeig_apply_vcycle`` call (W = 28
columns by default: the 20 wanted pairs plus 8 buffer vectors of the timed solve).  The first
``k_smooth_f4`` launch of the process is LEVEL's pre-smoothing sweep and the first ``k_spmm_f4``
launch is LEVEL's restriction, with only a format conversion before them, so a profiler can
take them with ``-k regex:<kernel> -c 1`` and nothing else in flight.  ``defect LEVEL`` runs
the defect r_j = lambda_j M u_j - A u_j of the same block through ``amgeig_apply_defect``
(one ``k_defect_df`` launch in the mixed precision, after one conversion).
"""

import argparse

import numpy as np

from . import amgeig as ae
from .inputs import hierarchy, meshes


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("mode", choices=["vcycle", "defect"])
    ap.add_argument("level", type=int)
    ap.add_argument("--width", type=int, default=28)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    args = ap.parse_args(argv)
    p = meshes.lshape_2d(m_half=512, seed=2)
    blob, h = hierarchy.problem_blob(p, coarse_cap=400)
    prec = ae.AMGEIG_MIXED_FP32 if args.precision == "mixed" else ae.AMGEIG_FP64
    with ae.Hierarchy(blob) as hh:
        if not 0 <= args.level < len(hh.sizes):
            raise SystemExit(f"level must be in [0, {len(hh.sizes) - 1}]")
        n = hh.sizes[args.level]
        b = np.random.default_rng(0).standard_normal((n, args.width))
        if args.mode == "defect":
            lam = np.linspace(10.0, 400.0, args.width)
            r, rr = ae.amgeig_apply_defect(hh.handle, args.level, b, lam, ae.options(precision=prec))
            print(f"defect level {args.level}: {n} rows x {args.width} columns, |r| = {float(np.linalg.norm(r)):.6e}")
            return
        x = ae.amgeig_apply_vcycle(hh.handle, args.level, b, ae.options(precision=prec))
        print(f"vcycle level {args.level}: {n} rows x {args.width} columns, |x| = {float(np.linalg.norm(x)):.6e}")


if __name__ == "__main__":
    main()
