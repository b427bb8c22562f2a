"""Run one configuration of the pad update (or of the surrogate network) a
few times, for a profiler to capture.

    python -m paper_2105_08798_gb300.profile_case --workload NAME --precision P [--applies N] [--rhs R] [--L L]
    python -m paper_2105_08798_gb300.profile_case --workload NAME --hmatrix [--applies N] [--rhs R] [--L L]
    python -m paper_2105_08798_gb300.profile_case --mlp-rows N [--width H] [--applies N]

The first form builds a plan for a named workload, tabulates it and runs
``--applies`` pad updates at the given precision on device-resident inputs
(``--rhs R``, ``--L L``: the workload's ring geometry with R right-hand sides
and L repeats, for a capture that holds fewer bytes on the device);
with ``--hmatrix`` it builds the H-matrix of the plan's Green matrix (eps 1e-5,
gamma 2, b_min 20) and runs its applies instead;
the last runs the fused surrogate network on N rows of random features.
Exits non-zero on any error; prints one line of timings.
"""

from __future__ import annotations

import argparse
import sys
import time


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="ring4000x6000_L256_rhs64_iso")
    ap.add_argument("--precision", default="bf16x2")
    ap.add_argument("--applies", type=int, default=2)
    ap.add_argument("--rhs", type=int, default=0, help="right-hand sides (default: the workload's)")
    ap.add_argument("--L", type=int, default=0, help="repeats along the line (default: the workload's)")
    ap.add_argument("--hmatrix", action="store_true", help="apply the H-matrix of the plan's Green matrix")
    ap.add_argument("--mlp-rows", type=int, default=0)
    ap.add_argument("--width", type=int, default=128)
    args = ap.parse_args(argv)

    import torch

    from . import build, fbc, inputs

    build.build()
    fbc.load()
    if args.mlp_rows:
        with fbc.Surrogate(width=args.width, seed=1) as S:
            x = torch.rand((args.mlp_rows, 4), device="cuda") * 2 - 1
            for _ in range(args.applies):
                S.forward(x, bf16_weights=True)
            S.sync_status()
        print(f"surrogate forward: {args.applies} x {args.mlp_rows} rows, width {args.width}")
        return 0
    w = inputs.WORKLOADS[args.workload]
    R = args.rhs if args.rhs > 0 else w.n_rhs
    L = args.L if args.L > 0 else w.L
    xy_i, xy_p = w.geometry()
    with fbc.Plan(xy_i, xy_p, L, w.material, precision=args.precision, max_rhs=R) as plan:
        H = None
        if args.hmatrix:
            H = fbc.HMatrix(plan)
        else:
            plan.tabulate()
        op = H if H is not None else plan
        fd = torch.from_numpy(inputs.forces(R, w.n_i, L, w.seed)).cuda()
        ud = torch.zeros((R, w.n_p, L, 3), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        times = []
        for _ in range(args.applies):
            t0 = time.perf_counter()
            op.apply(fd, ud)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        if H is not None:
            info = H.info()
            H.close()
        else:
            plan.sync_status()
    what = "hmatrix" if args.hmatrix else args.precision
    extra = (f" (factors {info['factor_bytes'] / 1e9:.2f} GB, rank sum {info['rank_sum']}, build {info['build_ms'] / 1e3:.1f} s)"
             if args.hmatrix else "")
    print(f"{w.name} L {L} rhs {R} {what}: applies " + " ".join(f"{t * 1e3:.1f} ms" for t in times) + extra)
    return 0


if __name__ == "__main__":
    sys.exit(main())
