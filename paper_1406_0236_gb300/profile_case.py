"""Run one operator of the library on a named workload, for profilers and timing.

    python -m paper_1406_0236_gb300.profile_case --workload spheroids8_258560 \
        --op interbody32 --repeat 2 [--rhs 1] [--autotune] [--engine -1] [--modal-engine -1] \
        [--fp64-engine -1] [--accel-eps 1e-8]

ops: interbody32, interbody64, interbody_df (B sigma), local_inverse64, local_inverse32 (D^{-1} y),
apply64, apply32, solve_mixed, solve_fp64, compress.  Prints the mean time per call measured
with CUDA events.  Inputs are seeded random densities (ops) or the workload's plane
waves (solves).  --engine picks the FP32 inter-body engine and --modal-engine the FP32
modal GEMM engine (see Solver.set_interbody_engine / set_modal_engine; -1 automatic).
--accel-eps > 0 computes the skeletons of the accelerated scheme (Sec. 5) first, so the
solves run on the reduced system; compress times the skeleton computation itself.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="spheroids8_258560")
    ap.add_argument("--op", default="interbody32")
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--rhs", type=int, default=1)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--engine", type=int, default=-1)
    ap.add_argument("--modal-engine", type=int, default=-1)
    ap.add_argument("--fp64-engine", type=int, default=-1,
                    help="FP64 / double-float inter-body engine (Solver.set_fp64_interbody_engine)")
    ap.add_argument("--accel-eps", type=float, default=0.0)
    args = ap.parse_args()

    import numpy as np
    import torch

    import workloads as W
    from paper_1406_0236_gb300 import Options, Solver

    wl = W.by_name(args.workload)
    prec = 1 if args.op.endswith("32") or args.op == "solve_mixed" else (2 if args.op.endswith("_df") else 0)
    s = Solver.from_workload(wl, Options(precision=min(prec, 1), gmres_tol=1e-8, verify_final=0),
                             stream=torch.cuda.current_stream().cuda_stream)
    s.set_interbody_engine(args.engine)
    s.set_modal_engine(args.modal_engine)
    s.set_fp64_interbody_engine(args.fp64_engine)
    needs_build = not args.op.startswith("interbody")
    if needs_build:
        s.build_scattering_matrices()
    if args.autotune:
        s.autotune(args.rhs, 1 if prec == 1 else 2)
    if args.accel_eps > 0 and args.op != "compress":
        s.compress(args.accel_eps)
    N = s.N
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn((N, args.rhs), dtype=torch.complex128, device="cuda", generator=g)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dirs = W.uniform_directions(args.rhs, 3) if args.rhs > 1 else np.array([[0, 0, 1.0]])

    def run():
        if args.op.startswith("interbody"):
            s.interbody(x, precision=prec)
        elif args.op.startswith("local_inverse"):
            s.local_inverse(x, precision=prec)
        elif args.op.startswith("apply"):
            s.apply(x, precision=prec)
        elif args.op == "compress":
            s.compress(args.accel_eps)
        else:
            s.solve_plane_waves(dirs)

    run()
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.repeat):
        run()
    ev1.record()
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "op": args.op, "rhs": args.rhs, "N": N,
                      "ms_per_call": ev0.elapsed_time(ev1) / args.repeat}))


if __name__ == "__main__":
    main()
