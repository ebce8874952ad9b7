"""Error of the reduced-precision storage modes against the FP64 oracle (not collected by pytest).

The 3-D cavity at Re = 1000 (lid u = 0.1, tau = 3 u N / Re + 1/2) on an N^3 lattice is run for a
number of steps by the CUDA library in FP32, FP16-shifted and BF16-shifted storage (and FP64), and
by the FP64 oracle; the script prints, per storage type, the error of the populations, density,
velocity, per-cell sensor and 16^3 block maxima, and the agreement of the top-10 % and threshold
flags.  Run on a GPU machine:

    python tests/precision_report.py --n 128 --steps 5000
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--re", type=float, default=1000.0)
    ap.add_argument("--block", type=int, default=16)
    args = ap.parse_args()

    import __graft_entry__

    __graft_entry__.build()
    import oracle as O
    import paper_1507_06767_gb300 as L

    n, u = args.n, 0.1
    tau = O.tau_from_re(u, n, args.re)
    T = 4.0 * (4.0 / 3.0) * tau * u / n

    gpu = {}
    for name in ("F64", "F32", "F16S", "BF16S"):
        lat = L.Lattice(19, n, n, n, tau, dtype=getattr(L, "LBM_" + name), lid=(u, 0.0))
        L.lbm_set_sensor_field(lat.h, 1)
        t0 = time.perf_counter()
        lat.step(args.steps)
        f = lat.populations()
        gpu[name] = dict(f=f, rho_u=lat.moments(), K=lat.sensor_field(),
                         bmax=lat.sensor(args.block), top=lat.flag_top(0.1, block=args.block),
                         thr=lat.flag(T, block=args.block), secs=time.perf_counter() - t0)
        lat.close()

    o = O.Oracle(19, n, n, n, tau, lid=(u, 0.0, 0.0))
    t0 = time.perf_counter()
    f_ref, K_ref = o.run(o.rest(), args.steps, sensor_last=True)
    oracle_s = time.perf_counter() - t0
    _, rho_ref, u_ref = o.sensor(f_ref)
    bref = O.block_max(K_ref, args.block)
    finite = bool(np.isfinite(f_ref).all())

    report = {"n": n, "steps": args.steps, "re": args.re, "tau": tau, "threshold": T,
              "oracle_finite": finite, "oracle_seconds": round(oracle_s, 1),
              "oracle_threads": O.threads(), "umax_ref": float(np.abs(u_ref).max()),
              "Kmax_ref": float(K_ref.max()), "modes": {}}
    for name, g in gpu.items():
        rho, uu = g["rho_u"]
        ok_top, ncmp_top, nex_top = O.flags_agree(g["top"], bref, "top", 0.1, 1e-4)
        ref_top = O.flags_top(bref, 0.1)
        ref_thr = O.flags_threshold(bref, T)
        report["modes"][name] = {
            "f_rel": float(np.abs(g["f"] - f_ref).max() / np.abs(f_ref).max()),
            "rho_abs": float(np.abs(rho - rho_ref).max()),
            "u_rel": float(np.abs(uu - u_ref).max() / np.abs(u_ref).max()),
            "K_rel_field": float(np.abs(g["K"] - K_ref).max() / K_ref.max()),
            "K_rel_blockmax": float(np.abs(g["bmax"] - bref).max() / bref.max()),
            "K_rel_blockmax_median": float(np.median(np.abs(g["bmax"] - bref) / bref)),
            "top10_agree": float((g["top"] == ref_top).mean()),
            "top10_agree_outside_1e-4_band": ok_top,
            "threshold_agree": float((g["thr"] == ref_thr).mean()),
            "gpu_seconds": round(g["secs"], 2),
        }
    print(json.dumps(report, indent=1))


if __name__ == "__main__":
    main()
