"""Per-configuration parity report of the GPU path against the FP64 oracle.

Runs each configuration from the same input on the GPU (FP64, FP32 with
full g storage, FP32 with compact g storage) and on the oracle, and prints
one JSON object per case with max |phi - phi_oracle|, max |u - u_oracle|
(over both components) and the contact angle of both sides:
  - the 100 x 50 BGK drop, 2000 steps;
  - the 200 x 100 sweep (BGK, MRT, MRT with the momentum-relaxing Step-2
    reading; viscosity ratio 1 and 10; 60, 90 and 120 degrees), 20000 steps;
  - the 512 x 512 cut of the 8192^2 spinodal MRT workload, 1000 steps.
A side whose run turned non-finite is reported as such.  Test
infrastructure: needs a CUDA device and the compiled oracle.

    python tests/parity_report.py [--only drop|sweep|spinodal]
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lbinputs  # noqa: E402

STORAGES = (("fp64", "fp64", False), ("fp32", "fp32", False), ("fp32c", "fp32", True))


def gpu_run(lbf, kw, nx, ny, init, steps, precision, compact):
    sim = lbf.Lattice(lbf.params(precision=precision, compact_g=compact, **kw), nx, ny)
    try:
        init(sim)
        sim.step(steps)
        _, phi, ux, uy, st = sim.moments()
        if st["nonfinite"]:
            return None
        try:
            theta = sim.contact_angle()[0]
        except Exception:
            theta = None
        return phi, ux, uy, theta
    finally:
        sim.close()


def oracle_run(orc, kw, nx, ny, init, steps):
    lat = orc.OracleLattice(orc.params(**kw), nx, ny)
    init(lat)
    lat.step(steps)
    _, phi, ux, uy = lat.moments()
    if not np.isfinite(phi).all():
        return None
    try:
        theta = orc.contact_angle(phi)[0]
    except Exception:
        theta = None
    return phi, ux, uy, theta


def compare(name, ref, runs, with_angle):
    out = {"case": name}
    out["oracle_theta"] = None if ref is None or not with_angle else round(ref[3], 4)
    for key, res in runs.items():
        if ref is None or res is None:
            out[key] = {"nonfinite": res is None, "oracle_nonfinite": ref is None}
            continue
        d = {"max_dphi": float("%.3e" % np.abs(res[0] - ref[0]).max()),
             "max_du": float("%.3e" % max(np.abs(res[1] - ref[1]).max(),
                                          np.abs(res[2] - ref[2]).max()))}
        if with_angle and res[3] is not None and ref[3] is not None:
            d["theta"] = round(res[3], 4)
            d["dtheta"] = float("%.2e" % abs(res[3] - ref[3]))
        out[key] = d
    print(json.dumps(out), flush=True)


def case(lbf, orc, name, kw, nx, ny, init_gpu, init_orc, steps, with_angle=True):
    ref = oracle_run(orc, kw, nx, ny, init_orc, steps)
    runs = {key: gpu_run(lbf, kw, nx, ny, init_gpu, steps, prec, compact)
            for key, prec, compact in STORAGES}
    compare(name, ref, runs, with_angle)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=("drop", "sweep", "spinodal"), default=None)
    args = ap.parse_args()
    import __graft_entry__

    __graft_entry__.build()
    import oracle as orc
    import paper_0812_1282_gb300 as lbf

    if args.only in (None, "drop"):
        c = lbinputs.DROP_100x50
        drop = lambda s: s.init_drop(c["R"], c["cx"], c["cy"])  # noqa: E731
        case(lbf, orc, "drop_100x50", c["params"], c["nx"], c["ny"], drop, drop, c["steps"])
    if args.only in (None, "sweep"):
        c = lbinputs.SWEEP_200x100
        drop = lambda s: s.init_drop(c["R"], c["cx"], c["cy"])  # noqa: E731
        for coll, relax in c["variants"]:
            for ratio, (ta, tb) in c["tau_pairs"].items():
                for theta in c["angles"]:
                    kw = dict(lbinputs.BASE, collision=coll, tau_alpha=ta, tau_beta=tb,
                              h_bottom=orc.wetting_h(theta), h_top=0.0,
                              step2_relax_momentum=relax)
                    name = "sweep_%s%s_R%d_%g" % (coll, "-relaxj" if relax else "", ratio, theta)
                    case(lbf, orc, name, kw, c["nx"], c["ny"], drop, drop, c["steps"])
    if args.only in (None, "spinodal"):
        c = lbinputs.SPINODAL_8192
        n = c["sub"]
        phi0 = lbinputs.random_field(n, n, c["amp"], c["seed"])
        init = lambda s: s.init_phi(phi0)  # noqa: E731
        case(lbf, orc, "spinodal_512", c["params"], n, n, init, init, c["steps"],
             with_angle=False)


if __name__ == "__main__":
    main()
