"""Writes sweep_200x100.json: FP64 oracle results for the 200x100 sessile-drop
sweep (BGK; MRT with the literal conserved-moment rates of Eq. diag; MRT with
the momentum rows relaxed on Step-2 nodes; viscosity ratio 1: tau 1/1, ratio
10: tau_alpha 1.5 in the drop, tau_beta 0.6 outside; wetting gradient of
Eq. (theory) for 60, 90 and 120 degrees; drop radius 40 on the bottom wall;
20000 steps).  A run whose fields turn non-finite is recorded with the first
checkpoint (every 500 steps) at which they were.

Calls only the oracle.  Usage: python tests/golden/make_sweep_200x100.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbinputs  # noqa: E402
import oracle  # noqa: E402


def run_case(c, coll, relax, ta, tb, theta):
    p = oracle.params(**lbinputs.BASE, collision=coll, tau_alpha=ta, tau_beta=tb,
                      h_bottom=oracle.wetting_h(theta), h_top=0.0,
                      step2_relax_momentum=relax)
    lat = oracle.OracleLattice(p, c["nx"], c["ny"])
    lat.init_drop(c["R"], c["cx"], c["cy"])
    case = {"collision": coll, "step2_relax_momentum": relax, "tau_alpha": ta,
            "tau_beta": tb, "theta_target": theta, "h": oracle.wetting_h(theta),
            "diverged_at": None}
    done = 0
    while done < c["steps"]:
        k = min(c["check_every"], c["steps"] - done)
        lat.step(k)
        done += k
        rho, phi, ux, uy = lat.moments()
        if not (np.isfinite(rho).all() and np.isfinite(phi).all()):
            case["diverged_at"] = done
            return case
    th, R, xc, yc = oracle.contact_angle(phi)
    case.update({"theta": th, "R_fit": R, "xc": xc, "yc": yc,
                 "max_u": float(np.hypot(ux, uy).max()),
                 "mass": float(rho.sum()), "order": float(phi.sum())})
    return case


def main():
    c = lbinputs.SWEEP_200x100
    out = {"source": "FP64 oracle (oracle/lb_oracle.c) via tests/golden/make_sweep_200x100.py",
           "nx": c["nx"], "ny": c["ny"], "R": c["R"], "steps": c["steps"], "cases": []}
    for coll, relax in c["variants"]:
        for ratio, (ta, tb) in c["tau_pairs"].items():
            for theta in c["angles"]:
                t0 = time.time()
                case = run_case(c, coll, relax, ta, tb, theta)
                case["ratio"] = ratio
                out["cases"].append(case)
                res = ("diverged by step %d" % case["diverged_at"] if case["diverged_at"]
                       else "%.3f max|u| %.3e" % (case["theta"], case["max_u"]))
                print(coll, "relax" if relax else "literal", ratio, theta, "->", res,
                      "%.0fs" % (time.time() - t0), flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_200x100.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
