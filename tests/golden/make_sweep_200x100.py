"""Writes sweep_200x100.json: FP64 oracle results for the 200x100 sessile-drop
sweep (BGK and MRT; viscosity ratio 1: tau 1/1, ratio 10: tau_alpha 1.5 in
the drop, tau_beta 0.6 outside; wetting gradient of Eq. (theory) for 60, 90
and 120 degrees; drop radius 40 on the bottom wall; 20000 steps).

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


def main():
    c = lbinputs.SWEEP_200x100
    out = {"source": "FP64 oracle (oracle/lb_oracle.c) via tests/golden/make_sweep_200x100.py",
           "nx": c["nx"], "ny": c["ny"], "R": c["R"], "steps": c["steps"], "cases": []}
    for coll in c["collisions"]:
        for ratio, (ta, tb) in c["tau_pairs"].items():
            for theta in c["angles"]:
                p = oracle.params(**lbinputs.BASE, collision=coll, tau_alpha=ta, tau_beta=tb,
                                  h_bottom=oracle.wetting_h(theta), h_top=0.0)
                lat = oracle.OracleLattice(p, c["nx"], c["ny"])
                lat.init_drop(c["R"], c["cx"], c["cy"])
                t0 = time.time()
                lat.step(c["steps"])
                rho, phi, ux, uy = lat.moments()
                th, R, xc, yc = oracle.contact_angle(phi)
                case = {"collision": coll, "ratio": ratio, "tau_alpha": ta, "tau_beta": tb,
                        "theta_target": theta, "h": oracle.wetting_h(theta),
                        "theta": th, "R_fit": R, "xc": xc, "yc": yc,
                        "max_u": float(np.hypot(ux, uy).max()),
                        "mass": float(rho.sum()), "order": float(phi.sum())}
                out["cases"].append(case)
                print(coll, ratio, theta, "->", round(th, 3), "max|u| %.3e" % case["max_u"],
                      "%.0fs" % (time.time() - t0), flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_200x100.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
