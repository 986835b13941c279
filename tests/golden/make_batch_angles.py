"""Writes batch_angles.json: the FP64 oracle's contact angle after 10000
steps for the 16 smallest domains of the batched sessile-drop workload
(lbinputs.batch_specs: seed 2026, sides 64..512, theta 30..150 degrees,
viscosity ratio 1, 3 or 10; MRT), for both readings of the Step-2 momentum
rates.  A run whose fields turn non-finite is recorded as diverged.

Calls only the oracle.  Usage: python tests/golden/make_batch_angles.py
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

STEPS = 10000
N_SMALLEST = 16


def main():
    specs = lbinputs.batch_specs()
    order = sorted(range(len(specs)), key=lambda d: (specs[d]["nx"] * specs[d]["ny"], d))
    out = {"source": "FP64 oracle via tests/golden/make_batch_angles.py", "steps": STEPS,
           "domains": []}
    for d in order[:N_SMALLEST]:
        s = specs[d]
        rec = {"dom": d, "nx": s["nx"], "ny": s["ny"], "theta_target": s["theta"],
               "ratio": s["ratio"]}
        for relax in (False, True):
            p = oracle.params(**lbinputs.BASE, collision="mrt", tau_alpha=s["tau_alpha"],
                              tau_beta=s["tau_beta"], h_bottom=oracle.wetting_h(s["theta"]),
                              h_top=0.0, step2_relax_momentum=relax)
            lat = oracle.OracleLattice(p, s["nx"], s["ny"])
            lat.init_drop(s["R"], s["cx"], s["cy"])
            t0 = time.time()
            lat.step(STEPS)
            _, phi, ux, uy = lat.moments()
            key = "relax" if relax else "literal"
            if not np.isfinite(phi).all():
                rec[key] = {"diverged": True}
            else:
                rec[key] = {"diverged": False, "theta": oracle.contact_angle(phi)[0],
                            "max_u": float(np.hypot(ux, uy).max())}
            print(d, s["nx"], s["ny"], round(s["theta"], 1), s["ratio"], key, rec[key],
                  "%.0fs" % (time.time() - t0), flush=True)
        out["domains"].append(rec)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_angles.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
