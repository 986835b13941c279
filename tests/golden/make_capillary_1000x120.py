"""Writes capillary_1000x120.json: the FP64 oracle's capillary filling run
(Sec. VI) on the 1000 x 120 set-up (reservoir 200 x 120, channel 800 x 40,
h(60 degrees) on the channel walls, MRT, tau_alpha 1.5 / tau_beta 0.6),
100000 steps: front position x_front, filled length l = x_front - 199.5 and
advancing angle every 500 steps, for both readings of the Step-2 momentum
rates.  A run whose fields turn non-finite is recorded with the first
checkpoint at which they were.

Calls only the oracle.  Usage: python tests/golden/make_capillary_1000x120.py
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


def run(c, relax):
    p = oracle.params(**c["params"], step2_relax_momentum=relax)
    lat = oracle.OracleLattice(p, c["nx"], c["ny"])
    lat.init_channel(c["res_len"], c["ch_w"], oracle.wetting_h(c["theta"]), c["h_block"])
    y0 = (c["ny"] - c["ch_w"]) // 2
    fl = lat.cls == 0
    rho0 = float(lat.moments()[0][fl].sum())
    rec = {"step2_relax_momentum": relax, "t": [], "x_front": [], "l": [], "theta": [],
           "diverged_at": None}
    t0 = time.time()
    while lat.t < c["steps"]:
        lat.step(c["every"])
        rho, phi, ux, uy = lat.moments()
        if not np.isfinite(phi[fl]).all():
            rec["diverged_at"] = lat.t
            break
        xf, th, _ = oracle.meniscus(phi, lat.cls, c["res_len"], c["nx"], y0, y0 + c["ch_w"])
        rec["t"].append(lat.t)
        rec["x_front"].append(xf)
        rec["l"].append(xf - (c["res_len"] - 0.5))
        rec["theta"].append(th)
        if lat.t % 10000 == 0:
            print("relax" if relax else "literal", lat.t, "l=%.3f theta=%.2f" % (rec["l"][-1], th),
                  "%.0fs" % (time.time() - t0), flush=True)
    if rec["diverged_at"] is None:
        rec["mass_drift"] = float(rho[fl].sum()) - rho0
        rec["max_u"] = float(np.hypot(ux, uy)[fl].max())
    return rec


def main():
    c = lbinputs.CAPILLARY_1000x120
    out = {"source": "FP64 oracle via tests/golden/make_capillary_1000x120.py",
           "nx": c["nx"], "ny": c["ny"], "res_len": c["res_len"], "ch_w": c["ch_w"],
           "theta": c["theta"], "steps": c["steps"], "every": c["every"],
           "runs": [run(c, False), run(c, True)]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "capillary_1000x120.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
