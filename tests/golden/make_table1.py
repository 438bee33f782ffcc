"""Writes tests/golden/table1_oracle.json: the FP64 oracle (oracle/ only) run on the
non-porous double-diffusive cavity of Sec. 4.1 (aspect ratio 2, 100 x 200, Ra = 1e5,
Pr = 1, Le = 2, N = -0.8, eps = 1, Da = 1e8, Ma = 0.1) until the mean Nu and Sh
change by less than 1e-6 (relative) over 50,000 steps.  Table 1 of the paper
prints Nu = 3.402, Sh = 4.398, |u_x|max = 39.275, |u_y|max = 86.375 for its own
(node-based) wall scheme.

With --nee the same cavity is run with the paper's own walls (Sec. 3.3: 101 x 201
nodes on the walls, L = 100) into tests/golden/table1_nee_oracle.json.

Usage: python tests/golden/make_table1.py [threads] [--nee]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import oracle as O  # noqa: E402

NX, NY = 100, 200
ARGS = (NX, NY, 1e5, 1e8, 1.0, 1.0, 2.0, -0.8)


def main():
    nee = "--nee" in sys.argv
    args = [a for a in sys.argv[1:] if a != "--nee"]
    threads = int(args[0]) if args else (os.cpu_count() or 1)
    O.set_threads(threads)
    p = O.derive(NX + 1, NY + 1, *ARGS[2:], nee=True) if nee else O.derive(*ARGS)
    o = O.Oracle(p, seed=7, noise=1e-3)
    chunk = 50000
    prev = None
    t0 = time.time()
    while True:
        o.step(chunk)
        ns = o.nusselt_sherwood()
        print(o.t, ns.tolist(), f"{time.time() - t0:.0f}s", flush=True)
        if prev is not None and np.max(np.abs(ns - prev) / np.abs(ns)) < 1e-6:
            break
        prev = ns
        if o.t >= 3_000_000:
            break
    fl = o.fields()
    alpha = p.nu / p.Pr
    out = {
        "source": "oracle/ (FP64 CPU), tests/golden/make_table1.py",
        "case": "Sec. 4.1 cavity: 100 x 200, Ra 1e5, Pr 1, Le 2, N -0.8, eps 1, Da 1e8, seed 7"
                + (", walls on nodes (101 x 201 nodes, Sec. 3.3)" if nee else ", halfway walls"),
        "steps": int(o.t),
        "nu_left": float(ns[0]), "sh_left": float(ns[1]), "nu_right": float(ns[2]),
        "sh_right": float(ns[3]),
        "ux_max_alpha_over_L": float(np.abs(fl["ux"]).max() * NX / alpha),
        "uy_max_alpha_over_L": float(np.abs(fl["uy"]).max() * NX / alpha),
    }
    name = "table1_nee_oracle.json" if nee else "table1_oracle.json"
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
