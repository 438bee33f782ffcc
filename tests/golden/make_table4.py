"""Writes tests/golden/table4_oracle.json: the FP64 oracle (oracle/ only) on the
lid-driven porous cavity of Sec. 4.3 (128 x 128, Gr = 1e2, eps = 0.95, Re = 100,
Da = 0.1, Pr = 1, Le = 1, U0 = 0.1) for several buoyancy ratios N, each run until
the mean Nu and Sh of the bottom wall change by less than 1e-7 (relative) over
20,000 steps.  Table 4 of the paper prints Nu = Sh at the bottom wall.

With --nee the same cavity is run with the paper's own walls (Sec. 3.3: 129 x 129 nodes
on the walls, L = 128) into tests/golden/table4_nee_oracle.json.

Usage: python tests/golden/make_table4.py [N values, comma separated] [--nee]
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

ARGS = dict(nx=128, ny=128, Re=100.0, Gr=1e2, Da=0.1, eps=0.95, Pr=1.0, Le=1.0)


def run(job):
    N, nee = job
    from oracle import oracle as O
    O.set_threads(1)
    n = 1 if nee else 0
    p = O.derive_lid(ARGS["nx"] + n, ARGS["ny"] + n, ARGS["Re"], ARGS["Gr"], ARGS["Da"],
                     ARGS["eps"], ARGS["Pr"], ARGS["Le"], N, nee=nee)
    o = O.Oracle(p, seed=11, noise=1e-3)
    prev = None
    t0 = time.time()
    while True:
        o.step(20000)
        ns = o.nusselt_sherwood_tb()
        if prev is not None and np.max(np.abs(ns[:2] - prev[:2]) / np.abs(ns[:2])) < 1e-7:
            break
        prev = ns
        if o.t >= 2_000_000:
            break
    print(N, o.t, ns.tolist(), f"{time.time() - t0:.0f}s", flush=True)
    return {"N": N, "steps": int(o.t), "nu_bottom": float(ns[0]), "sh_bottom": float(ns[1]),
            "nu_top": float(ns[2]), "sh_top": float(ns[3])}


def main():
    nee = "--nee" in sys.argv
    args = [a for a in sys.argv[1:] if a != "--nee"]
    Ns = [float(x) for x in args[0].split(",")] if args else \
        [-1500.0, -500.0, -100.0, 100.0, 500.0]
    with mp.get_context("spawn").Pool(len(Ns)) as pool:
        rows = pool.map(run, [(N, nee) for N in Ns])
    out = {"source": "oracle/ (FP64 CPU), tests/golden/make_table4.py",
           "case": "Sec. 4.3 lid-driven porous cavity, 128 x 128, Gr 1e2, eps 0.95, Re 100, "
                   "Da 0.1, Pr 1, Le 1, U0 0.1, seed 11"
                   + (", walls on nodes (129 x 129 nodes, Sec. 3.3)" if nee else ", halfway walls"),
           "rows": rows}
    name = "table4_nee_oracle.json" if nee else "table4_oracle.json"
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
