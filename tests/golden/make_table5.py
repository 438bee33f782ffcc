"""Writes tests/golden/table5_oracle.json: the FP64 oracle (oracle/ only) on the
lid-driven porous cavity of Sec. 4.3 with eps = 0.6 (128 x 128, Gr = 1e2, Re = 100,
Da = 0.1, Pr = 1, Le = 1, U0 = 0.1) for N = -1500 and -500, with the paper's
equilibria and with the coupled equilibria of model A (Eqs. 30-32), each run until
the mean Nu and Sh of the bottom wall change by less than 1e-7 (relative) over
20,000 steps.  Table 5 of the paper prints these means: equal for the paper's
model, different for model A.

Usage: python tests/golden/make_table5.py
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

ARGS = dict(nx=128, ny=128, Re=100.0, Gr=1e2, Da=0.1, eps=0.6, Pr=1.0, Le=1.0)


def run(job):
    N, model_a = job
    from oracle import oracle as O
    O.set_threads(1)
    p = O.derive_lid(ARGS["nx"], ARGS["ny"], ARGS["Re"], ARGS["Gr"], ARGS["Da"], ARGS["eps"],
                     ARGS["Pr"], ARGS["Le"], N)
    if model_a:
        O.to_model_a(p)
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
    print(N, model_a, o.t, ns.tolist(), f"{time.time() - t0:.0f}s", flush=True)
    return {"N": N, "model_a": model_a, "steps": int(o.t), "nu_bottom": float(ns[0]),
            "sh_bottom": float(ns[1]), "nu_top": float(ns[2]), "sh_top": float(ns[3])}


def main():
    jobs = [(N, ma) for N in (-1500.0, -500.0) for ma in (False, True)]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        rows = pool.map(run, jobs)
    out = {"source": "oracle/ (FP64 CPU), tests/golden/make_table5.py",
           "case": "Sec. 4.3 lid-driven porous cavity, 128 x 128, Gr 1e2, eps 0.6, Re 100, Da 0.1, "
                   "Pr 1, Le 1, U0 0.1, seed 11, halfway walls",
           "rows": rows}
    with open(os.path.join(HERE, "table5_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
