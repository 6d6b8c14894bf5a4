"""Objective targets for the "time to oracle-best" measurement -- test infrastructure.

Runs the FP64 oracle (``oracle.pdbo.run``) on a subset of the restarts of a benchmark workload
for the workload's full iteration count and records the best objective it reaches.  The GPU run
starts the same restarts from the same x^0 (the SplitMix64 rule keyed by seed, restart and
coordinate), so the target is the value the oracle's own run of those restarts attains.

Usage (writes tests/golden/oracle_targets.json; takes a few minutes and ~12 GB of host memory
for the n = 20,000 workload):

    python -m oracle.targets
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

from . import pdbo as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "golden", "oracle_targets.json")


def dense_target(n=20000, restarts_sub=4, iters=2000, eval_every=50, seed=0):
    sys.path.insert(0, ROOT)
    import workloads as W
    Q, c = W.dense_qubo(n, seed=seed)
    p = W.dense_params(Q, restarts=restarts_sub, iters=iters, eval_every=eval_every, seed=seed)
    t0 = time.time()
    out = O.run(Q, c, **p.asdict())
    el = time.time() - t0
    trace = [int(F.min()) for _, F in out["evals"]]
    return {
        "workload": f"dense QUBO n={n}, entries U[-100,100], seed {seed}",
        "restarts": list(range(restarts_sub)), "iters": iters, "eval_every": eval_every,
        "params": p.asdict(), "F_best": out["F_star"], "t_best": out["t_star"], "r_best": out["r_star"],
        "trace_min_F": trace, "oracle_seconds": round(el, 1),
        "how": "oracle.pdbo.run (FP64) on restarts 0..R-1 of the workload; written by oracle/targets.py",
    }


def main():
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["dense_n20000_b1024_seed0"] = dense_target()
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps({k: {"F_best": v["F_best"], "t_best": v["t_best"]} for k, v in data.items()}))


if __name__ == "__main__":
    main()
