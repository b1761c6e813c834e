"""Writes tests/golden/oracle_trace.json from the CPU oracle alone.

The file freezes the oracle's per-step trace for two small runs (the config-1
workload for 12 steps, and a 3D +-J instance for 8 steps) so that any later
change of the oracle's arithmetic shows up in tests/test_oracle_golden.py.
Run:  python tests/golden/make_oracle_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

RUNS = {
    "ising2d_L16_R1000": dict(dim=2, L=16, R0=1000, K=100, theta=10, seed=1, steps=12),
    "ea3d_L6_R500": dict(dim=3, L=6, model=O.MODEL_PMJ, R0=500, K=50, theta=10, beta_max=3.0,
                         seed=4, coupling_seed=77, instance_id=3, steps=8),
}


def trace(spec: dict) -> list:
    spec = dict(spec)
    steps = spec.pop("steps")
    run = O.Run(O.make_config(**spec))
    rows = []
    for i in range(steps + 1):
        if i > 0:
            assert run.step() == 0
        o = run.observables()
        rows.append({
            "step": int(o["step"]), "R": int(o["R"]),
            "sumE": int(o["sumE"]), "sumE2": int(o["sumE2"]),
            "sumAbsM": int(o["sumAbsM"]), "sumM2": int(o["sumM2"]),
            "lnZ": float(o["lnZ"]).hex(),
            "spins_sha256": hashlib.sha256(run.spins().tobytes()).hexdigest(),
            "counts_sha256": hashlib.sha256(run.counts().tobytes()).hexdigest() if i else None,
        })
    return rows


def main():
    out = {"note": "written by tests/golden/make_oracle_golden.py from oracle/ only",
           "runs": {name: {"spec": spec, "trace": trace(spec)} for name, spec in RUNS.items()}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_trace.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
