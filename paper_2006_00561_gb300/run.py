"""Command-line population-annealing run on one GPU.

    python -m paper_2006_00561_gb300.run --dim 3 --L 8 --model pmj --R0 4194304 --K 150 \
        --beta-max 3 --steps 3

Creates one run (Sec. 2: initial population at beta0, then per step the
reweight of Eq. 3 / 4, resampling, theta Metropolis sweeps and the
measurement), advances it by --steps steps (all K when omitted) and prints
the last step's observables, with the device time per step, as one JSON line.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None) -> dict:
    import torch

    from . import pa as P
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--L", type=int, default=64)
    ap.add_argument("--model", choices=["ferro", "pmj"], default="ferro")
    ap.add_argument("--layout", choices=["packed", "int8"], default="packed")
    ap.add_argument("--R0", type=int, default=1 << 17)
    ap.add_argument("--K", type=int, default=200)
    ap.add_argument("--theta", type=int, default=10)
    ap.add_argument("--beta0", type=float, default=0.0)
    ap.add_argument("--beta-max", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--coupling-seed", type=int, default=0)
    ap.add_argument("--resample", choices=["nearest", "poisson", "multinomial"], default="nearest")
    ap.add_argument("--heat", action="store_true", help="start from the ground state")
    ap.add_argument("--steps", type=int, default=None)
    a = ap.parse_args(argv)
    cfg = P.make_config(
        dim=a.dim, L=a.L, model=P.MODEL_PMJ if a.model == "pmj" else P.MODEL_FERRO,
        layout=P.LAYOUT_PACKED if a.layout == "packed" else P.LAYOUT_INT8, K=a.K, theta=a.theta,
        R0=a.R0, beta0=a.beta0, beta_max=a.beta_max, seed=a.seed, coupling_seed=a.coupling_seed,
        init=P.INIT_GROUND if a.heat else P.INIT_RANDOM,
        resample={"nearest": P.RESAMPLE_NEAREST, "poisson": P.RESAMPLE_POISSON,
                  "multinomial": P.RESAMPLE_MULTINOMIAL}[a.resample])
    stream = torch.cuda.Stream()
    run = P.Run(cfg, stream=stream)
    steps = a.K if a.steps is None else min(a.steps, a.K)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        run.step()
    e1.record(stream)
    torch.cuda.synchronize()
    out = run.observables()
    out["ms_per_step"] = e0.elapsed_time(e1) / max(steps, 1)
    run.close()
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
