"""Runs the CPU oracle and the CUDA engine side by side on the same seeded
configuration and compares them after every step (test helper)."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

OBS_INT = ("step", "R", "sumE", "sumE2", "sumAbsM", "sumM2")
OBS_FP = ("beta", "lnQ", "lnZ", "e", "cv", "m_abs", "chi")
FP_RTOL = 1e-12  # FP64 observables: ln() may differ in the last ulp, the rest is exact IEEE


def configs(P, dim=2, L=16, model=0, layout=1, R0=1000, K=100, theta=10, beta0=0.0,
            beta_max=1.0, seed=1, coupling_seed=0, instance_id=0, capacity=0, init=0,
            resample=0):
    o = O.make_config(dim=dim, L=L, model=model, K=K, theta=theta, instance_id=instance_id,
                      R0=R0, capacity=capacity, beta0=beta0, beta_max=beta_max, seed=seed,
                      coupling_seed=coupling_seed, init=init, resample=resample)
    g = P.make_config(dim=dim, L=L, model=model, layout=layout, K=K, theta=theta,
                      instance_id=instance_id, R0=R0, capacity=capacity, beta0=beta0,
                      beta_max=beta_max, seed=seed, coupling_seed=coupling_seed, init=init,
                      resample=resample)
    return o, g


def close(a: float, b: float, rtol=FP_RTOL) -> bool:
    return abs(a - b) <= rtol * max(1.0, abs(a), abs(b))


def compare_obs(go: dict, oo: dict, where=""):
    for k in OBS_INT:
        assert go[k] == oo[k], (where, k, go[k], oo[k])
    for k in OBS_FP:
        assert close(go[k], oo[k]), (where, k, go[k], oo[k])


def compare_state(P, grun, orun, step: int, full_spins=True):
    where = f"step {step}"
    st = grun.state()
    assert st["status_bits"] == 0, (where, st)
    assert st["step"] == orun.step_index == step, where
    assert st["R"] == orun.R, (where, st["R"], orun.R)
    assert st["parity"] == orun.parity
    if full_spins:
        assert np.array_equal(grun.spins(), orun.spins()), where
    assert np.array_equal(grun.dump(P.DUMP_EBIN), orun.ebin()), where
    assert np.array_equal(grun.dump(P.DUMP_MAG), orun.mag()), where
    assert np.array_equal(grun.dump(P.DUMP_HIST), orun.hist()), where
    if step > 0:
        assert st["R_prev"] == orun.R_prev, where
        assert st["kref"] == orun.kref, where
        assert st["S"] == orun.S, (where, st["S"], orun.S)
        assert np.array_equal(grun.dump(P.DUMP_TAB_N), orun.tab_n()), where
        assert np.array_equal(grun.dump(P.DUMP_TAB_F), orun.tab_F()), where
        assert np.array_equal(grun.dump(P.DUMP_COUNTS), orun.counts()), where
        assert np.array_equal(grun.dump(P.DUMP_OFFSETS), orun.offsets()), where
    compare_obs(grun.observables(), orun.observables(), where)


def run_lockstep(P, steps: int, use_graph=False, every=1, stream_chunks=0, **kw):
    """stream_chunks > 0 steps the engine by pa_step_stream with that many
    ranges and checks the host copy of every step against pa_dump."""
    ocfg, gcfg = configs(P, **kw)
    orun = O.Run(ocfg)
    grun = P.Run(gcfg)
    host = copy_stream = None
    if stream_chunks:
        import torch
        st = grun.state()
        host = torch.zeros(st["capacity"] * st["stride"], dtype=torch.uint8, pin_memory=True)
        copy_stream = torch.cuda.Stream()
    try:
        assert np.array_equal(grun.dump(P.DUMP_COUPLINGS), orun.couplings())
        compare_state(P, grun, orun, 0)
        for i in range(1, steps + 1):
            assert orun.step() == 0
            if use_graph:
                grun.run_steps(1)
            elif stream_chunks:
                R = grun.step_stream(host, stream_chunks, copy_stream)
                assert R == orun.R
                grun.observables()  # waits for the copies
                stride = grun.state()["stride"]
                raw = grun.dump(P.DUMP_SPINS_RAW).reshape(-1)
                assert np.array_equal(host.numpy()[: R * stride], raw[: R * stride]), i
            else:
                grun.step()
            if i % every == 0 or i == steps:
                compare_state(P, grun, orun, i)
        hist = grun.history(0, steps + 1)
        for i, h in enumerate(hist):
            assert h["step"] == i
        compare_obs(hist[-1], orun.observables(), "history")
    finally:
        grun.close()
        orun.close()
