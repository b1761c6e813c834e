"""Parity of the CUDA path with the CPU oracle (element by element, same seeds).

Bit-exact: spins, energy levels, magnetisations, histograms, tau tables
(n, F), the normaliser S, copy counts, offsets (replica order) and every
integer observable.  FP64 observables within 1e-12 relative (only ln() may
differ in its last ulp).  Sizes span several resample tiles and a ragged
last tile; edge cases cover R0 = 1, theta = 0, a zero temperature step,
capacity overflow, running past step K, and CUDA-graph replay.
"""
from __future__ import annotations

import numpy as np
import pytest

from lockstep import configs, run_lockstep
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


def test_config1_int8_L16_first_steps(P):
    """2D L = 16, int8 spins, R0 = 1000, beta 0 -> 1 in 100 steps, theta = 10."""
    run_lockstep(P, steps=25, dim=2, L=16, layout=0, R0=1000, K=100, theta=10, seed=1)


@pytest.mark.slow
def test_config1_int8_L16_full_run(P):
    run_lockstep(P, steps=100, every=5, dim=2, L=16, layout=0, R0=1000, K=100, theta=10, seed=1)


def test_config1_packed_layout_gives_the_same_run(P):
    run_lockstep(P, steps=20, dim=2, L=16, layout=1, R0=1000, K=100, theta=10, seed=1)


@pytest.mark.parametrize("L", [4, 8, 32, 64, 128])
def test_packed_2d_sizes(P, L):
    R0 = {4: 3000, 8: 2500, 32: 700, 64: 300, 128: 64}[L]
    run_lockstep(P, steps=6, dim=2, L=L, layout=1, R0=R0, K=12, theta=3, beta_max=1.2,
                 seed=100 + L, instance_id=L)


@pytest.mark.parametrize("theta,model", [(1, 0), (26, 0), (27, 0), (30, 1)])
def test_l64_sweep_counts_around_the_step_table_limit(P, theta, model):
    """The L = 64 register kernel reads the round-3 Philox products from a
    table formed per launch for up to 26 sweeps and forms them itself beyond:
    both forms, ferromagnet and +-J, follow the oracle bit for bit."""
    extra = dict(coupling_seed=9, instance_id=4) if model else {}
    run_lockstep(P, steps=2, dim=2, L=64, layout=1, model=model, R0=96, K=4, theta=theta,
                 beta_max=1.0, seed=300 + theta, **extra)


@pytest.mark.parametrize("L", [4, 8, 64])
def test_int8_2d_sizes(P, L):
    run_lockstep(P, steps=5, dim=2, L=L, layout=0, R0=600, K=10, theta=2, beta_max=1.0,
                 seed=200 + L)


@pytest.mark.parametrize("L,layout", [(2, 1), (4, 1), (6, 1), (8, 1), (10, 1), (12, 1), (16, 1),
                                      (2, 0), (6, 0), (10, 0)])
def test_ea_3d_sizes(P, L, layout):
    R0 = {2: 3000, 4: 2100, 6: 900, 8: 500, 10: 300, 12: 150, 16: 64}[L]
    run_lockstep(P, steps=5, dim=3, L=L, model=1, layout=layout, R0=R0, K=10, theta=3,
                 beta_max=3.0, seed=300 + L, coupling_seed=77 + L, instance_id=5)


def test_ea_2d_pm_j(P):
    run_lockstep(P, steps=6, dim=2, L=16, model=1, layout=1, R0=900, K=12, theta=4,
                 beta_max=2.0, seed=9, coupling_seed=10)


@pytest.mark.parametrize("L,R0", [(64, 400), (128, 70)])
def test_ea_2d_pm_j_register_kernels(P, L, R0):
    """2D +-J at L = 64 and 128 through the register-resident kernels."""
    run_lockstep(P, steps=6, dim=2, L=L, model=1, layout=1, R0=R0, K=12, theta=3,
                 beta_max=2.0, seed=90 + L, coupling_seed=91 + L, instance_id=L)


def test_ferromagnet_3d(P):
    run_lockstep(P, steps=5, dim=3, L=8, model=0, layout=1, R0=700, K=10, theta=3,
                 beta_max=0.6, seed=12)


@pytest.mark.parametrize("L,layout", [(16, 1), (64, 1), (16, 0), (128, 1)])
def test_heating_from_the_ground_state(P, L, layout):
    """Heating (Sec. 2): ground-state start at beta0 = 2, beta decreasing."""
    run_lockstep(P, steps=8, dim=2, L=L, layout=layout, R0=1500 if L < 128 else 80, K=40,
                 theta=2, beta0=2.0, beta_max=0.0, init=1, seed=60 + L)


@pytest.mark.parametrize("L,layout,beta0,beta_end", [(16, 1, 0.0, 1.0), (64, 1, 0.0, 1.0),
                                                     (16, 0, 0.0, 1.0), (16, 1, 2.0, 0.0)])
def test_adaptive_schedule(P, L, layout, beta0, beta_end):
    """Adaptive temperature steps: the engine picks the same next beta as the
    oracle (bit for bit) and the resample / sweep at it match."""
    init = 1 if beta0 > beta_end else 0
    from lockstep import compare_state
    ocfg, gcfg = configs(P, dim=2, L=L, layout=layout, R0=1200, K=40, theta=2, beta0=beta0,
                         beta_max=beta_end, seed=70 + L, init=init)
    orun, grun = O.Run(ocfg), P.Run(gcfg)
    for i in range(1, 9):
        H = orun.hist()
        b_o = O.adaptive_next(H, orun.R, orun.beta, beta_end, 0.8)
        b_g = grun.adaptive_beta(0.8, beta_end)
        assert b_g == b_o, (i, b_g, b_o)
        assert orun.resample_to(b_o) == 0 and orun.sweep(2) == 0
        grun.resample_to(b_g)
        grun.sweep(2)
        compare_state(P, grun, orun, i)
        assert grun.observables()["beta"] == b_o
    # back on the fixed schedule: the next step's dbeta starts from the adaptive
    # beta (and may change sign), the one after is the schedule's own
    for i in range(9, 12):
        assert orun.step() == 0
        grun.step()
        compare_state(P, grun, orun, i)
    # and adaptive again, once more, through a CUDA graph in between
    b_o = O.adaptive_next(orun.hist(), orun.R, orun.beta, beta_end, 0.9)
    assert grun.adaptive_beta(0.9, beta_end) == b_o
    assert orun.resample_to(b_o) == 0 and orun.sweep(2) == 0
    grun.resample_to(b_o)
    grun.sweep(2)
    compare_state(P, grun, orun, 12)
    for i in range(13, 15):
        assert orun.step() == 0
    grun.run_steps(2)
    compare_state(P, grun, orun, 14)
    grun.close()
    orun.close()


def test_adaptive_step_reaches_the_end_and_stops(P):
    """A run driven by adaptive steps reaches beta_end exactly; past K it reports
    PA_ERR_DONE; an invalid target beta is rejected."""
    _, gcfg = configs(P, dim=2, L=8, layout=1, R0=2000, K=30, theta=2, beta_max=0.3, seed=88)
    run = P.Run(gcfg)
    with pytest.raises(P.PaError) as e:
        run.resample_to(-0.5)
    assert e.value.code == -1
    n = 0
    while run.observables()["beta"] < 0.3:
        run.resample_to(run.adaptive_beta(0.5, 0.3))
        run.sweep(2)
        n += 1
        assert n <= 30
    assert run.observables()["beta"] == 0.3
    while run.state()["step"] < 30:
        run.resample_to(0.3)
    with pytest.raises(P.PaError) as e:
        run.resample_to(0.3)
    assert e.value.code == -8
    run.close()


@pytest.mark.parametrize("spec", [
    dict(dim=2, L=16, layout=1, R0=1000, K=100, theta=10, seed=21),
    dict(dim=2, L=16, layout=0, R0=1000, K=100, theta=10, seed=22),
    dict(dim=2, L=64, layout=1, R0=2300, K=20, theta=2, seed=23),
    dict(dim=2, L=8, layout=1, R0=5001, K=16, theta=2, beta_max=1.5, seed=24),
    dict(dim=3, L=8, model=1, layout=1, R0=900, K=10, theta=3, beta_max=3.0, seed=25,
         coupling_seed=26, instance_id=3),
    dict(dim=2, L=16, layout=1, R0=1500, K=40, theta=2, beta0=2.0, beta_max=0.0, init=1,
         seed=27),
], ids=["2d_L16_packed", "2d_L16_int8", "2d_L64", "ragged_tiles", "3d_L8_pmj", "heating"])
def test_poisson_resampling(P, spec):
    """The Poisson draw of Sec. 2: copy counts, offsets and the population
    (whose size now fluctuates as Poisson(R0)) bit for bit with the oracle."""
    run_lockstep(P, steps=8, resample=1, **spec)


@pytest.mark.parametrize("spec", [
    dict(dim=2, L=16, layout=1, R0=1000, K=100, theta=10, seed=121),
    dict(dim=2, L=16, layout=0, R0=1000, K=100, theta=10, seed=122),
    dict(dim=2, L=64, layout=1, R0=2300, K=20, theta=2, seed=123),
    dict(dim=2, L=8, layout=1, R0=5001, K=16, theta=2, beta_max=1.5, seed=124),
    dict(dim=3, L=8, model=1, layout=1, R0=900, K=10, theta=3, beta_max=3.0, seed=125,
         coupling_seed=126, instance_id=3),
    dict(dim=2, L=16, layout=1, R0=1500, K=40, theta=2, beta0=2.0, beta_max=0.0, init=1,
         seed=127),
    dict(dim=2, L=16, layout=1, R0=1, K=6, theta=2, beta_max=0.5, seed=128),
], ids=["2d_L16_packed", "2d_L16_int8", "2d_L64", "ragged_tiles", "3d_L8_pmj", "heating",
        "single_replica"])
def test_multinomial_resampling(P, spec):
    """Multinomial resampling: R0 draws by exact fixed-point cumulative weights;
    copy counts, offsets, population (exactly R0) bit for bit with the oracle."""
    run_lockstep(P, steps=8 if spec["K"] >= 8 else spec["K"], resample=2, **spec)


def test_multinomial_graph_replay(P):
    run_lockstep(P, steps=6, use_graph=True, resample=2, dim=2, L=64, layout=1, R0=3000, K=20,
                 theta=2, beta_max=1.0, seed=129)


def test_poisson_resampling_graph_replay(P):
    run_lockstep(P, steps=8, use_graph=True, resample=1, dim=2, L=64, layout=1, R0=3000, K=20,
                 theta=2, beta_max=1.0, seed=28)


def test_poisson_capacity_overflow_is_reported(P):
    ocfg, gcfg = configs(P, dim=2, L=8, R0=200, capacity=200, K=50, theta=1, beta_max=3.0,
                         seed=1, resample=1)
    orun, grun = O.Run(ocfg), P.Run(gcfg)
    code = 0
    for _ in range(50):
        orc = orun.step()
        grun.step()
        code = grun.status()
        if orc:
            assert orc == -3
            break
    assert code == -4  # PA_ERR_CAPACITY
    grun.close()


def test_several_tiles_with_ragged_tail(P):
    """R0 = 5001: three resample tiles, the last one nearly empty."""
    run_lockstep(P, steps=8, dim=2, L=8, layout=1, R0=5001, K=16, theta=2, beta_max=1.5, seed=13)


def test_single_replica(P):
    run_lockstep(P, steps=6, dim=2, L=16, layout=1, R0=1, K=6, theta=2, beta_max=0.3, seed=14)


def test_theta_zero(P):
    run_lockstep(P, steps=6, dim=2, L=16, layout=1, R0=800, K=6, theta=0, beta_max=1.0, seed=15)


def test_zero_temperature_step_is_identity(P):
    ocfg, gcfg = configs(P, dim=2, L=16, R0=500, K=4, theta=0, beta0=0.4, beta_max=0.4, seed=16)
    run = P.Run(gcfg)
    s0 = run.spins()
    for _ in range(4):
        run.step()
        assert (run.dump(P.DUMP_COUNTS) == 1).all()
        assert np.array_equal(run.dump(P.DUMP_OFFSETS), np.arange(500, dtype=np.uint32))
        assert np.array_equal(run.spins(), s0)
    run.close()


def test_graph_replay_equals_plain_steps(P):
    run_lockstep(P, steps=10, use_graph=True, dim=2, L=64, layout=1, R0=2300, K=20, theta=2,
                 beta_max=1.0, seed=17)


@pytest.mark.parametrize("spec,chunks", [
    (dict(dim=2, L=64, layout=1, R0=2300, K=20, theta=2, seed=17), 7),           # L = 64 kernel
    (dict(dim=2, L=128, layout=1, R0=150, K=8, theta=2, seed=18), 3),            # L = 128 kernel
    (dict(dim=2, L=16, layout=1, R0=1000, K=12, theta=3, seed=19), 5),           # replica-sliced
    (dict(dim=3, L=10, model=1, layout=1, R0=300, K=8, theta=2, beta_max=3.0, seed=20,
          coupling_seed=21), 4),                                                  # replica-sliced, 3D +-J
    (dict(dim=2, L=16, layout=0, R0=700, K=10, theta=2, seed=22), 64),           # int8, ranges < 32
    (dict(dim=2, L=8, layout=1, R0=40, K=6, theta=2, seed=23), 1),
    (dict(dim=2, L=64, layout=1, R0=900, K=10, theta=2, seed=24, resample=1), 5),  # Poisson
    (dict(dim=3, L=8, model=1, layout=1, R0=700, K=8, theta=2, beta_max=3.0, seed=25,
          coupling_seed=26, resample=2), 3),                                      # multinomial
])
def test_streamed_step_equals_the_oracle(P, spec, chunks):
    """pa_step_stream: the sweeps of a step in slot ranges with the copy of
    each range to host memory on a second stream.  Same run as pa_step (and the
    oracle), and the host copy equals the device population."""
    run_lockstep(P, steps=min(spec["K"], 6), stream_chunks=chunks, beta_max=spec.pop("beta_max", 1.0),
                 **spec)


def test_streamed_step_rejects_bad_arguments(P):
    import torch
    _, gcfg = configs(P, dim=2, L=16, R0=100, K=4)
    run = P.Run(gcfg)
    st = run.state()
    host = torch.zeros(st["capacity"] * st["stride"], dtype=torch.uint8, pin_memory=True)
    cs = torch.cuda.Stream()
    for chunks in (0, 65):
        with pytest.raises(P.PaError) as e:
            run.step_stream(host, chunks, cs)
        assert e.value.code == -1
    with pytest.raises(P.PaError) as e:  # too small for the capacity
        P.pa_step_stream(run.h, host.data_ptr(), host.numel() - 1, 2, cs.cuda_stream)
    assert e.value.code == -1
    with pytest.raises(P.PaError) as e:  # the run's own stream
        P.pa_step_stream(run.h, host.data_ptr(), host.numel(), 2, run.stream.cuda_stream)
    assert e.value.code == -1
    assert run.state()["step"] == 0  # nothing was enqueued
    run.close()


def test_streamed_step_reports_capacity_overflow(P):
    import torch
    _, gcfg = configs(P, dim=2, L=8, R0=200, capacity=200, K=50, theta=1, beta_max=3.0, seed=1)
    run = P.Run(gcfg)
    st = run.state()
    host = torch.zeros(st["capacity"] * st["stride"], dtype=torch.uint8, pin_memory=True)
    cs = torch.cuda.Stream()
    with pytest.raises(P.PaError) as e:
        for _ in range(50):
            run.step_stream(host, 4, cs)
    assert e.value.code == -4  # PA_ERR_CAPACITY
    run.close()


def test_philox_ceiling_kernel_draws_the_sweep_blocks(P):
    """pa_bench_philox (the generator alone, in the L = 64 kernel's launch
    shape): each thread's xor word equals the xor of the oracle's Philox
    blocks (2g, b, SWEEP << 28, warp) over its half-sweeps and its 16 blocks."""
    import torch
    n = P.pa_bench_philox_threads()
    assert n > 0 and n % 512 == 0
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    seed = 0x0123456789ABCDEF
    P.pa_bench_philox(seed, 3, out.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy().view(np.uint32)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for t in (0, 1, 31, 32, 513, n - 1):
        want = 0
        for g in range(3):
            for b in range(16 * (t % 32), 16 * (t % 32) + 16):
                w = O.philox((2 * g, b, 2 << 28, t // 32), key)
                want ^= int(w[0]) ^ int(w[1]) ^ int(w[2]) ^ int(w[3])
        assert int(got[t]) == want, t
    with pytest.raises(P.PaError):
        P.pa_bench_philox(seed, 3, out.data_ptr(), n - 1, 0)


def test_lookback_timeout_is_reported_and_the_context_survives(P):
    """The resample's only wait (tile t waits for tile t - 1's prefix) is
    bounded.  With tile 0's prefix withheld (test hook), tile 1's wait runs out
    after its poll limit: the step finishes, the sticky PA_ERR_TIMEOUT is
    reported, and the context keeps working (a fresh run matches the oracle)."""
    import time
    _, gcfg = configs(P, dim=2, L=16, R0=5000, K=4, theta=1, seed=3)  # 3 resample tiles
    run = P.Run(gcfg)
    run.step()
    assert run.status() == 0
    with pytest.raises(P.PaError):
        P.pa_debug(run.h, 2)  # unknown bit
    P.pa_debug(run.h, P.DEBUG_WITHHOLD_PREFIX)
    t0 = time.perf_counter()
    run.step()
    assert run.status() == -5  # PA_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    run.close()
    run_lockstep(P, steps=2, dim=2, L=16, R0=5000, K=4, theta=1, seed=3)


def test_capacity_overflow_is_reported(P):
    ocfg, gcfg = configs(P, dim=2, L=8, R0=200, capacity=200, K=50, theta=1, beta_max=3.0,
                         seed=1)
    orun, grun = O.Run(ocfg), P.Run(gcfg)
    code = 0
    for _ in range(50):
        orc = orun.step()
        grun.step()
        code = grun.status()
        if orc:
            assert orc == -3
            break
    assert code == -4  # PA_ERR_CAPACITY
    assert grun.state()["R"] <= 200
    grun.close()


def test_stepping_past_K_is_reported(P):
    _, gcfg = configs(P, dim=2, L=8, R0=100, K=2, theta=1)
    run = P.Run(gcfg)
    run.step()
    run.step()
    assert run.status() == 0
    run.step()
    assert run.status() == -8  # PA_ERR_DONE
    assert run.state()["step"] == 2
    run.close()


def test_workspace_too_small_is_rejected(P):
    import torch
    _, gcfg = configs(P, dim=2, L=16, R0=100, K=2)
    n = P.pa_workspace_size(gcfg)
    ws = torch.empty(n - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PaError) as e:
        P.pa_init(gcfg, ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -7
    ws = torch.empty(n + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PaError) as e:
        P.pa_init(gcfg, ws.data_ptr() + 16, n, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -7


def test_run_cli_prints_observables(P):
    """python -m paper_2006_00561_gb300.run: one small run, one JSON line equal
    to the oracle's observables."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    proc = subprocess.run([sys.executable, "-m", "paper_2006_00561_gb300.run", "--dim", "3", "--L",
                           "6", "--model", "pmj", "--R0", "500", "--K", "6", "--theta", "2",
                           "--beta-max", "2", "--seed", "31", "--coupling-seed", "32"],
                          cwd=root, capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-1500:]
    got = json.loads(proc.stdout.strip().splitlines()[-1])
    orun = O.Run(O.make_config(dim=3, L=6, model=1, R0=500, K=6, theta=2, beta_max=2.0, seed=31,
                               coupling_seed=32))
    for _ in range(6):
        assert orun.step() == 0
    want = orun.observables()
    for k in ("step", "R", "sumE", "sumE2", "sumAbsM", "sumM2"):
        assert got[k] == want[k], k
    assert abs(got["lnZ"] - want["lnZ"]) <= 1e-12 * abs(want["lnZ"])
    assert got["ms_per_step"] > 0
