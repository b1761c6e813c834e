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


def test_ferromagnet_3d(P):
    run_lockstep(P, steps=5, dim=3, L=8, model=0, layout=1, R0=700, K=10, theta=3,
                 beta_max=0.6, seed=12)


@pytest.mark.parametrize("L,layout", [(16, 1), (64, 1), (16, 0), (128, 1)])
def test_heating_from_the_ground_state(P, L, layout):
    """Heating (Sec. 2): ground-state start at beta0 = 2, beta decreasing."""
    run_lockstep(P, steps=8, dim=2, L=L, layout=layout, R0=1500 if L < 128 else 80, K=40,
                 theta=2, beta0=2.0, beta_max=0.0, init=1, seed=60 + L)


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
