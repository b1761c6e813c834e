"""Checkpoint / resume: a run restored from a checkpoint continues bit for
bit like the run that wrote it (spins, levels, histograms, counts, offsets,
observables history), for the packed and int8 layouts and a +-J instance;
a checkpoint is refused by a run with another configuration.

The step recursion of Sec. 2 makes a run at a step boundary a pure function
of its state, so a restored run must also follow the CPU oracle's
uninterrupted run of the same configuration: those tests compare the CUDA
path only with the oracle, at every step after the restore."""
from __future__ import annotations

import numpy as np
import pytest
from lockstep import compare_obs, compare_state, configs

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


SPECS = [
    dict(dim=2, L=64, layout=1, R0=3000, K=20, theta=3, beta_max=1.0, seed=41),
    dict(dim=2, L=16, layout=0, R0=2500, K=20, theta=3, beta_max=1.0, seed=42),
    dict(dim=3, L=8, layout=1, model=1, R0=1800, K=20, theta=3, beta_max=3.0, seed=43,
         coupling_seed=44, instance_id=9),
]


@pytest.mark.parametrize("spec", SPECS, ids=["2d_L64_packed", "2d_L16_int8", "3d_L8_pmj"])
def test_restored_run_continues_identically(P, spec):
    a = P.Run(P.make_config(**spec))
    for _ in range(7):
        a.step()
    blob = a.checkpoint()
    a.run_steps(3)
    a.step()
    b = P.Run(P.make_config(**spec))
    b.step()  # some unrelated progress that the restore must replace
    b.restore(blob)
    assert b.state()["step"] == 7
    b.step()
    b.run_steps(3)
    sa, sb = a.state(), b.state()
    for k in ("step", "R", "R_prev", "kref", "sweeps_done", "S", "lnZ", "lnQ", "status_bits"):
        assert sa[k] == sb[k], k
    for what in (P.DUMP_SPINS_RAW, P.DUMP_EBIN, P.DUMP_MAG, P.DUMP_HIST, P.DUMP_COUNTS,
                 P.DUMP_OFFSETS, P.DUMP_TAB_N, P.DUMP_TAB_F):
        assert np.array_equal(a.dump(what), b.dump(what)), what
    assert a.history(0, 12) == b.history(0, 12)
    a.close()
    b.close()


def test_checkpoint_refused_by_another_configuration(P):
    a = P.Run(P.make_config(**SPECS[0]))
    a.step()
    blob = a.checkpoint()
    other = P.Run(P.make_config(**dict(SPECS[0], seed=999)))
    with pytest.raises(P.PaError) as e:
        other.restore(blob)
    assert e.value.code == -1
    bad = bytearray(blob)
    bad[0] ^= 0xFF
    with pytest.raises(P.PaError):
        a.restore(bytes(bad))
    with pytest.raises(P.PaError):
        a.restore(blob[:100])


def test_restored_adaptive_run_continues_identically(P):
    """A run on adaptive temperature steps resumes at its own beta: the step
    after the restore takes its temperature step from there."""
    spec = dict(dim=2, L=16, layout=1, R0=2000, K=30, theta=2, beta_max=1.0, seed=45)
    a = P.Run(P.make_config(**spec))
    for _ in range(4):
        a.resample_to(a.adaptive_beta(0.7, 1.0))
        a.sweep(2)
    blob = a.checkpoint()
    a.step()
    a.resample_to(a.adaptive_beta(0.7, 1.0))
    a.sweep(2)
    b = P.Run(P.make_config(**spec))
    for _ in range(6):
        b.resample_to(b.adaptive_beta(0.5, 1.0))  # another trajectory, to be replaced
        b.sweep(2)
    b.restore(blob)
    assert b.observables()["beta"] == a.history(4, 1)[0]["beta"]
    b.step()
    b.resample_to(b.adaptive_beta(0.7, 1.0))
    b.sweep(2)
    for what in (P.DUMP_SPINS_RAW, P.DUMP_HIST, P.DUMP_COUNTS, P.DUMP_OFFSETS):
        assert np.array_equal(a.dump(what), b.dump(what)), what
    assert a.history(0, 7) == b.history(0, 7)
    a.close()
    b.close()


def _compare_restored(P, grun, orun, step):
    """State right after a restore: the population, its levels, magnetisations,
    histogram and observables (the counts and offsets of the last resample are
    not part of a checkpoint)."""
    st = grun.state()
    assert st["status_bits"] == 0
    assert st["step"] == orun.step_index == step
    assert st["R"] == orun.R
    assert np.array_equal(grun.spins(), orun.spins())
    assert np.array_equal(grun.dump(P.DUMP_EBIN), orun.ebin())
    assert np.array_equal(grun.dump(P.DUMP_MAG), orun.mag())
    assert np.array_equal(grun.dump(P.DUMP_HIST), orun.hist())
    compare_obs(grun.observables(), orun.observables(), f"restored at step {step}")


@pytest.mark.parametrize("spec", SPECS, ids=["2d_L64_packed", "2d_L16_int8", "3d_L8_pmj"])
def test_restored_run_follows_the_oracle(P, spec):
    """The oracle runs uninterrupted for K steps.  The CUDA run is checkpointed
    at step 7 and thrown away; a fresh run makes unrelated progress, restores
    the checkpoint and continues by single steps and graph-replayed steps.  At
    every step after the restore its whole state equals the oracle's."""
    ocfg, gcfg = configs(P, **spec)
    orun = O.Run(ocfg)
    a = P.Run(gcfg)
    for _ in range(7):
        assert orun.step() == 0
        a.step()
    compare_state(P, a, orun, 7)
    blob = a.checkpoint()
    a.close()
    b = P.Run(gcfg)
    b.step()
    b.step()  # unrelated progress that the restore must replace
    b.restore(blob)
    _compare_restored(P, b, orun, 7)
    for i in range(8, spec["K"] + 1):
        assert orun.step() == 0
        if i % 3 == 0:
            b.run_steps(1)
        else:
            b.step()
        compare_state(P, b, orun, i)
    hist = b.history(0, spec["K"] + 1)
    compare_obs(hist[-1], orun.observables(), "history")
    b.close()
    orun.close()


def test_restored_adaptive_run_follows_the_oracle(P):
    """Adaptive temperature steps across a checkpoint: four adaptive steps, a
    checkpoint, a restore into a fresh run, then a scheduled step and more
    adaptive steps; the oracle takes the same decisions uninterrupted, and the
    restored run equals it (beta bit for bit) at every step."""
    spec = dict(dim=2, L=16, layout=1, R0=2000, K=30, theta=2, beta_max=1.0, seed=45)
    ocfg, gcfg = configs(P, **spec)
    orun = O.Run(ocfg)
    a = P.Run(gcfg)
    for i in range(1, 5):
        b_o = O.adaptive_next(orun.hist(), orun.R, orun.beta, 1.0, 0.7)
        assert a.adaptive_beta(0.7, 1.0) == b_o
        assert orun.resample_to(b_o) == 0 and orun.sweep(2) == 0
        a.resample_to(b_o)
        a.sweep(2)
        compare_state(P, a, orun, i)
    blob = a.checkpoint()
    a.close()
    b = P.Run(gcfg)
    for _ in range(3):
        b.resample_to(b.adaptive_beta(0.5, 1.0))  # another trajectory, to be replaced
        b.sweep(2)
    b.restore(blob)
    _compare_restored(P, b, orun, 4)
    assert b.observables()["beta"] == orun.beta
    assert orun.step() == 0
    b.step()
    compare_state(P, b, orun, 5)
    for i in range(6, 9):
        b_o = O.adaptive_next(orun.hist(), orun.R, orun.beta, 1.0, 0.7)
        assert b.adaptive_beta(0.7, 1.0) == b_o
        assert orun.resample_to(b_o) == 0 and orun.sweep(2) == 0
        b.resample_to(b_o)
        b.sweep(2)
        compare_state(P, b, orun, i)
    b.close()
    orun.close()
