"""Checkpoint / resume: a run restored from a checkpoint continues bit for
bit like the run that wrote it (spins, levels, histograms, counts, offsets,
observables history), for the packed and int8 layouts and a +-J instance;
a checkpoint is refused by a run with another configuration."""
from __future__ import annotations

import numpy as np
import pytest

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
