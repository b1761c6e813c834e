"""End-to-end pins of the oracle's whole PA run against exact thermodynamics.

Population annealing estimates ln Z(beta_i) = N ln 2 + sum_l ln Q_l (Eq. 3,
Eq. 5 read as -beta F) and population averages (Sec. 2).  Over M independent
seeds the mean estimate must sit within the 3-standard-error level (Student-t
bound for the estimated standard error) of:
  * Kaufman's exact ln Z of the 16 x 16 torus (the paper's model, Eq. 6, at the
    config-1 workload: R0 = 1000, beta 0 -> 1 in 100 steps, theta = 10),
  * brute-force ln Z of the 4 x 4 torus and of a 2 x 2 x 2 +-J instance.
The runs also check the invariants the oracle tracks: energies recomputed from
scratch equal the tracked ones and sum_k H_k = R after every step, and the
population stays within a few sqrt(R0) of R0.
"""
from __future__ import annotations

import multiprocessing as mpc
import os

import numpy as np
import pytest

import exact

CHECK_STEPS_L16 = (20, 44, 60, 100)


def _run_seed(args):
    kind, seed = args
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import oracle as O
    if kind == "L16":
        cfg = O.make_config(dim=2, L=16, R0=1000, K=100, theta=10, seed=seed)
        checks = CHECK_STEPS_L16
    elif kind == "L4":
        cfg = O.make_config(dim=2, L=4, R0=3000, K=40, theta=4, beta_max=1.2, seed=seed)
        checks = (10, 20, 40)
    elif kind == "L4_poisson":
        cfg = O.make_config(dim=2, L=4, R0=3000, K=40, theta=4, beta_max=1.2, seed=seed,
                            resample=O.RESAMPLE_POISSON)
        checks = (10, 20, 40)
    elif kind == "L4_multinomial":
        cfg = O.make_config(dim=2, L=4, R0=3000, K=40, theta=4, beta_max=1.2, seed=seed,
                            resample=O.RESAMPLE_MULTINOMIAL)
        checks = (10, 20, 40)
    elif kind == "L16_multinomial":
        cfg = O.make_config(dim=2, L=16, R0=1000, K=100, theta=10, seed=seed,
                            resample=O.RESAMPLE_MULTINOMIAL)
        checks = CHECK_STEPS_L16
    elif kind == "L16_poisson":
        cfg = O.make_config(dim=2, L=16, R0=1000, K=100, theta=10, seed=seed,
                            resample=O.RESAMPLE_POISSON)
        checks = CHECK_STEPS_L16
    elif kind == "L4_heat":
        cfg = O.make_config(dim=2, L=4, R0=3000, K=40, theta=4, beta0=2.0, beta_max=0.0,
                            init=O.INIT_GROUND, seed=seed)
        checks = (10, 20, 30, 40)
    elif kind == "L8_heat":
        cfg = O.make_config(dim=2, L=8, R0=4000, K=100, theta=10, beta0=2.0, beta_max=0.0,
                            init=O.INIT_GROUND, seed=seed)
        checks = (40, 70, 100)
    else:
        cfg = O.make_config(dim=3, L=2, model=O.MODEL_PMJ, R0=3000, K=40, theta=4,
                            beta_max=2.0, seed=seed, coupling_seed=6)
        checks = (10, 20, 40)
    if kind == "L16_adaptive":
        cfg = O.make_config(dim=2, L=16, R0=1000, K=400, theta=10, seed=seed)
        run = O.Run(cfg)
        betas = [0.0]
        while run.beta < 1.0:
            b = O.adaptive_next(run.hist(), run.R, run.beta, 1.0, 0.85)
            assert b > run.beta
            assert run.resample_to(b) == 0
            assert run.sweep(cfg.theta) == 0
            betas.append(run.beta)
        o = run.observables()
        return {"betas": betas, "lnZ": o["lnZ"], "e": o["sumE"] / o["R"]}, run.check_failures, []
    run = O.Run(cfg)
    out, Rs = {}, []
    for i in range(1, cfg.K + 1):
        assert run.step() == 0
        o = run.observables()
        Rs.append(o["R"])
        if i in checks:
            out[i] = (o["beta"], o["lnZ"], o["sumE"] / o["R"], o["cv"], o["m_abs"], o["chi"])
    return out, run.check_failures, Rs


_RUNS_CACHE: dict = {}


def _runs(kind, seeds):
    """Whole oracle runs of one kind, one per seed, in spawned processes; the
    results are kept for the other tests of this module that read the same
    runs."""
    key = (kind, tuple(seeds))
    if key not in _RUNS_CACHE:
        ctx = mpc.get_context("spawn")
        with ctx.Pool(min(len(seeds), os.cpu_count() or 1)) as pool:
            _RUNS_CACHE[key] = pool.map(_run_seed, [(kind, s) for s in seeds])
    return _RUNS_CACHE[key]


def _assert_within(vals, want, p_two_sided=0.0027):
    """The mean of M independent estimates within the bound of a two-sided
    test at the level of 3 normal standard errors: with the standard error
    estimated from the same M values, (mean - want) / se is Student-t with
    M - 1 degrees of freedom, whose quantile replaces the normal 3."""
    from scipy.stats import t as student_t
    vals = np.asarray(vals, dtype=np.float64)
    se = vals.std(ddof=1) / np.sqrt(vals.size)
    nsig = float(student_t.ppf(1.0 - p_two_sided / 2.0, vals.size - 1))
    assert abs(vals.mean() - want) < nsig * se + 1e-12 * abs(want), (vals.mean(), want, se, nsig)


@pytest.mark.slow
def test_pa_lnZ_and_energy_match_kaufman_L16():
    res = _runs("L16", list(range(100, 120)))
    R0 = 1000
    for out, fails, Rs in res:
        assert fails == 0
        assert max(abs(r - R0) for r in Rs) <= 2.5 * np.sqrt(R0)
    for i in CHECK_STEPS_L16:
        beta = res[0][0][i][0]
        _assert_within([r[0][i][1] for r in res], float(exact.kaufman_lnZ(16, beta)))
        _assert_within([r[0][i][2] / 256 for r in res], exact.kaufman_energy_per_site(16, beta))


@pytest.mark.slow
def test_pa_specific_heat_matches_kaufman_L16():
    """C_v per site of the config-1 population (R0 = 1000, 100 steps, theta =
    10) at beta = 0.2, 0.44 (near the L = 16 peak) and 0.6 within 3 SE of
    beta^2 d^2 ln Z / d beta^2 / N through Kaufman's closed form, over the same
    20 runs as the ln Z pin."""
    res = _runs("L16", list(range(100, 120)))
    for i in (20, 44, 60):
        beta = res[0][0][i][0]
        _assert_within([r[0][i][3] for r in res], exact.kaufman_cv_per_site(16, beta))


def _pa_vs_dos(kind, dos, pop_sigmas=2.5):
    res = _runs(kind, list(range(40, 56)))
    for out, fails, Rs in res:
        assert fails == 0
        assert max(abs(r - 3000) for r in Rs) <= pop_sigmas * np.sqrt(3000)
    for i in res[0][0]:
        beta = res[0][0][i][0]
        if beta == 0.0:
            _assert_within([r[0][i][1] for r in res], 16 * np.log(2.0))
            continue
        _assert_within([r[0][i][1] for r in res], float(exact.lnZ_from_dos(dos, beta)))
        _assert_within([r[0][i][2] for r in res], exact.mean_energy_from_dos(dos, beta))


@pytest.mark.slow
def test_pa_lnZ_matches_bruteforce_2d_L4():
    from oracle import oracle as O
    J = np.ones(32, dtype=np.int8)
    dos = exact.density_of_states(2 * O.energy(2, 4, J, s)[0] - 32 for s in exact.all_states(16))
    _pa_vs_dos("L4", dos)


@pytest.mark.slow
def test_pa_observables_match_bruteforce_2d_L4():
    """The population averages of Sec. 2 that the oracle reports -- specific
    heat C_v, mean absolute magnetisation <|m|> and susceptibility chi -- within
    3 SE of their exact Boltzmann values for the 4 x 4 torus at beta = 0.3, 0.6
    and 1.2.  The exact values come from enumerating all 2^16 states with their
    own energy and magnetisation (exact.joint_dos_2d_torus): C_v as
    beta^2 d^2 ln Z / d beta^2 / N, <M^2> as the second field derivative of
    ln Z, <|M|> as a direct Boltzmann sum; so a wrong formula for any of the
    three (a lost beta, <M>^2 in place of <|M|>^2, a root-mean-square in place
    of the mean of |M|) fails here, whatever the population.  The same runs
    (16 seeds, R0 = 3000) serve the ln Z pin above."""
    g = exact.joint_dos_2d_torus(4)
    res = _runs("L4", list(range(40, 56)))
    for i in res[0][0]:
        beta = res[0][0][i][0]
        want = exact.exact_observables(g, 16, beta)
        _assert_within([r[0][i][3] for r in res], want["cv"])
        _assert_within([r[0][i][4] for r in res], want["m_abs"])
        _assert_within([r[0][i][5] for r in res], want["chi"])


@pytest.mark.slow
def test_pa_poisson_resampling_matches_bruteforce_2d_L4():
    """Poisson resampling (the draw Sec. 2 prescribes): ln Z and <E> within 3 SE
    of brute force; the population is then Poisson(R0) at every step, so it
    stays within 5 sqrt(R0) of R0 over 16 x 40 steps."""
    from oracle import oracle as O
    J = np.ones(32, dtype=np.int8)
    dos = exact.density_of_states(2 * O.energy(2, 4, J, s)[0] - 32 for s in exact.all_states(16))
    _pa_vs_dos("L4_poisson", dos, pop_sigmas=5.0)


@pytest.mark.slow
def test_pa_poisson_resampling_matches_kaufman_L16():
    """The config-1 workload with Poisson resampling: ln Z and <E>/N within 3 SE
    of Kaufman at four temperatures; the population's spread across steps and
    seeds is that of Poisson(R0) (variance R0 within 20 %)."""
    res = _runs("L16_poisson", list(range(700, 716)))
    allR = np.concatenate([np.array(Rs, dtype=np.float64) for _, _, Rs in res])
    assert abs(allR.var() / 1000 - 1.0) < 0.2
    for out, fails, _ in res:
        assert fails == 0
    for i in CHECK_STEPS_L16:
        beta = res[0][0][i][0]
        _assert_within([r[0][i][1] for r in res], float(exact.kaufman_lnZ(16, beta)))
        _assert_within([r[0][i][2] / 256 for r in res], exact.kaufman_energy_per_site(16, beta))


@pytest.mark.slow
def test_pa_multinomial_resampling_matches_bruteforce_2d_L4():
    """Multinomial resampling: ln Z and <E> within 3 SE of brute force, and the
    population is exactly R0 after every step."""
    from oracle import oracle as O
    J = np.ones(32, dtype=np.int8)
    dos = exact.density_of_states(2 * O.energy(2, 4, J, s)[0] - 32 for s in exact.all_states(16))
    _pa_vs_dos("L4_multinomial", dos, pop_sigmas=0.0)


@pytest.mark.slow
def test_pa_multinomial_resampling_matches_kaufman_L16():
    res = _runs("L16_multinomial", list(range(800, 816)))
    for out, fails, Rs in res:
        assert fails == 0
        assert all(r == 1000 for r in Rs)
    for i in CHECK_STEPS_L16:
        beta = res[0][0][i][0]
        _assert_within([r[0][i][1] for r in res], float(exact.kaufman_lnZ(16, beta)))
        _assert_within([r[0][i][2] / 256 for r in res], exact.kaufman_energy_per_site(16, beta))


@pytest.mark.slow
def test_pa_heating_recovers_bruteforce_2d_L4():
    """Heating (Sec. 2) from the ground state at beta0 = 2 down to beta = 0: ln Z
    along the way matches brute force, and at beta = 0 it recovers N ln 2."""
    from oracle import oracle as O
    J = np.ones(32, dtype=np.int8)
    dos = exact.density_of_states(2 * O.energy(2, 4, J, s)[0] - 32 for s in exact.all_states(16))
    _pa_vs_dos("L4_heat", dos)


@pytest.mark.slow
def test_pa_heating_recovers_kaufman_L8():
    """Heating the 8 x 8 torus from its ground state at beta0 = 2 through the
    transition down to beta = 0 (R0 = 4000, 100 steps, theta = 10): ln Z within
    3 SE of Kaufman on the way and of the exact N ln 2 at the end.  (PA's
    finite-population bias shrinks like 1/R0 while the standard error shrinks
    like 1/sqrt(R0); R0 = 4000 keeps the bias well inside 3 SE.)"""
    res = _runs("L8_heat", list(range(300, 316)))
    for out, fails, Rs in res:
        assert fails == 0
    for i in (40, 70, 100):
        beta = res[0][0][i][0]
        want = 64 * np.log(2.0) if beta == 0.0 else float(exact.kaufman_lnZ(8, beta))
        _assert_within([r[0][i][1] for r in res], want)


@pytest.mark.slow
def test_pa_adaptive_schedule_matches_kaufman_L16():
    """Adaptive temperature steps (overlap target 0.85) from beta 0 to 1 on the
    16 x 16 torus: ln Z(1) and <E>/N within 3 SE of Kaufman; the steps shrink
    where the energy distribution narrows less than it shifts (near beta_c)."""
    res = _runs("L16_adaptive", list(range(500, 516)))
    for out, fails, _ in res:
        assert fails == 0
        b = np.array(out["betas"])
        assert b[-1] == 1.0 and (np.diff(b) > 0).all()
    _assert_within([r[0]["lnZ"] for r in res], float(exact.kaufman_lnZ(16, 1.0)))
    _assert_within([r[0]["e"] / 256 for r in res], exact.kaufman_energy_per_site(16, 1.0))
    steps = np.diff(res[0][0]["betas"])
    mids = 0.5 * (np.array(res[0][0]["betas"][1:]) + np.array(res[0][0]["betas"][:-1]))
    assert steps[(mids > 0.4) & (mids < 0.5)].mean() < steps[mids < 0.1].mean()


@pytest.mark.slow
def test_pa_lnZ_matches_bruteforce_3d_L2_pm_j():
    from oracle import oracle as O
    cfg = O.make_config(dim=3, L=2, model=O.MODEL_PMJ, coupling_seed=6)
    J = O.couplings(cfg)
    dos = exact.density_of_states(2 * O.energy(3, 2, J, s)[0] - 24 for s in exact.all_states(8))
    _pa_vs_dos("L2_3d", dos)
