"""Planted mistakes: each one is applied to a copy of oracle/pa_oracle.c on the
CPU, compiled, and the pins of test_oracle_pins.py / test_oracle_pa_statistics.py
/ test_redistribute.py are run against it.  Every plausible slip listed here must make a pin fail; a
mutant that passes means a hole in the pins."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "pa_oracle.c")

# (name, original text, planted mistake, pins to run)
MUTANTS = [
    ("philox_swapped_multipliers", "uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;",
     "uint64_t p0 = (uint64_t)M1 * (uint64_t)x0;", "philox"),
    ("philox_key_bumped_first", "    for (int round = 0; round < 10; ++round) {\n        uint64_t p0",
     "    for (int round = 0; round < 10; ++round) {\n        k0 += W0; k1 += W1;\n        uint64_t p0",
     "philox"),
    ("delta_e_sign", "return 2 * spins[s] * local;", "return -2 * spins[s] * local;",
     "delta_e or zero_temperature or boltzmann"),
    ("delta_e_drops_backward_bond", "        local += J[dn * dim + d] * spins[dn];\n", "",
     "delta_e"),
    ("delta_e_wrong_backward_coupling", "local += J[dn * dim + d] * spins[dn];",
     "local += J[s * dim + d] * spins[dn];", "delta_e or gauge or boltzmann"),
    ("energy_counts_satisfied_bonds", "if (J[s * dim + d] * spins[s] * spins[t] < 0) ++u;",
     "if (J[s * dim + d] * spins[s] * spins[t] > 0) ++u;", "kaufman or delta_e"),
    ("energy_wrong_coupling_index", "if (J[s * dim + d] * spins[s] * spins[t] < 0) ++u;",
     "if (J[t * dim + d] * spins[s] * spins[t] < 0) ++u;", "gauge or delta_e"),
    ("threshold_one_class_for_all", "accept = u < T[dE / 4 - 1];", "accept = u < T[0];",
     "boltzmann"),
    ("threshold_compare_reversed", "accept = u < T[dE / 4 - 1];",
     "accept = u >= T[dE / 4 - 1];", "beta_zero or boltzmann"),
    ("weight_wrong_level_spacing", "return exp(-(fabs(dbeta) * (double)(4 * j)));",
     "return exp(-(fabs(dbeta) * (double)(2 * j)));", "weights or tau_table or lnQ"),
    ("weight_signed_dbeta", "return exp(-(fabs(dbeta) * (double)(4 * j)));",
     "return exp(-(dbeta * (double)(4 * j)));", "weights"),
    ("lnQ_sign_of_reference_energy", "- dbeta * (double)Eref;", "+ dbeta * (double)Eref;",
     "lnQ"),
    ("tau_normalised_by_current_R", "r->S = or_tau_table(r->H, r->bins, Dtab, c->R0,",
     "r->S = or_tau_table(r->H, r->bins, Dtab, r->R,", "lnZ_and_energy_match_kaufman"),
    ("tau_missing_reference_shift",
     "            int64_t j = heating ? kref - k : k - kref;\n            if (j >= 0) acc",
     "            int64_t j = heating ? kref - k : k;\n            if (j >= 0) acc", "tau_table"),
    ("counts_compare_reversed", "r[i] = n[k] + (u < F[k] ? 1u : 0u);",
     "r[i] = n[k] + (u > F[k] ? 1u : 0u);", "copy_counts"),
    ("offsets_inclusive", "        r->o[j] = (uint32_t)total;\n        total += r->r[j];",
     "        total += r->r[j];\n        r->o[j] = (uint32_t)total;", "copies_are_exact"),
    ("init_one_word_per_block", "spins[s] = (out[s & 3] >> 31) ? -1 : 1;",
     "spins[s] = (out[0] >> 31) ? -1 : 1;", "fair_coins"),
    ("cv_sign", "(mE2 - mE * mE)", "(mE2 + mE * mE)", "observables"),
    # observables against exact Boltzmann values (not against a restatement)
    ("cv_missing_beta_squared", "o->cv = ((o->beta * o->beta) * (mE2 - mE * mE)) / Nd;",
     "o->cv = (mE2 - mE * mE) / Nd;", "observables_match_bruteforce or specific_heat"),
    ("cv_not_per_site", "o->cv = ((o->beta * o->beta) * (mE2 - mE * mE)) / Nd;",
     "o->cv = (o->beta * o->beta) * (mE2 - mE * mE);",
     "observables_match_bruteforce or specific_heat"),
    ("chi_signed_mean_for_abs_mean", "o->chi = (o->beta * (mM2 - mA * mA)) / Nd;",
     "o->chi = (o->beta * mM2) / Nd;", "observables_match_bruteforce"),
    ("chi_missing_beta", "o->chi = (o->beta * (mM2 - mA * mA)) / Nd;",
     "o->chi = (mM2 - mA * mA) / Nd;", "observables_match_bruteforce"),
    ("m_abs_root_mean_square", "o->m_abs = mA / Nd;", "o->m_abs = sqrt(mM2) / Nd;",
     "observables_match_bruteforce"),
    ("heating_uses_lowest_level",
     "{\n    int64_t kref = -1;\n    if (heating) {\n        for (int64_t k = bins - 1; k >= 0; --k)",
     "{\n    int64_t kref = -1;\n    if (heating) {\n        for (int64_t k = 0; k < bins; ++k)",
     "tau_table"),
    ("overlap_heating_uses_lowest_level",
     "dbeta < 0.0;\n    int64_t kref = -1;\n    if (heating) {\n        for (int64_t k = bins - 1;"
     " k >= 0; --k)",
     "dbeta < 0.0;\n    int64_t kref = -1;\n    if (heating) {\n        for (int64_t k = 0; k < bins;"
     " ++k)", "overlap"),
    ("overlap_uses_max", "a = a + (p < q ? p : q);", "a = a + (p > q ? p : q);", "overlap"),
    ("poisson_thinning_reversed", "if (next_u(&s) < F[k]) ++count;",
     "if (next_u(&s) >= F[k]) ++count;", "poisson_counts"),
    ("poisson_fraction_dropped", "uint32_t events = poisson1(&s, T, len);",
     "uint32_t events = 0;", "poisson_counts"),
    ("poisson1_wrong_factorial", "if (m > 0) term = term / (double)m;",
     "if (m > 0) term = term / (double)(m + 1);", "poisson1_thresholds or poisson_counts"),
    ("poisson_one_unit_draw_short", "for (uint32_t j = 0; j < n[k]; ++j)",
     "for (uint32_t j = 1; j < n[k]; ++j)", "poisson_counts"),
    ("poisson_one_stream_for_all", "or_ustream s = { c, (uint32_t)i,", "or_ustream s = { c, 0u,",
     "poisson_counts_are_independent"),
    ("multinomial_last_replica_never_drawn", "int64_t lo = 0, hi = R - 1;          /* first i",
     "int64_t lo = 0, hi = R - 2;          /* first i", "multinomial"),
    ("multinomial_low_word_only",
     "uint64_t v = (uint64_t)out[2 * (j & 1)] | ((uint64_t)out[2 * (j & 1) + 1] << 32);",
     "uint64_t v = (uint64_t)out[2 * (j & 1)];", "multinomial"),
    ("multinomial_one_draw_short", "for (int64_t j = 0; j < c->R0; ++j) {\n        uint32_t out[4];\n"
     "        draw(c->seed, (uint32_t)(j >> 1)",
     "for (int64_t j = 0; j < c->R0 - 1; ++j) {\n        uint32_t out[4];\n"
     "        draw(c->seed, (uint32_t)(j >> 1)", "multinomial"),
    ("multinomial_pair_shares_words",
     "uint64_t v = (uint64_t)out[2 * (j & 1)] | ((uint64_t)out[2 * (j & 1) + 1] << 32);",
     "uint64_t v = (uint64_t)out[0] | ((uint64_t)out[1] << 32);", "multinomial"),
    ("ground_state_lnZ_wrong_sign", "r->lnZ = log(2.0) + c->beta0 *",
     "r->lnZ = log(2.0) - c->beta0 *", "heating_starts"),
    # the exchange between virtual GPUs (or_permute)
    ("permute_tracked_energy_left_behind", "            r->U2[dst] = r->U[from];\n        }\n"
     "    int8_t* ts", "        }\n    int8_t* ts", "permute_moves_whole_replicas"),
    ("permute_ignores_the_source_slot", "int64_t from = src[q] + k;", "int64_t from = dst;",
     "permute_moves_whole_replicas"),
    ("permute_repeats_the_segment_start", "int64_t from = src[q] + k;",
     "int64_t from = src[q];", "permute_moves_whole_replicas"),
    ("permute_lengths_not_checked", "    if (total != r->R) return -1;\n    int64_t dst = 0;",
     "    int64_t dst = 0;", "permute_moves_whole_replicas"),
]


def _build_mutant(tmp, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    d = tmp
    shutil.copy(os.path.join(ROOT, "oracle", "pa_oracle.h"), d)
    with open(os.path.join(d, "pa_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(d, "libmutant.so")
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", lib,
                    os.path.join(d, "pa_oracle.c"), "-lm"], check=True)
    return lib


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new,keys", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, keys):
    lib = _build_mutant(str(tmp_path), old, new)
    env = dict(os.environ, PA_ORACLE_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           os.path.join(HERE, "test_oracle_pins.py"),
           os.path.join(HERE, "test_oracle_pa_statistics.py"),
           os.path.join(HERE, "test_redistribute.py"), "-k", keys]
    proc = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900, cwd=ROOT)
    tail = proc.stdout[-400:]
    assert "passed" in tail or "failed" in tail, tail + proc.stderr[-400:]
    assert proc.returncode == 1 and "failed" in tail, f"mutant {name} survived:\n{tail}"
