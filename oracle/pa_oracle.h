/*
 * pa_oracle.h -- plain, slow, single-threaded CPU oracle of one population-
 * annealing (PA) run.  TEST INFRASTRUCTURE ONLY: it is called by the tests,
 * by __graft_entry__.smoke() and by the cpu_baseline leg of bench.py, never by
 * the product path.  It shares no code, header, table or constant generator
 * with the CUDA engine under paper_2006_00561_gb300/.
 *
 * What it computes (Russkov, Chulkevich & Shchur, "Algorithm for the replica
 * redistribution in the implementation of parallel annealing method on the
 * hybrid supercomputer architecture", Sec. 2 and Sec. 3):
 *   - Eq. 6 Hamiltonian on an L^d periodic lattice (d = 2 ferromagnet, or the
 *     +-J Edwards-Anderson variant with one coupling per bond),
 *   - an initial population of R0 uniformly random states at beta0 (Sec. 2),
 *   - per annealing step i: the partition-function ratio Q (Eq. 3), the
 *     normalised weights tau (Eq. 4), resampling into exact copies (Sec. 2:
 *     the Poisson draw, or its nearest-integer variant), theta
 *     checkerboard Metropolis sweeps at beta_i, then observables and the
 *     free-energy recursion (Eq. 5, read as ln Z_i = N ln 2 + sum ln Q).
 *
 * Spins are int8 +-1, sites are visited one by one in ascending order.  The
 * random numbers come from Philox4x32-10 written here from its published
 * definition (Salmon, Moraes, Dror & Shaw, SC'11), with counters keyed by the
 * logical site, so that any implementation of the same rules produces the
 * same bits.  Parity pins for every function live in tests/test_oracle_*.py.
 */
#ifndef PA_ORACLE_H
#define PA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Counter tags (top four bits of counter word 3; the low 28 bits hold the
 * instance id). */
#define OR_TAG_INIT     1u
#define OR_TAG_SWEEP    2u
#define OR_TAG_RESAMPLE 3u
#define OR_TAG_COUPLING 4u
#define OR_TAG_POISSON  5u
#define OR_TAG_MULTINOMIAL 6u

/* Copy-count rules of the resampling step (Sec. 2). */
#define OR_RESAMPLE_NEAREST 0  /* r = floor(tau) + [u < frac(tau)]        */
#define OR_RESAMPLE_POISSON 1  /* r ~ Poisson(tau)                         */
#define OR_RESAMPLE_MULTINOMIAL 2  /* R0 draws, replica i w.p. tau_i / sum tau */

#define OR_MODEL_FERRO 0   /* J_ij = +1 on every bond (Eq. 6)            */
#define OR_MODEL_PMJ   1   /* J_ij = +-1 with p = 1/2, one draw per bond */

typedef struct {
    int32_t  dim;           /* 2 or 3                                    */
    int32_t  L;             /* even, >= 2                                */
    int32_t  model;         /* OR_MODEL_FERRO | OR_MODEL_PMJ             */
    int32_t  K;             /* annealing steps                           */
    int32_t  theta;         /* Metropolis sweeps per step                */
    int32_t  instance_id;   /* < 2^28                                    */
    int64_t  R0;            /* initial population                        */
    int64_t  capacity;      /* largest population accepted               */
    double   beta0, beta_max;
    uint64_t seed;          /* Philox key of init / sweep / resample     */
    uint64_t coupling_seed; /* Philox key of the +-J bonds               */
    int32_t  init;          /* OR_INIT_RANDOM | OR_INIT_GROUND           */
    int32_t  resample;      /* OR_RESAMPLE_NEAREST | _POISSON | _MULTINOMIAL */
} or_config;

/* Initial population: uniform random states (cooling from beta0 = 0) or the
 * ferromagnet's ground state, all spins +1 (heating from near T = 0; Sec. 2
 * describes both protocols). */
#define OR_INIT_RANDOM 0
#define OR_INIT_GROUND 1

/* Observables after the sweeps at beta_i (Sec. 2: population averages). */
typedef struct {
    int64_t step, R;
    int64_t sumE, sumE2, sumAbsM, sumM2;
    double  beta, lnQ, lnZ;
    double  e, cv, m_abs, chi;
} or_obs;

/* ---- building blocks (each one a pure function) ---------------------- */
void     or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double   or_beta(const or_config* c, int32_t i);
uint64_t or_threshold(double beta, int32_t dE);
double   or_weight(double dbeta, int64_t j);
int64_t  or_num_bins(int32_t dim, int32_t L);

void     or_init_couplings(const or_config* c, int8_t* J /* [N*dim] */);
void     or_init_replica(const or_config* c, int64_t slot, int8_t* spins /* [N] */);
void     or_energy(int32_t dim, int32_t L, const int8_t* J, const int8_t* spins,
                   int64_t* U, int64_t* M);
int64_t  or_delta_e(int32_t dim, int32_t L, const int8_t* J, const int8_t* spins, int64_t s);
/* theta sweeps of one replica; g0 = global index of the first sweep;
 * T[c] = threshold for dE = 4(c+1).  Returns the tracked change of U. */
int64_t  or_sweep_replica(const or_config* c, const int8_t* J, int8_t* spins,
                          int64_t slot, int64_t g0, int32_t nsweeps, const uint64_t T[3]);
/* Eq. 3 / Eq. 4 on an energy histogram.  Writes n[], F[] (zero below kref),
 * returns S and the index of the lowest occupied bin. */
double   or_tau_table(const uint32_t* H, int64_t bins, const double* Dtab, int64_t R0,
                      int32_t heating, uint32_t* n, uint32_t* F, int64_t* kref);
void     or_copy_counts(const or_config* c, int32_t step, const uint32_t* ebin, int64_t R,
                        const uint32_t* n, const uint32_t* F, uint32_t* r);
/* Poisson(1) inversion table: T[m] = floor(2^32 P(X <= m)), X ~ Poisson(1),
 * for m = 0, 1, ... up to and including the first entry that reaches
 * 2^32 - 1 (at most cap entries).  Returns the number of entries. */
int32_t  or_poisson1_thresholds(uint32_t* T, int32_t cap);
/* Multinomial copy counts: R0 draws, replica i with probability
 * t_i / sum_j t_j, t_i = n_k 2^32 + F_k (k = level of replica i). */
void     or_copy_counts_multinomial(const or_config* c, int32_t step, const uint32_t* ebin,
                                    int64_t R, const uint32_t* n, const uint32_t* F, uint32_t* r);
/* Poisson copy counts r_i ~ Poisson(tau_k), tau_k = n_k + F_k / 2^32. */
void     or_copy_counts_poisson(const or_config* c, int32_t step, const uint32_t* ebin,
                                int64_t R, const uint32_t* n, const uint32_t* F, uint32_t* r);
void     or_derive_obs(or_obs* o, int64_t N);

/* Histogram overlap between the population at the current beta (levels H,
 * R replicas) and its reweighting to beta + dbeta:
 *   alpha = sum_k min(H_k / R, H_k w_k / sum_j H_j w_j),
 *   w_k = D[|k - kref|] of or_weight.  Sums run over k ascending from 0.0. */
double   or_overlap(const uint32_t* H, int64_t bins, int64_t R, double dbeta);
/* Adaptive step: the largest beta_next in [beta, beta_end] (or (beta_end,
 * beta] when heating) whose overlap is >= target, by 60 bisection steps on
 * |dbeta| (beta_end itself when its overlap suffices). */
double   or_adaptive_next(const uint32_t* H, int64_t bins, int64_t R, double beta,
                          double beta_end, double target);

/* ---- a whole run ------------------------------------------------------- */
typedef struct or_run or_run;
or_run*  or_create(const or_config* c);      /* NULL on bad config */
void     or_destroy(or_run* r);
int      or_resample(or_run* r);              /* beta_{i-1} -> beta_i; 0 ok, <0 error */
/* Resample to an arbitrary next inverse temperature (the step index still
 * advances by one; the thresholds of that step follow beta_next). */
int      or_resample_to(or_run* r, double beta_next);
double   or_current_beta(const or_run* r);
int      or_sweep(or_run* r, int32_t nsweeps);/* at beta_i, then measure           */
/* Replica exchange between virtual GPUs (Sec. 3): reorders the population's
 * slots; new slots take old slots src[q] .. src[q] + len[q] - 1 in order.
 * 0 ok, -1 if the segments leave [0, R) or do not cover R slots. */
int      or_permute(or_run* r, int32_t nseg, const int64_t* src, const int64_t* len);
int      or_step(or_run* r);                  /* or_resample + or_sweep(theta)      */
void     or_observables(const or_run* r, or_obs* out);
/* views into the run's current state (valid until the next call) */
int64_t        or_R(const or_run* r);
int64_t        or_N(const or_run* r);
int64_t        or_bins(const or_run* r);
int32_t        or_step_index(const or_run* r);
int64_t        or_sweep_counter(const or_run* r);
const int8_t*  or_spins(const or_run* r);     /* [R*N]                   */
const uint32_t* or_ebin(const or_run* r);     /* [R]                     */
const int32_t* or_mag(const or_run* r);       /* [R]                     */
const uint32_t* or_hist(const or_run* r);     /* [bins]                  */
const uint32_t* or_counts(const or_run* r);   /* [R_prev] of last resample */
const uint32_t* or_offsets(const or_run* r);  /* [R_prev]                */
const uint32_t* or_tab_n(const or_run* r);    /* [bins]                  */
const uint32_t* or_tab_F(const or_run* r);    /* [bins]                  */
const int8_t*  or_couplings(const or_run* r); /* [N*dim]                 */
int64_t        or_R_prev(const or_run* r);
int64_t        or_kref(const or_run* r);
double         or_S(const or_run* r);
int64_t        or_parity(const or_run* r);    /* U mod 2 (fixed per instance) */
int64_t        or_check_failures(const or_run* r); /* invariant failures seen */
double         or_lnQ(const or_run* r);       /* ln Q of the last resample  */
double         or_lnZ(const or_run* r);       /* N ln 2 + sum of ln Q       */

#ifdef __cplusplus
}
#endif
#endif
