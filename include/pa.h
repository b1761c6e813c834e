/*
 * pa.h -- C ABI of the GB300 population-annealing (PA) engine.
 *
 * Method: population annealing as stated in Russkov, Chulkevich & Shchur,
 * "Algorithm for the replica redistribution in the implementation of parallel
 * annealing method on the hybrid supercomputer architecture", Sec. 2:
 *   - start from R0 replicas at beta0 (Sec. 2, uniform states at beta0 = 0),
 *   - each step i moves the population from beta_{i-1} to beta_i: the
 *     partition-function ratio Q (Eq. 3), normalised weights tau (Eq. 4),
 *     resampling into exact copies (Sec. 2), theta Metropolis sweeps,
 *     observables, and the free-energy recursion (Eq. 5),
 * for the Ising model of Eq. 6 (2D ferromagnet) and its +-J Edwards-Anderson
 * variant (2D or 3D).  Everything runs on one GPU; the population never
 * leaves device memory except through pa_dump / pa_observables.
 *
 * Conventions for every entry point:
 *   - Return value: PA_OK (0) or a negative PA_ERR_* code; pa_strerror() names
 *     it.  A call that returns an error changes no state.
 *   - Device errors that happen inside an asynchronous step (population above
 *     capacity, a lookback wait that ran out, an invariant that failed) are
 *     recorded in a sticky status word in device memory; the next
 *     synchronising call (pa_observables, pa_status, pa_dump) reports them.
 *   - Memory: the library never allocates device memory.  The caller passes
 *     one device buffer of pa_workspace_size() bytes (256-byte aligned) and
 *     keeps it alive until pa_free(); the library owns only a small host
 *     handle.  Streams are plain cudaStream_t values passed as void*.
 *   - Threads: one pa_run must not be used from two host threads at once.
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PA_OK               0
#define PA_ERR_INVALID_ARG (-1)  /* NULL pointer, K < 1, R0 < 1, beta_max < beta0 ... */
#define PA_ERR_ODD_L       (-2)  /* the checkerboard update needs an even L           */
#define PA_ERR_UNSUPPORTED (-3)  /* (dim, L, layout) has no compiled kernel           */
#define PA_ERR_CAPACITY    (-4)  /* population above the configured capacity         */
#define PA_ERR_TIMEOUT     (-5)  /* a bounded device-side wait gave up                 */
#define PA_ERR_CUDA        (-6)  /* a CUDA runtime call failed                         */
#define PA_ERR_WORKSPACE   (-7)  /* workspace NULL, too small or not 256-B aligned     */
#define PA_ERR_DONE        (-8)  /* resample asked beyond step K                       */
#define PA_ERR_EMPTY       (-9)  /* the population died out (R = 0)                    */
#define PA_ERR_INVARIANT   (-10) /* device check failed: sum_k H_k != R                */

/* ---- models and layouts ------------------------------------------------ */
#define PA_MODEL_FERRO   0  /* J_ij = +1 on every bond: Eq. 6                           */
#define PA_MODEL_PMJ     1  /* J_ij = +-1, p = 1/2 per bond, drawn from coupling_seed   */

#define PA_LAYOUT_INT8   0  /* one int8 (+1/-1) per site, row-major s = x + L y (+L^2 z) */
#define PA_LAYOUT_PACKED 1  /* one bit per site (1 = spin -1); rows along x of
                               ceil(L/32) little-endian 32-bit words             */

/* Supported sizes (anything else returns PA_ERR_UNSUPPORTED):
 *   dim 2: L in {4, 8, 16, 32, 64, 128};  dim 3: L in {2, 4, 6, 8, 10, 12, 16}. */

/* One PA run.  beta_i = beta0 + (beta_max - beta0) * i / K, i = 0..K (Sec. 3
 * uses a constant step); beta_max is the final inverse temperature and may be
 * below beta0 (heating).  capacity = largest population the workspace holds;
 * 0 selects R0 + 16 ceil(sqrt(R0)) + 1024.  instance_id < 2^28 separates the
 * random streams of runs that share a seed.  init chooses the initial
 * population (Sec. 2 describes both protocols): PA_INIT_RANDOM, uniform random
 * states (cooling from beta0 = 0, ln Omega = N ln 2), or PA_INIT_GROUND, the
 * ferromagnet's ground state with all spins +1 (heating from near T = 0,
 * ln Omega = ln 2 + beta0 dim N for the two ground states). */
#define PA_INIT_RANDOM 0
#define PA_INIT_GROUND 1
/* Copy counts of the resampling step (Sec. 2), from the normalised weight
 * tau_k = n_k + F_k / 2^32 of the replica's level (Eq. 4):
 *   PA_RESAMPLE_NEAREST  r = n_k + [u < F_k], one 32-bit uniform per replica;
 *   PA_RESAMPLE_POISSON  r ~ Poisson(tau_k), the draw Sec. 2 prescribes: the
 *     event count of a unit-rate Poisson process on [0, tau_k], i.e. n_k
 *     Poisson(1) counts (inversion against pa_poisson1_table) plus one
 *     Poisson(1) count thinned with keep probability F_k / 2^32; uniforms from
 *     Philox blocks (i, step, b, POISSON|id), b = 0, 1, ..., fractional count
 *     and its thinning draws first.  The population is then Poisson(R0). */
#define PA_RESAMPLE_NEAREST 0
#define PA_RESAMPLE_POISSON 1
/*   PA_RESAMPLE_MULTINOMIAL  the new population is R0 independent draws from
 *     the old one, replica i with probability t_i / sum_j t_j where
 *     t_i = n_k 2^32 + F_k (tau in 32.32 fixed point, so the cumulative weights
 *     C_i are exact); draw j uses the 64-bit uniform v of Philox block
 *     (j >> 1, step, 0, MULTINOMIAL|id) (words 2(j & 1) low, 2(j & 1) + 1 high),
 *     the point x = floor(v C_{R-1} / 2^64) and the first replica with C_i > x.
 *     The population stays exactly R0.  In a batch, the draws of each such
 *     run are launched per run between the batched reweight and resample. */
#define PA_RESAMPLE_MULTINOMIAL 2
typedef struct {
    int32_t  dim;           /* 2 or 3                                  */
    int32_t  L;             /* linear size, even                        */
    int32_t  model;         /* PA_MODEL_*                               */
    int32_t  layout;        /* PA_LAYOUT_*                              */
    int32_t  K;             /* number of annealing steps, >= 1          */
    int32_t  theta;         /* Metropolis sweeps per step, >= 0         */
    int32_t  instance_id;   /* 0 .. 2^28-1                              */
    int32_t  init;          /* PA_INIT_RANDOM | PA_INIT_GROUND          */
    int64_t  R0;            /* initial population, 1 .. 2^31            */
    int64_t  capacity;      /* 0 = default                              */
    double   beta0, beta_max;
    uint64_t seed;          /* Philox key: init, sweeps, resampling     */
    uint64_t coupling_seed; /* Philox key of the +-J couplings          */
    int32_t  resample;      /* PA_RESAMPLE_NEAREST | _POISSON | _MULTINOMIAL */
    int32_t  reserved;      /* must be 0                                */
} pa_config;

/* Population averages after the sweeps at beta_i (Sec. 2), from exact
 * integer sums over the population: E = 2U - dim N (U = unsatisfied bonds),
 * M = sum of spins.
 *   e     = <E>/N                  cv  = beta^2 (<E^2> - <E>^2) / N
 *   m_abs = <|M|>/N                chi = beta (<M^2> - <|M|>^2) / N
 *   lnQ   = ln Q(beta_{i-1}, beta_i) of Eq. 3 (0 at step 0)
 *   lnZ   = N ln 2 + sum_{l<=i} ln Q_l, i.e. -beta_i F(beta_i) of Eq. 5 when
 *           beta0 = 0 (ln of the number of states at infinite temperature). */
typedef struct {
    int64_t step, R;
    int64_t sumE, sumE2, sumAbsM, sumM2;
    double  beta, lnQ, lnZ;
    double  e, cv, m_abs, chi;
} pa_obs;

typedef struct pa_run pa_run;

/* Bytes of device workspace one run needs; 0 if the config is invalid. */
size_t pa_workspace_size(const pa_config* cfg);

/* Creates a run in the caller's workspace and enqueues, on `stream`, the
 * initial population at beta0 (uniform random states), the couplings, and
 * the measurement of step 0.  The host tables (Metropolis thresholds and the
 * Eq. 3 weights of every step) are built here in IEEE double and copied to
 * the workspace; this is the only host-to-device copy of a run.
 * *out receives the handle.  Returns PA_ERR_WORKSPACE if `bytes` is too small
 * or the pointer is not 256-byte aligned. */
int pa_init(const pa_config* cfg, void* dev_workspace, size_t bytes, void* stream,
            pa_run** out);

/* Step i = current + 1 of the annealing (beta_{i-1} -> beta_i), first half:
 * energy histogram -> Q (Eq. 3) and the per-energy tau table (Eq. 4) ->
 * copy counts r_j by the rule pa_config.resample selects (Sec. 2's
 * resampling step): PA_RESAMPLE_NEAREST, r_j = floor(tau) + [u_j < frac(tau)];
 * PA_RESAMPLE_POISSON, r_j ~ Poisson(tau), the draw Sec. 2 prescribes;
 * PA_RESAMPLE_MULTINOMIAL, R0 independent draws weighted by tau -> exclusive
 * scan -> gather of exact copies into the other population buffer.
 * Asynchronous on the run's stream; needs a measured population (a sweep,
 * possibly of 0 sweeps, since the last resample). */
int pa_resample(pa_run* run);

/* nsweeps checkerboard Metropolis sweeps at the current beta_i, then the
 * energy/magnetisation of every replica, the energy histogram and the
 * observables record of step i.  nsweeps = 0 only measures.  Asynchronous. */
int pa_sweep(pa_run* run, int32_t nsweeps);

/* Redistribution of the population between virtual GPUs (Sec. 3: after the
 * resampling step the replicas are exchanged so that every GPU holds about
 * R / N of them, by the main block algorithm or the naive per-replica one).
 * On one GPU the N "GPUs" are consecutive slot ranges of the population, and
 * the exchange is a permutation of the new population's slots.  It is split
 * in two calls around the host's exchange plan:
 *   pa_resample_begin  the first half of pa_resample (reweight, copy counts,
 *                      exclusive scan) without the gather: afterwards
 *                      PA_DUMP_COUNTS / PA_DUMP_OFFSETS and pa_dump(STATE)
 *                      give R_i and the offspring ranges (the offspring of
 *                      old slots [a, b) are new slots [o_a, o_b)).
 *   pa_resample_finish the gather, into a slot order given as nseg segments
 *                      of the new population: post-exchange slots are filled
 *                      in order with new slots seg_src[q] ..
 *                      seg_src[q] + seg_len[q] - 1 for q = 0 .. nseg - 1
 *                      (host arrays; 1 <= nseg <= PA_MAX_SEGMENTS; each
 *                      segment inside [0, R_i) and the lengths summing to
 *                      R_i, else PA_ERR_INVALID_ARG).  One segment (0, R_i)
 *                      is the plain step's order.  Synchronises (reads R_i).
 * The replicas move in device memory: every slot's spins, energy level and
 * magnetisation are written once, by the same gather that completes a plain
 * resample.  Between the two calls every other stepping call, pa_load,
 * pa_checkpoint, pa_restore and pa_batch_init return PA_ERR_INVALID_ARG. */
#define PA_MAX_SEGMENTS 1024
int pa_resample_begin(pa_run* run);
int pa_resample_finish(pa_run* run, int32_t nseg, const int64_t* seg_src, const int64_t* seg_len);

/* pa_resample followed by pa_sweep(theta). */
int pa_step(pa_run* run);

/* pa_step with the new population streamed to host memory while it is swept
 * (Sec. 2's step; the copy out is for callers that keep the population on the
 * host).  The reweight and resample of step i run on the run's stream, and the
 * call waits for them to learn R_i and the buffer of the new population.  The
 * theta sweeps then run over `chunks` ranges of consecutive slots (bounds are
 * multiples of 32; the last range ends at R_i), and after each range its
 * replicas are copied in the device layout (stride bytes each, as
 * PA_DUMP_SPINS_RAW gives them) to host_dst + first_slot * stride on
 * copy_stream, while the next range sweeps.  The measurement follows on the
 * run's stream, which then waits for the last copy: once pa_observables (or
 * any synchronising call) returns, host_dst holds replicas 0 .. R_i - 1.
 * Results are bit-identical to pa_step.
 *   host_dst     pinned host memory for the copies to overlap the sweeps;
 *                bytes >= capacity * stride;
 *   chunks       1 .. 64;
 *   copy_stream  a cudaStream_t other than the run's;
 *   R_out        receives R_i (may be NULL).
 * PA_ERR_INVALID_ARG for bad arguments (nothing enqueued); the sticky error of
 * the resample (e.g. PA_ERR_CAPACITY) if it failed, with nothing swept. */
int pa_step_stream(pa_run* run, void* host_dst, size_t bytes, int32_t chunks, void* copy_stream,
                   int64_t* R_out);

/* The random-number ceiling of the register sweep kernels (a measurement,
 * not part of a run): the Philox4x32-10 blocks of the L = 64 kernel, one
 * persistent 16-warp block per SM (the shape in which the generator alone
 * runs fastest; the sweep kernel runs 12 warps), one warp per replica, each
 * lane drawing 16 blocks per half-sweep with the half-sweep products
 * shared and the round-2 and round-3 block products from shared-memory
 * tables (as the sweep kernel draws them; the round-3 table is rebuilt every
 * 48 half-sweeps), with nothing done to the uniforms but an xor into one word per
 * thread.  Thread t writes out_dev[t] = xor over half-sweeps g < halfsweeps
 * and blocks b = 16 (t mod 32) .. + 15 of the four words of the block with
 * counter (2g, b, SWEEP << 28, t / 32) under key `seed`.  Uniforms drawn:
 * pa_bench_philox_threads() * halfsweeps * 64.  out_dev: device memory of
 * at least pa_bench_philox_threads() words, else PA_ERR_INVALID_ARG.
 * Asynchronous on `stream` (cudaStream_t). */
int64_t pa_bench_philox_threads(void);
int pa_bench_philox(uint64_t seed, int32_t halfsweeps, void* out_dev, int64_t out_words,
                    void* stream);

/* Integer-pipe throughput of this GPU (a measurement, not part of a run): the
 * peak the sweep kernels' integer work is reported against.  The paper has no
 * counterpart; its kernels' bound (Sec. 2: theta Metropolis sweeps per step)
 * is integer issue here.  One launch of pa_bench_intops_threads() resident
 * threads, each running `iters` iterations of pa_bench_intops_per_iter()
 * independent dependency chains, one instruction per chain and iteration, of
 * the kind selected:
 *   PA_INTOPS_LOP3       three-input logic op (lop3.b32)
 *   PA_INTOPS_IMAD       32-bit multiply-add (mad.lo.u32)
 *   PA_INTOPS_WIDE       32 x 32 -> 64 multiply with a 64-bit add (mad.wide.u32)
 *   PA_INTOPS_LOP3_IMAD  the two interleaved 1:1
 *   PA_INTOPS_LOP3_WIDE  lop3 and mad.wide interleaved 1:1
 *   PA_INTOPS_MULWIDE_XOR  x <- hi(x b) xor lo(x b): mul.wide.u32 then a
 *                        two-input xor, both halves consumed -- one multiply
 *                        of a Philox4x32 round with its xor; two instructions
 *                        per chain step
 * Chain steps executed = threads * iters * per_iter.  out_dev: device memory
 * of at least pa_bench_intops_threads() 32-bit words (one folded result per
 * thread), else PA_ERR_INVALID_ARG; an unknown kind or iters < 1 is
 * PA_ERR_INVALID_ARG.  Asynchronous on `stream` (cudaStream_t). */
#define PA_INTOPS_LOP3      0
#define PA_INTOPS_IMAD      1
#define PA_INTOPS_WIDE      2
#define PA_INTOPS_LOP3_IMAD 3
#define PA_INTOPS_LOP3_WIDE 4
#define PA_INTOPS_MULWIDE_XOR 5
int64_t pa_bench_intops_threads(void);
int64_t pa_bench_intops_per_iter(void);
int pa_bench_intops(int32_t kind, int32_t iters, void* out_dev, int64_t out_words, void* stream);

/* Test hooks for the failure paths (0 in normal operation).
 * PA_DEBUG_WITHHOLD_PREFIX: the resample's tile 0 does not publish its
 * lookback prefix, so tile 1's wait for it (at most 2^22 polls, about a
 * second or two) runs out: the kernel sets the sticky PA_ERR_TIMEOUT, gives up
 * that lookback and finishes (its copies land inside the population
 * buffer, at wrong offsets), and the next synchronising call returns
 * PA_ERR_TIMEOUT.  No fault, no hang: the context stays usable.  Takes effect
 * from the next enqueued step; not for graph replay.  Returns PA_OK, or
 * PA_ERR_INVALID_ARG for unknown bits. */
#define PA_DEBUG_WITHHOLD_PREFIX 1u
int pa_debug(pa_run* run, uint32_t flags);

/* nsteps calls of pa_step, replayed from a CUDA graph of one step that is
 * captured on first use (on a private stream, then launched on the run's
 * stream).  Same results as nsteps pa_step calls. */
int pa_run_steps(pa_run* run, int32_t nsteps);

/* Synchronises the run's stream and copies the observables of the latest
 * measured step into *out.  Reports sticky device errors. */
int pa_observables(pa_run* run, pa_obs* out);

/* Copies the records of steps first .. first+n-1 (each written when that step
 * was measured) into out[0..n-1].  Synchronises. */
int pa_observables_history(pa_run* run, int32_t first, int32_t n, pa_obs* out);

/* Synchronises and returns the sticky device status as a PA_ERR_* code. */
int pa_status(pa_run* run);

/* Test / inspection hook: synchronises and copies one array of the current
 * state into host memory.  `bytes` must be at least the size pa_dump_size()
 * reports.  The spin dump PA_DUMP_SPINS is converted to int8 +-1 in site
 * order s = x + L y (+ L^2 z), whatever the layout. */
#define PA_DUMP_SPINS      0  /* int8  [R][N]                                  */
#define PA_DUMP_EBIN       1  /* u32   [R]   energy level k = U >> 1           */
#define PA_DUMP_MAG        2  /* i32   [R]   magnetisation M                   */
#define PA_DUMP_HIST       3  /* u32   [bins] histogram of k (last measurement)*/
#define PA_DUMP_COUNTS     4  /* u32   [R_prev] copy counts r of last resample */
#define PA_DUMP_OFFSETS    5  /* u32   [R_prev] exclusive scan o of the counts */
#define PA_DUMP_TAB_N      6  /* u32   [bins] floor(tau_k) of last resample    */
#define PA_DUMP_TAB_F      7  /* u32   [bins] floor(frac(tau_k) 2^32)          */
#define PA_DUMP_COUPLINGS  8  /* int8  [N][dim] J of bond (s, s + e_d)         */
#define PA_DUMP_SPINS_RAW  9  /* bytes [R][stride] device layout               */
#define PA_DUMP_STATE     10  /* pa_state                                       */
int64_t pa_dump_size(pa_run* run, int32_t what);
int pa_dump(pa_run* run, int32_t what, void* host_dst, size_t bytes);

/* pa_dump restricted to replicas first .. first+count-1 of a per-replica array
 * (PA_DUMP_SPINS, _SPINS_RAW, _EBIN, _MAG: slots of the current population;
 * _COUNTS, _OFFSETS: slots of the population that entered the last resample).
 * bytes >= count * (N, stride or 4).  PA_ERR_INVALID_ARG if the range leaves
 * the population.  Synchronises. */
int pa_dump_range(pa_run* run, int32_t what, int64_t first, int64_t count, void* host_dst,
                  size_t bytes);

/* Scalar run state as seen by the device.  sources counts, over every
 * resample of the run so far, the replicas that received at least one copy
 * (the replicas whose spins the gather reads). */
typedef struct {
    int64_t step, R, R_prev, kref, sweeps_done, status_bits;
    double  lnQ, lnZ, S;
    int64_t N, bins, stride, capacity, parity;
    int64_t sources;
} pa_state;

/* Host-side tables the engine uploads, for bitwise comparison before any
 * kernel runs (no GPU needed): T[c] = floor(2^32 exp(-beta_i 4(c+1))), c=0..2,
 * the Metropolis acceptance thresholds at beta_i, and D[j] = exp(-|beta_i -
 * beta_{i-1}| 4 j), j = 0..bins-1, the Eq. 3 weights of the level j steps
 * away from the reference level (levels are 4 apart; the reference is the
 * lowest occupied level when cooling, the highest when heating).  D is not
 * written for step 0. */
int pa_tables(const pa_config* cfg, int32_t step, uint64_t T[3], double* D, int64_t bins);

/* The Poisson(1) inversion table of PA_RESAMPLE_POISSON, host side:
 * T[m] = floor(2^32 P(X <= m)), X ~ Poisson(1), m = 0, 1, ... up to and
 * including the first entry that reaches 2^32 - 1.  Writes at most cap entries
 * and returns how many the table has (13), or PA_ERR_INVALID_ARG. */
int pa_poisson1_table(uint32_t* T, int32_t cap);

/* Energy levels of (dim, L): dim L^dim / 2 + 1. */
int64_t pa_num_bins(int32_t dim, int32_t L);

/* Replaces the current population with `count` replicas read from host memory
 * (what = PA_DUMP_SPINS: int8 +-1 per site in site order; PA_DUMP_SPINS_RAW:
 * the device layout, `stride` bytes per replica as pa_dump gives it), then
 * measures it (energy levels, magnetisations, histogram, observables record
 * of the current step) exactly as pa_sweep(run, 0) does.  count must lie in
 * 1 .. capacity; bytes >= count * (N or stride).  The step index, ln Z and
 * the sweep counter are kept, so dump + load round-trips a population.
 * With pinned host memory the copy is asynchronous on the run's stream; the
 * caller keeps host_src alive until the stream reaches it. */
int pa_load(pa_run* run, int32_t what, const void* host_src, int64_t count, size_t bytes);

/* Adaptive temperature step (Sec. 3 points to the adaptive step of its
 * reference).  pa_adaptive_beta synchronises, reads the energy histogram of the
 * measured population at the current beta, and returns in *beta_next the
 * largest step towards beta_end (smaller than beta for heating) whose
 * reweighted histogram still overlaps the current one by at least
 * overlap_target, where overlap = sum_k min(H_k / R, H_k w_k / sum_j H_j w_j)
 * and w_k = exp(-|dbeta| 4 |k - kref|) (60 bisection steps on |dbeta|; beta_end
 * itself when its overlap suffices).  The decision is taken on the host in
 * IEEE double with libm exp, in a fixed order.
 * Call it between steps (after the sweeps of the current step), when the
 * histogram describes the current population.
 * pa_resample_to is pa_resample towards an arbitrary beta_next >= 0: the step
 * index i advances by one, and step i's beta, thresholds and weight table are
 * replaced (weight tables of such steps go to two slots reserved in the
 * workspace).  Later pa_step / pa_resample calls keep the fixed schedule's
 * betas, the first of them with its temperature step taken from beta_next, so
 * adaptive and scheduled steps can be mixed.  Synchronises; PA_ERR_DONE once
 * the step index would pass K. */
int pa_adaptive_beta(pa_run* run, double overlap_target, double beta_end, double* beta_next);
int pa_resample_to(pa_run* run, double beta_next);

/* Checkpoint / resume.  Random numbers are keyed by step, sweep index, slot
 * and site, so the complete state of a run at a step boundary is its
 * population (spins, energy levels, magnetisations), its energy histogram,
 * the per-step records and a few scalars (step, population sizes, sweep
 * counter, ln Z, ln Q, S).  pa_checkpoint writes them to host memory
 * (pa_checkpoint_size bytes; synchronises; refuses a run with a sticky error).
 * The current step's beta is stored too, so a run on adaptive steps resumes
 * from where it stood.  pa_restore loads such a checkpoint into a run created
 * with the same pa_config (compared byte for byte; PA_ERR_INVALID_ARG
 * otherwise), after which the run continues exactly as the checkpointed one
 * would have. */
int64_t pa_checkpoint_size(pa_run* run);
int pa_checkpoint(pa_run* run, void* host_dst, size_t bytes);
int pa_restore(pa_run* run, const void* host_src, size_t bytes);

/* Kernel timing (for benchmarks): while enabled, every kernel the run
 * enqueues outside a CUDA graph is bracketed by CUDA events on the run's
 * stream.  pa_profile_read synchronises and returns, per kernel kind
 * (0 reweight/tau, 1 resample: counts + scan + gather, 2 sweep, 3 observables),
 * the number of launches and their summed device time in ms since the last
 * reset. */
int pa_profile(pa_run* run, int32_t enable);
int pa_profile_read(pa_run* run, int64_t launches[4], double ms[4], int32_t reset);

/* ---- batched form ---------------------------------------------------------
 * Many independent runs (for example a disorder ensemble of +-J instances of
 * mixed L and R0) advanced together: one step of every run costs one launch
 * per phase -- reweight (one CTA per run), resample (one global tile space in
 * which each run's tiles are claimed in order), one sweep launch per class of
 * runs sharing (layout, dim, L, model), observables (one CTA per run) --
 * instead of four launches per run.  Every run gives exactly the bits it gives
 * when stepped alone with pa_step.  The runs keep their own workspaces; the
 * batch holds only their descriptors, in a workspace of
 * pa_batch_workspace_size(nruns) bytes.  While a batch steps its runs, do not
 * call pa_step/pa_sweep/pa_resample on them; pa_batch_sync() waits for the
 * batch stream and returns the first sticky error of any run, after which the
 * per-run read calls (pa_observables, pa_dump, ...) see the batch's results. */
typedef struct pa_batch pa_batch;
size_t pa_batch_workspace_size(int32_t nruns);
int pa_batch_init(pa_run* const* runs, int32_t nruns, void* dev_workspace, size_t bytes,
                  void* stream, pa_batch** out);
/* pa_batch_init for callers that keep work in flight (a serving loop that
 * builds the next batch while the current one runs): the remaining steps of
 * every run come from the caller (steps_left[i], 0 .. K, host memory) instead
 * of the device, and nothing is waited for -- the descriptor uploads are
 * ordered on `stream` before the batch's first step.  The runs must not be
 * stepped by other work on other streams between this call and the batch's
 * steps unless the caller orders that work before them. */
int pa_batch_init_async(pa_run* const* runs, int32_t nruns, const int32_t* steps_left,
                        void* dev_workspace, size_t bytes, void* stream, pa_batch** out);
/* One annealing step of every run (PA_ERR_DONE once any run reached K). */
int pa_batch_step(pa_batch* batch);
/* nsteps steps replayed from a CUDA graph of one batched step. */
int pa_batch_run_steps(pa_batch* batch, int32_t nsteps);
int pa_batch_sync(pa_batch* batch);
/* Phase timing of a batched step (for benchmarks): while enabled, every step
 * enqueued by pa_batch_step (not graph replays) is bracketed by CUDA events on
 * the batch stream.  pa_batch_profile_read synchronises and returns the number
 * of timed steps and their summed device time in ms per phase: 0 reweight of
 * every run, 1 resample (multinomial draws, counts, scan, gather), 2 the sweep
 * classes (fork to join of their parallel branches), 3 observables. */
int pa_batch_profile(pa_batch* batch, int32_t enable);
int pa_batch_profile_read(pa_batch* batch, int64_t* steps, double ms[4], int32_t reset);
/* Sweep classes and their launch shape: info = {layout, dim, L, model,
 * number of runs, warps per block, slots, slots per claim}.  The classes of
 * one step run as parallel branches.  pa_batch_set_shape chooses one class's
 * warps per block (2, 4 or 8; the L = 64 register kernel has 16 only; 0 keeps
 * the current value) and slots per claim (1, 2, 4, 8, 16 or 32; 0 picks the
 * largest that leaves about four claims per resident warp).  Results do not
 * depend on the shape. */
int pa_batch_num_classes(pa_batch* batch);
int pa_batch_class_info(pa_batch* batch, int32_t cls, int32_t info[8]);
int pa_batch_set_shape(pa_batch* batch, int32_t cls, int32_t warps, int32_t chunk);
void pa_batch_free(pa_batch* batch);

/* ---- copy counts and scan without device allocation ---------------------
 * The paper has no counterpart to this entry point: it exists for callers that
 * cannot allocate device memory at all -- code that runs while a CUDA graph is
 * being captured, plugins whose host process owns every allocation, embedded
 * callers with a fixed memory budget -- and so cannot provide pa_init's
 * workspace.
 *
 * For R replicas with energy levels d_ebin[0..R-1] (device memory) and the
 * per-level tables d_tab_n / d_tab_F [bins] of a resample (as PA_DUMP_TAB_N /
 * PA_DUMP_TAB_F give them), it writes the nearest-integer copy counts
 * d_counts[i] = n[k] + [u_i < F[k]], their exclusive scan d_offsets[i], and
 * the new population size *d_total, all in device memory, asynchronously on
 * `stream`.  u_i is the resampling uniform of replica i at annealing step
 * `step` under `seed` and `instance_id`, so the output equals the counts and
 * offsets pa_resample computes for the same population.
 *
 * It allocates nothing: the scratch of its single-pass scan lives in a static
 * device array of about 33 KB that every GPU loading this library holds until
 * the process exits.  R may be at most PA_NOALLOC_MAX_REPLICAS; larger R (or a
 * negative one, NULL pointers, bins < 1, a negative step or an instance id
 * >= 2^28) returns PA_ERR_INVALID_ARG before anything is enqueued.
 * The first call in each CUDA context (a device's primary context, or a
 * context the caller created and made current) looks up the array's address
 * in that context and caches it under the context's id; make that first call
 * before any stream capture.  Every call reuses the same array and clears what
 * it reads before writing it (the tile counter, the status bits and the
 * lookback descriptors of its tiles), so nothing an earlier call left behind
 * can leak into its result; but two calls whose kernels overlap on the GPU --
 * on different streams, or from different threads -- race and give wrong
 * results: serialise them.
 * *d_total reads 0xFFFFFFFF if a level was >= bins (that replica counts 0
 * copies) or if a bounded wait inside the scan gave up. */
#define PA_NOALLOC_MAX_REPLICAS 8388608
int pa_copy_counts_scan_noalloc(const uint32_t* d_ebin, int64_t R, const uint32_t* d_tab_n,
                                const uint32_t* d_tab_F, int64_t bins, uint64_t seed,
                                int32_t step, int32_t instance_id, uint32_t* d_counts,
                                uint32_t* d_offsets, uint32_t* d_total, void* stream);

/* Releases the host handle (and its CUDA graph).  The workspace stays the
 * caller's. */
void pa_free(pa_run* run);

const char* pa_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* PA_H */
