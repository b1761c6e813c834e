// pa_internal.cuh -- device-side data of one population-annealing run and the
// launchers the host engine (pa_engine.cu) calls.  Every array lives in the
// caller's workspace; the kernels read the run's scalars (population size,
// step index, buffer parity, sweep counter) from device memory, so a step can
// be enqueued or replayed from a CUDA graph without any host round trip.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pa.h"

namespace pa {

// Counter tags: top four bits of Philox counter word 3 (low 28 bits: instance).
constexpr uint32_t TAG_INIT = 1u;
constexpr uint32_t TAG_SWEEP = 2u;
constexpr uint32_t TAG_RESAMPLE = 3u;
constexpr uint32_t TAG_COUPLING = 4u;
constexpr uint32_t TAG_POISSON = 5u;
constexpr uint32_t TAG_MULTINOMIAL = 6u;
constexpr int P1_MAX = 16;  // entries of the Poisson(1) inversion table

// Sticky status bits of DevState::status.
constexpr uint32_t ST_CAPACITY = 1u;
constexpr uint32_t ST_TIMEOUT = 2u;
constexpr uint32_t ST_EMPTY = 4u;
constexpr uint32_t ST_DONE = 8u;
constexpr uint32_t ST_INVARIANT = 16u;

// Scalars of a run, in device memory (first 256 bytes of the workspace).
struct DevState {
    uint32_t step;          // current beta index i
    uint32_t R;             // current population size
    uint32_t R_prev;        // population entering the last resample
    uint32_t epoch;         // bumped by every reweight; tags lookback descriptors
    uint32_t tile_counter;  // dynamic tile ids of the resample kernel
    uint32_t status;        // sticky ST_* bits
    uint32_t cur;           // population buffer holding the current replicas
    uint32_t src;           // buffer the last resample read from
    uint32_t sweep_base;    // global index of the next Metropolis sweep
    uint32_t active;        // 1 if the reweight of this step succeeded
    uint32_t kref;          // lowest occupied energy level at the last reweight
    uint32_t negbonds;      // number of J = -1 bonds (U mod 2 = negbonds mod 2)
    double lnQ, lnZ, S;
    unsigned long long sweeps_done;
    unsigned long long tau_done;  // CTAs of the running multi-CTA reweight that are done
    unsigned long long sources;   // replicas with a copy count > 0, summed over all resamples
    unsigned long long pad[1];
};
static_assert(sizeof(DevState) <= 256, "DevState must fit its slot");

// Per-step record, same layout as pa_obs.
static_assert(sizeof(pa_obs) == 104, "pa_obs layout");

// Everything a kernel needs, passed by value.
struct RunDev {
    DevState* st;
    uint8_t* spins[2];          // population buffers, cap_alloc * stride bytes each
    uint32_t* ebin[2];          // energy level k = U >> 1 per replica
    int32_t* mag[2];            // magnetisation per replica
    uint32_t* counts;           // copy counts of the last resample
    uint32_t* offsets;          // exclusive scan of the counts
    uint32_t* srcmap;           // [cap] source replica of every slot the last resample filled
    uint32_t* srcmap2;          // [cap] the same after a redistribution permuted the slots
    unsigned long long* accum;  // [2] = sum |M|, sum M^2 of the running measurement
    uint32_t* hist;             // [bins] energy histogram of the running measurement
    uint32_t* tab_n;            // [bins] floor(tau_k)
    uint32_t* tab_F;            // [bins] floor(frac(tau_k) * 2^32)
    const uint32_t* thr;        // [(K+1)*4]: T0, T1, T2 (clamped to u32), bit c of [3] = T_c is 2^32
    const double* dtab;         // [ndist * bins] Eq. 3 weights
    const uint32_t* dsel;       // [K+1] weight table of step i
    const double* beta;         // [K+1]
    const double* dbeta;        // [K+1] beta_i - beta_{i-1} (negative when heating)
    unsigned long long* desc;   // [tiles] lookback descriptors
    unsigned long long* mn_cum;   // multinomial: [cap] cumulative fixed-point weights C_i
    unsigned long long* mn_tiles; // multinomial: [tiles + 1] tile prefixes, then the total
    pa_obs* obs;                // [K+1] per-step records
    uint32_t* jpk;              // packed couplings [dim][nwords] (bit set: J = -1), PMJ only
    int8_t* j8;                 // int8 couplings [N][dim], PMJ only
    uint64_t seed, coupling_seed;
    uint32_t instance;          // instance id (< 2^28)
    int32_t dim, L, layout, model, K;
    int64_t N, bins;
    uint32_t stride;            // bytes per replica (multiple of 16)
    uint32_t nwords;            // packed: 32-bit words per replica
    uint32_t cap;               // logical capacity
    uint32_t cap_alloc;         // slots in each buffer
    uint32_t R0;
    uint32_t tiles;             // descriptors available
    uint32_t rk0[10], rk1[10];  // Philox round keys of `seed` (key + r * Weyl constant)
    uint32_t one;               // the value 1, opaque to the compiler (multiply-add tests)
    int32_t theta;              // sweeps per annealing step
    int32_t init;               // PA_INIT_RANDOM | PA_INIT_GROUND
    int32_t resample;           // PA_RESAMPLE_NEAREST | PA_RESAMPLE_POISSON
    uint32_t p1_len;            // entries of p1
    uint32_t p1[P1_MAX];        // Poisson(1) thresholds floor(2^32 P(X <= m))
    // Slots the plain sweep kernels visit: [slot_lo, min(R, slot_hi)).  0 and
    // 0xffffffff (the whole population) except in the launches of a
    // streamed step, whose bounds are multiples of 32.
    uint32_t slot_lo, slot_hi;
    uint32_t debug;  // PA_DEBUG_* test hooks, 0 in normal operation
};

// A batch of runs stepped together (pa_batch_* in include/pa.h).  Arrays in
// the batch workspace; counters are cleared by the batched reweight kernel at
// the start of every step.
struct BatchDev {
    const RunDev* runs;          // [nruns]
    uint32_t nruns;
    const uint32_t* tile_base;   // [nruns + 1] prefix sums of each run's resample tiles
    uint32_t total_tiles;
    uint32_t any_poisson;        // some run resamples by the Poisson rule
    uint32_t any_multinomial;    // some run resamples by multinomial draws
    uint32_t* counters;          // [0]: resample tiles, [1 + c]: sweep chunks of class c
    uint32_t ncounters;
};

// One (layout, dim, L, model) class of a batch: the runs one sweep kernel
// instantiation serves.  Global slot g of the class lies in run run_ids[j]
// when slot_base[j] <= g < slot_base[j + 1] (capacities rounded up to 32, so
// a chunk of `chunk` slots never straddles two runs).
struct BatchSweepArgs {
    const RunDev* runs;
    const uint32_t* run_ids;     // [n]
    const uint32_t* slot_base;   // [n + 1]
    uint32_t n;
    uint32_t total_slots;
    uint32_t* counter;           // chunk counter of this class
    uint32_t chunk;              // slots per claim: 1, 2, 4, 8, 16 or 32
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies whose high halves are xored with the other words and the key;
// the key advances by the two Weyl constants after every round.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = c0, b = c2;
        const uint32_t hiA = __umulhi(0xD2511F53u, a), loA = 0xD2511F53u * a;
        const uint32_t hiB = __umulhi(0xCD9E8D57u, b), loB = 0xCD9E8D57u * b;
        c0 = hiB ^ c1 ^ k0;
        c1 = loB;
        c2 = hiA ^ c3 ^ k1;
        c3 = loA;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Same generator with the ten round keys taken from precomputed tables (the
// kernel-parameter copy of RunDev::rk0/rk1), so no key addition is issued.
__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const uint32_t* rk0, const uint32_t* rk1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = c0, b = c2;
        const uint32_t hiA = __umulhi(0xD2511F53u, a), loA = 0xD2511F53u * a;
        const uint32_t hiB = __umulhi(0xCD9E8D57u, b), loB = 0xCD9E8D57u * b;
        c0 = hiB ^ c1 ^ rk0[r];
        c1 = loB;
        c2 = hiA ^ c3 ^ rk1[r];
        c3 = loA;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint32_t pick(const uint4& v, uint32_t j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// ---- launchers (defined in the kernel translation units) ----------------
bool sweep_supported(int layout, int dim, int L);
cudaError_t launch_init(const RunDev& d, cudaStream_t s);
cudaError_t launch_sweep(const RunDev& d, int nsweeps, int grid, cudaStream_t s);
int sweep_grid(const RunDev& d);
cudaError_t launch_tau(const RunDev& d, cudaStream_t s);
cudaError_t launch_resample(const RunDev& d, cudaStream_t s);
// Redistribution between virtual GPUs (pa_resample_begin / pa_resample_finish):
// the counts and scan alone, then the gather into a permuted slot order.
// Post-exchange slots [dst[q], dst[q+1]) take the pre-exchange slots starting
// at src[q].
constexpr int MAX_SEGMENTS = 1024;
struct SegList {
    uint32_t n;
    uint32_t dst[MAX_SEGMENTS + 1];
    uint32_t src[MAX_SEGMENTS];
};
cudaError_t launch_resample_scan(const RunDev& d, cudaStream_t s);
cudaError_t launch_remap_gather(const RunDev& d, const SegList& segs, cudaStream_t s);
cudaError_t launch_multinomial(const RunDev& d, cudaStream_t s);
cudaError_t launch_obs(const RunDev& d, int nsweeps, cudaStream_t s);
// specialised 2D ferromagnet, L = 64 or 128, packed (pa_sweep_l64.cu)
bool l64_applies(const RunDev& d);
int l64_block_warps(const RunDev& d);
int l64_grid(const RunDev& d);
cudaError_t launch_sweep_l64(const RunDev& d, int nsweeps, int grid, cudaStream_t s);
// The register kernels' generator alone (pa_bench_philox).
int philox_rate_threads();
cudaError_t launch_philox_rate(uint64_t seed, uint32_t halfsweeps, uint32_t* out, cudaStream_t s);
// batched forms (one launch for every run of a batch, or of one class)
cudaError_t launch_tau_batched(const BatchDev& b, cudaStream_t s);
cudaError_t launch_resample_batched(const BatchDev& b, cudaStream_t s);
cudaError_t launch_obs_batched(const BatchDev& b, cudaStream_t s);
// sweep of one class; `warps` selects the block shape (an autotuned knob:
// 2, 4 or 8 warps per block for the shared-memory kernels; the L = 64
// register kernel has one shape), grid 0 = one wave of resident blocks
cudaError_t launch_sweep_batched(const BatchSweepArgs& a, const RunDev& proto, int warps, int grid,
                                 cudaStream_t s);
int batched_sweep_grid(const RunDev& proto, int warps);
bool batched_warps_valid(const RunDev& proto, int warps);
bool l64_batched_applies(const RunDev& proto);
cudaError_t launch_sweep_l64_batched(const BatchSweepArgs& a, const RunDev& proto, int grid,
                                     cudaStream_t s);
int l64_batched_grid(const RunDev& proto);

// Resample tiles: RS_ITEMS consecutive replicas per thread, RS_THREADS threads.
#ifndef PA_RS_ITEMS
#define PA_RS_ITEMS 8
#endif
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = PA_RS_ITEMS;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

}  // namespace pa
