// pa_resample.cu -- reweighting and resampling of the population (Sec. 2,
// Eq. 3 and Eq. 4) and the per-step observables (Sec. 2, Eq. 5).
//
//  k_tau       up to 16 CTAs: the energy histogram H of the population at beta_{i-1}
//              gives kref (lowest occupied level when cooling, highest when
//              heating), S = sum_k H_k D[|k - kref|] with D[j] =
//              exp(-|beta_i - beta_{i-1}| 4 j), Q = S exp(-dbeta E(kref)) / R
//              (Eq. 3) and the per-level weights tau_k = R0 D[|k - kref|] / S
//              (Eq. 4, renormalised to R0), kept as n_k = floor(tau_k),
//              F_k = floor(frac(tau_k) 2^32).
//  k_resample  one pass over the population, one tile of RS_TILE replicas per
//              CTA: copy counts r_j = n_k + [u_j < F_k] (nearest-integer rule),
//              a single-pass exclusive scan with decoupled lookback across
//              tiles, and the gather of r_j exact copies of replica j into slots
//              o_j .. o_j + r_j - 1 of the other population buffer.
//  k_obs       one CTA: exact integer sums over the histogram and the
//              magnetisation accumulators, then the FP64 averages.
//
// Floating point: IEEE double with explicit _rn intrinsics (no contraction),
// summed in a fixed order, so the tables are the same bits as any other
// implementation of the same order; log() only feeds ln Q, never a decision.
#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr unsigned long long DESC_AGG = 1ull;
constexpr unsigned long long DESC_PREFIX = 2ull;
constexpr unsigned LOOKBACK_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long desc_make(unsigned long long flag, uint32_t epoch,
                                                         uint32_t value) {
    return (flag << 62) | ((unsigned long long)(epoch & 0x3fffffffu) << 32) | value;
}

// The batched kernels stage a run's descriptor in shared memory (PA_RS_STAGE
// = 1): read from global memory, its fields could alias the kernel's own
// global stores, so the compiler would reload them after every store.
#ifndef PA_RS_STAGE
#define PA_RS_STAGE 1
#endif
static_assert(sizeof(RunDev) % 4 == 0, "RunDev is copied in 32-bit words");

// Copies *src into the shared descriptor dst with all threads of the CTA; the
// caller synchronises before reading it.
__device__ __forceinline__ void stage_run(const RunDev* src, RunDev& dst) {
    const uint32_t* from = reinterpret_cast<const uint32_t*>(src);
    uint32_t* to = reinterpret_cast<uint32_t*>(&dst);
    for (uint32_t w = threadIdx.x; w < sizeof(RunDev) / 4; w += blockDim.x) to[w] = from[w];
}

// Reweight of one run by nblk 256-thread CTAs (plain: k_tau, batched: one
// CTA per run of k_tau_batched).  Every CTA finds kref and S itself (the same
// fixed order, so the same bits) and writes the tau entries of its share of
// the levels; the last CTA to finish, when every CTA has read the step index
// and R, advances the run's scalars.
__device__ __forceinline__ void tau_run(const RunDev& d, uint32_t blk, uint32_t nblk) {
    DevState* st = d.st;
    __shared__ double part[256];
    __shared__ uint32_t s_kref;
    __shared__ unsigned long long s_sum;
    const int t = threadIdx.x;
    const uint32_t i = st->step + 1;
    const uint32_t R = st->R;
    const uint32_t bins = (uint32_t)d.bins;
    if (i > (uint32_t)d.K || R == 0) {
        if (t == 0) {
            st->active = 0;
            atomicOr(&st->status, i > (uint32_t)d.K ? ST_DONE : ST_EMPTY);
        }
        return;
    }
    // reference level: lowest occupied when cooling, highest when heating
    const bool heating = d.dbeta[i] < 0.0;
    if (t == 0) {
        s_kref = heating ? 0u : 0xffffffffu;
        s_sum = 0;
    }
    __syncthreads();
    uint32_t kext = heating ? 0u : 0xffffffffu;
    bool any = false;
    unsigned long long hs = 0;
    for (uint32_t k = t; k < bins; k += 256) {
        const uint32_t h = d.hist[k];
        if (h) {
            any = true;
            kext = heating ? (k > kext ? k : kext) : (k < kext ? k : kext);
        }
        hs += h;
    }
    if (heating) {
        if (any) atomicMax(&s_kref, kext);
    } else {
        atomicMin(&s_kref, kext);
    }
    atomicAdd(&s_sum, hs);
    __syncthreads();
    const uint32_t kref = s_kref;
    const double* D = d.dtab + (size_t)d.dsel[i] * bins;
    // S in the fixed order: 256 contiguous chunks summed left to right, then a
    // pairwise tree over the chunk sums; level k weighs D[|k - kref|].
    const uint32_t ch = (bins + 255) / 256;
    double acc = 0.0;
    for (uint32_t k = t * ch; k < (t + 1) * ch && k < bins; ++k) {
        const int64_t j = heating ? (int64_t)kref - (int64_t)k : (int64_t)k - (int64_t)kref;
        if (j >= 0) acc = __dadd_rn(acc, __dmul_rn((double)d.hist[k], D[j]));
    }
    part[t] = acc;
    __syncthreads();
    for (int w = 256; w > 1; w >>= 1) {
        double v = 0.0;
        if (t < w / 2) v = __dadd_rn(part[2 * t], part[2 * t + 1]);
        __syncthreads();
        if (t < w / 2) part[t] = v;
        __syncthreads();
    }
    const double S = part[0];
    const double R0d = (double)d.R0;
    for (uint32_t k = blk * 256u + t; k < bins; k += nblk * 256u) {
        uint32_t n = 0, F = 0;
        const int64_t j = heating ? (int64_t)kref - (int64_t)k : (int64_t)k - (int64_t)kref;
        if (j >= 0) {
            const double tau = __ddiv_rn(__dmul_rn(R0d, D[j]), S);
            const double nk = floor(tau);
            n = (uint32_t)nk;
            F = (uint32_t)floor(__dmul_rn(__dsub_rn(tau, nk), 4294967296.0));
        }
        d.tab_n[k] = n;
        d.tab_F[k] = F;
    }
    if (nblk > 1) {
        __shared__ bool s_last;
        __syncthreads();
        if (t == 0) {
            __threadfence();
            s_last = atomicAdd(&st->tau_done, 1ull) == (unsigned long long)(nblk - 1);
        }
        __syncthreads();
        if (!s_last) return;
    }
    if (t == 0) {
        st->tau_done = 0;
        if (s_sum != (unsigned long long)R) atomicOr(&st->status, ST_INVARIANT);
        const long long parity = st->negbonds & 1u;
        const long long Eref = 2 * (2 * (long long)kref + parity) - (long long)d.dim * d.N;
        const double lnQ =
            __dsub_rn(__dsub_rn(log(S), log((double)R)), __dmul_rn(d.dbeta[i], (double)Eref));
        st->lnQ = lnQ;
        st->lnZ = __dadd_rn(st->lnZ, lnQ);
        st->S = S;
        st->kref = kref;
        st->step = i;
        st->R_prev = R;
        st->epoch = st->epoch + 1;
        st->tile_counter = 0;
        st->src = st->cur;
        st->cur = st->cur ^ 1u;
        st->active = 1;
    }
}

__global__ void __launch_bounds__(256) k_tau(RunDev d) { tau_run(d, blockIdx.x, gridDim.x); }

// Batched reweight: CTA r handles run r, then clears that run's histogram and
// magnetisation sums for the coming sweep (the reweight is their last
// reader); CTA 0 clears the batch's work counters.
__global__ void __launch_bounds__(256) k_tau_batched(BatchDev b) {
    if (blockIdx.x == 0 && threadIdx.x < b.ncounters) b.counters[threadIdx.x] = 0u;
#if PA_RS_STAGE
    __shared__ RunDev s_d;
    stage_run(&b.runs[blockIdx.x], s_d);
    __syncthreads();
    const RunDev& d = s_d;
#else
    const RunDev& d = b.runs[blockIdx.x];
#endif
    tau_run(d, 0, 1);
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < (uint32_t)d.bins; k += blockDim.x) d.hist[k] = 0u;
    if (threadIdx.x < 2) d.accum[threadIdx.x] = 0ull;
}

// PA_RS_COMPACT = 1: the gather walks only the tile's surviving replicas
// (count > 0), listed in order in shared memory, so that every 16-byte item a
// thread takes has a load behind it; 0 walks every replica of the tile.
#ifndef PA_RS_COMPACT
#define PA_RS_COMPACT 1
#endif

struct ResampleSmem {
    uint32_t r[RS_TILE];
    uint32_t o[RS_TILE];
#if PA_RS_COMPACT
    uint32_t surv[RS_TILE];             // tile indices of the surviving replicas
    uint32_t warp_nz[RS_THREADS / 32];  // survivors before each warp
    uint32_t nsurv;
#endif
    uint32_t warp[RS_THREADS / 32];
    uint32_t tile, excl;
};

// 16-byte loads in flight per thread in the gather.  Measured on GB300 at 2^21
// replicas, L = 64 (one-kernel form, same bits): 4 -> 0.368 ms, 5 -> 0.361
// ms, 6 -> 0.361 ms, 8 with 3 CTAs per SM -> 0.400 ms.
#ifndef PA_RS_GU
#define PA_RS_GU 6
#endif

// Counts, scan and gather of tile `tile` of one run (all threads of the CTA).
// Poisson(tau_k) copy count of replica i (Sec. 2), tau_k = n + F / 2^32: the
// event count of a unit-rate Poisson process on [0, tau_k].  The fractional
// interval contributes a Poisson(1) count thinned with keep probability
// F / 2^32, each unit interval a Poisson(1) count, every one drawn by
// inversion against the 32-bit thresholds p1.  Uniforms: words of the Philox
// blocks (i, step, b, POISSON|id), b = 0, 1, ..., consumed in that order.
// A level with n above the capacity overflows whatever the draw: its count is
// then n itself, which the capacity check rejects, instead of n draws.
__device__ __noinline__ uint32_t poisson_count(const RunDev& d, uint32_t i, uint32_t step,
                                               uint32_t n, uint32_t F) {
    if (n > d.cap) return n;
    const uint32_t ctr3 = (TAG_POISSON << 28) | d.instance;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    uint4 blk = philox(i, step, 0u, ctr3, k0, k1);
    uint32_t b = 1, w = 0;
    auto next = [&]() -> uint32_t {
        if (w == 4) {
            blk = philox(i, step, b, ctr3, k0, k1);
            ++b;
            w = 0;
        }
        return pick(blk, w++);
    };
    auto unit = [&]() -> uint32_t {
        const uint32_t u = next();
        uint32_t m = 0;
        while (m < d.p1_len && u >= d.p1[m]) ++m;
        return m;
    };
    uint32_t count = 0;
    const uint32_t events = unit();
    for (uint32_t e = 0; e < events; ++e) count += next() < F ? 1u : 0u;
    for (uint32_t j = 0; j < n; ++j) count += unit();
    return count;
}

// RULE 0 compiles the nearest-integer rule alone (the register budget of the
// HBM-bound default path); 1 adds the per-run Poisson branch; 2 takes the
// counts that the multinomial draw has left in d.counts; 3 chooses among the
// three per run (batches that mix the rules).
//
// SPLIT = false: the tile also gathers its replicas' spins (the batched form).
// SPLIT = true: the tile writes, for each slot it fills, the index of the
// source replica (srcmap) with the copied energy level and magnetisation, and
// k_gather copies the spins afterwards over the whole new population (the
// plain form).
template <int RULE, bool SPLIT = false>
__device__ __forceinline__ void resample_tile(const RunDev& d, uint32_t tile, ResampleSmem& sm) {
    DevState* st = d.st;
    uint32_t* s_r = sm.r;
    uint32_t* s_o = sm.o;
    uint32_t* s_warp = sm.warp;
    uint32_t& s_excl = sm.excl;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t R = st->R_prev, epoch = st->epoch, src = st->src, step = st->step;
    const uint32_t base = tile * RS_TILE;
    if (base >= R) return;
    const uint32_t n_in = min((uint32_t)RS_TILE, R - base);

    // copy counts, RS_ITEMS consecutive replicas per thread
    const uint32_t* eb = d.ebin[src];
    const uint32_t ctr3 = (TAG_RESAMPLE << 28) | d.instance;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    uint32_t r[RS_ITEMS];
    uint32_t sum = 0;
    if (RULE == 2 || (RULE == 3 && d.resample == PA_RESAMPLE_MULTINOMIAL)) {
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) {
            const uint32_t i = base + (uint32_t)t * RS_ITEMS + j;
            const uint32_t v = i < R ? d.counts[i] : 0u;
            r[j] = v;
            sum += v;
        }
    } else if ((RULE == 1 || RULE == 3) && d.resample == PA_RESAMPLE_POISSON) {
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) {
            const uint32_t i = base + (uint32_t)t * RS_ITEMS + j;
            uint32_t v = 0;
            if (i < R) {
                const uint32_t k = eb[i];
                v = poisson_count(d, i, step, d.tab_n[k], d.tab_F[k]);
            }
            r[j] = v;
            sum += v;
        }
    } else
#pragma unroll
    for (int j0 = 0; j0 < RS_ITEMS; j0 += 4) {
        const uint32_t i0 = base + (uint32_t)t * RS_ITEMS + j0;
        uint4 u = make_uint4(0, 0, 0, 0);
        if (i0 < R) u = philox(i0 >> 2, step, 0u, ctr3, k0, k1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t i = i0 + j;
            uint32_t v = 0;
            if (i < R) {
                const uint32_t k = eb[i];
                v = d.tab_n[k] + (pick(u, (uint32_t)j) < d.tab_F[k] ? 1u : 0u);
            }
            r[j0 + j] = v;
            sum += v;
        }
    }
    // block-wide exclusive scan of the per-thread sums
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
#if PA_RS_COMPACT
    // and of the per-thread survivor counts
    uint32_t nz = 0;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) nz += r[j] ? 1u : 0u;
    uint32_t nzi = nz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, nzi, o);
        if (lane >= o) nzi += y;
    }
    if (lane == 31) sm.warp_nz[wid] = nzi;
#endif
    __syncthreads();
#if PA_RS_COMPACT
    if (wid == 1) {
        const uint32_t w = lane < RS_THREADS / 32 ? sm.warp_nz[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < RS_THREADS / 32) sm.warp_nz[lane] = wi - w;
        if (lane == RS_THREADS / 32 - 1) sm.nsurv = wi;
    }
#endif
    if (wid == 0) {
        uint32_t w = lane < RS_THREADS / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < RS_THREADS / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
        const uint32_t total = __shfl_sync(0xffffffffu, wi, RS_THREADS / 32 - 1);
        // decoupled lookback across tiles (one thread)
        if (lane == 0) {
            uint32_t excl = 0;
            if (tile == 0) {
                // the test hook withholds tile 0's prefix, so that tile 1's
                // bounded wait runs out (PA_DEBUG_WITHHOLD_PREFIX)
                if (!(d.debug & PA_DEBUG_WITHHOLD_PREFIX))
                    st_release(&d.desc[0], desc_make(DESC_PREFIX, epoch, total));
            } else {
                st_release(&d.desc[tile], desc_make(DESC_AGG, epoch, total));
                int p = (int)tile - 1;
                for (;;) {
                    unsigned long long v = 0;
                    unsigned spins = 0;
                    bool ok = false;
                    for (;;) {
                        v = ld_acquire(&d.desc[p]);
                        if ((v >> 62) != 0 && ((v >> 32) & 0x3fffffffu) == (epoch & 0x3fffffffu)) {
                            ok = true;
                            break;
                        }
                        if (++spins >= LOOKBACK_SPIN_LIMIT) break;
                        if (spins > 64) __nanosleep(64);
                    }
                    if (!ok) {
                        atomicOr(&st->status, ST_TIMEOUT);
                        break;
                    }
                    excl += (uint32_t)(v & 0xffffffffu);
                    if ((v >> 62) == DESC_PREFIX || p == 0) break;
                    --p;
                }
                st_release(&d.desc[tile], desc_make(DESC_PREFIX, epoch, excl + total));
            }
            s_excl = excl;
        }
    }
    __syncthreads();
    uint32_t o = s_excl + s_warp[wid] + (incl - sum);
#if PA_RS_COMPACT
    uint32_t p = sm.warp_nz[wid] + (nzi - nz);
#endif
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const uint32_t li = (uint32_t)t * RS_ITEMS + j;
        const uint32_t i = base + li;
#if PA_RS_COMPACT
        if (r[j]) sm.surv[p++] = li;  // r[j] = 0 beyond R
#endif
        if (i < R) {
            s_r[li] = r[j];
            s_o[li] = o;
            d.counts[i] = r[j];
            d.offsets[i] = o;
            if (i == R - 1) {
                const uint32_t Rnew = o + r[j];
                if (Rnew > d.cap) atomicOr(&st->status, ST_CAPACITY);
                if (Rnew == 0) atomicOr(&st->status, ST_EMPTY);
                st->R = Rnew > d.cap ? d.cap : Rnew;
            }
        }
        o += r[j];
    }
    __syncthreads();
#if PA_RS_COMPACT
    if (t == 0) atomicAdd(&st->sources, (unsigned long long)sm.nsurv);
#endif

#if PA_RS_COMPACT
    const uint32_t nlist = sm.nsurv;  // gather item j of the list: replica surv[j]
#else
    const uint32_t nlist = n_in;
#endif
    // gather: 16-byte chunks, consecutive threads on consecutive chunks; GU
    // independent loads in flight per thread before their stores
    if (!SPLIT) {
    constexpr int GU = PA_RS_GU;
    const uint32_t CH = d.stride >> 4;
    const uint4* __restrict__ srcp = reinterpret_cast<const uint4*>(d.spins[src]) + (size_t)base * CH;
    uint4* __restrict__ dstp = reinterpret_cast<uint4*>(d.spins[src ^ 1u]);
    const uint32_t items = nlist * CH;
    const bool pow2 = (CH & (CH - 1)) == 0;
    const int shift = __ffs(CH) - 1;
    for (uint32_t it0 = t; it0 < items; it0 += RS_THREADS * GU) {
        uint4 v[GU];
        uint32_t rr[GU], d0[GU], cc[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const uint32_t it = it0 + (uint32_t)u * RS_THREADS;
            rr[u] = 0;
            if (it < items) {
                const uint32_t jl = pow2 ? (it >> shift) : (it / CH);
                cc[u] = it - jl * CH;
#if PA_RS_COMPACT
                const uint32_t li = sm.surv[jl];
#else
                const uint32_t li = jl;
#endif
                rr[u] = s_r[li];
                d0[u] = s_o[li];
                if (rr[u]) v[u] = __ldg(srcp + (size_t)li * CH + cc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            for (uint32_t k = 0; k < rr[u]; ++k) {
                const uint32_t dst = d0[u] + k;
                if (dst < d.cap) __stcs(dstp + (size_t)dst * CH + cc[u], v[u]);
            }
        }
    }
    }
    const uint32_t* esrc = d.ebin[src] + base;
    const int32_t* msrc = d.mag[src] + base;
    uint32_t* edst = d.ebin[src ^ 1u];
    int32_t* mdst = d.mag[src ^ 1u];
    for (uint32_t jl = t; jl < nlist; jl += RS_THREADS) {
#if PA_RS_COMPACT
        const uint32_t li = sm.surv[jl];
#else
        const uint32_t li = jl;
#endif
        const uint32_t rr = s_r[li];
        if (rr == 0) continue;
        const uint32_t e = esrc[li];
        const int32_t m = msrc[li];
        for (uint32_t k = 0; k < rr; ++k) {
            const uint32_t dst = s_o[li] + k;
            if (dst < d.cap) {
                edst[dst] = e;
                mdst[dst] = m;
                if (SPLIT) d.srcmap[dst] = base + li;
            }
        }
    }
}

// Persistent: one wave of CTAs, each claiming tiles until none is left.
// Claims come in increasing order, so a tile's lookback only waits on tiles
// already claimed by running CTAs.
// Resident CTAs per SM the register budget of the nearest-integer and
// counts-from-memory rules is sized for (the Poisson rule takes 2).
#ifndef PA_RS_MINB
#define PA_RS_MINB 4
#endif
template <int RULE, bool SPLIT>
__global__ void __launch_bounds__(RS_THREADS, RULE == 1 ? 2 : PA_RS_MINB) k_resample(RunDev d) {
    __shared__ ResampleSmem sm;
    if (!d.st->active) return;
    const uint32_t R = d.st->R_prev;
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(&d.st->tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = sm.tile;
        if (tile * (uint32_t)RS_TILE >= R) break;
        resample_tile<RULE, SPLIT>(d, tile, sm);
        __syncthreads();  // sm is reused by the next tile
    }
}

// Gather of the new population (the plain form's second kernel): slot j of
// the other buffer receives the spins of replica srcmap[j], for every slot j <
// R_i, in 16-byte chunks.  Work item t is chunk t % CH of slot t / CH, so the
// stores of consecutive threads are consecutive and the loads of one slot's
// chunks are one contiguous source replica; a source with r copies is read
// by r neighbouring slots at nearly the same time, so its later reads hit
// L2.  Every thread keeps GA_U loads in flight: the map words first, then the
// data they point to, then the streaming stores.  Persistent: one wave of
// resident CTAs strides over all R_i * CH chunks.
#ifndef PA_GA_U
#define PA_GA_U 8
#endif
#ifndef PA_GA_MINB
#define PA_GA_MINB 3
#endif
constexpr int GA_THREADS = 256;
constexpr int GA_U = PA_GA_U;

// EM = true (the redistribution's gather) also copies every slot's energy
// level and magnetisation from the source replica.
template <bool EM>
__global__ void __launch_bounds__(GA_THREADS, PA_GA_MINB) k_gather(RunDev d) {
    const DevState* st = d.st;
    if (!st->active) return;
    const uint32_t Rn = st->R;  // clamped to the capacity by the scan
    const uint32_t src = st->src;
    const uint32_t CH = d.stride >> 4;
    const uint32_t last = d.cap_alloc - 1;
    const uint4* __restrict__ sp = reinterpret_cast<const uint4*>(d.spins[src]);
    uint4* __restrict__ dp = reinterpret_cast<uint4*>(d.spins[src ^ 1u]);
    const uint32_t* __restrict__ map = d.srcmap;
    if ((CH & 31u) == 0) {
        // a replica is a whole number of warp rows (L = 64: one 512-byte row
        // of 32 chunks): each warp takes groups of 32 consecutive slots, reads
        // their 32 map words in one coalesced load, and then copies GA_U
        // replicas at a time, lane l moving chunks l, l + 32, ... of each
        const uint32_t lane = threadIdx.x & 31u;
        const uint32_t rows = CH >> 5;
        const uint32_t nwarps = gridDim.x * (GA_THREADS / 32);
        for (uint32_t g = blockIdx.x * (GA_THREADS / 32) + (threadIdx.x >> 5); g * 32u < Rn;
             g += nwarps) {
            const uint32_t slot0 = g * 32u;
            const uint32_t nslot = min(32u, Rn - slot0);
            const uint32_t mine = lane < nslot ? min(__ldg(map + slot0 + lane), last) : 0u;
            for (uint32_t row = 0; row < rows; ++row) {
                const uint32_t c = row * 32u + lane;
                for (uint32_t k0 = 0; k0 < nslot; k0 += GA_U) {
                    uint4 v[GA_U];
#pragma unroll
                    for (int u = 0; u < GA_U; ++u) {
                        const uint32_t sidx = __shfl_sync(0xffffffffu, mine, (k0 + u) & 31u);
                        if (k0 + u < nslot) v[u] = __ldg(sp + (size_t)sidx * CH + c);
                    }
#pragma unroll
                    for (int u = 0; u < GA_U; ++u)
                        if (k0 + u < nslot) __stcs(dp + (size_t)(slot0 + k0 + u) * CH + c, v[u]);
                }
            }
        }
    } else {
        const unsigned long long items = (unsigned long long)Rn * CH;
        const unsigned long long nth = (unsigned long long)gridDim.x * GA_THREADS;
        const bool pow2 = (CH & (CH - 1)) == 0;
        const int shift = __ffs(CH) - 1;
        for (unsigned long long it0 = (unsigned long long)blockIdx.x * GA_THREADS + threadIdx.x;
             it0 < items; it0 += nth * GA_U) {
            uint32_t sidx[GA_U], c[GA_U];
#pragma unroll
            for (int u = 0; u < GA_U; ++u) {
                const unsigned long long it = it0 + (unsigned long long)u * nth;
                sidx[u] = 0;
                c[u] = 0;
                if (it < items) {
                    const uint32_t slot = pow2 ? (uint32_t)(it >> shift) : (uint32_t)(it / CH);
                    c[u] = (uint32_t)(it - (unsigned long long)slot * CH);
                    sidx[u] = min(__ldg(map + slot), last);  // a slot never holds more than cap_alloc
                }
            }
            uint4 v[GA_U];
#pragma unroll
            for (int u = 0; u < GA_U; ++u) {
                const unsigned long long it = it0 + (unsigned long long)u * nth;
                if (it < items) v[u] = __ldg(sp + (size_t)sidx[u] * CH + c[u]);
            }
#pragma unroll
            for (int u = 0; u < GA_U; ++u) {
                const unsigned long long it = it0 + (unsigned long long)u * nth;
                if (it < items) __stcs(dp + it, v[u]);
            }
        }
    }
    if (EM) {
        const uint32_t* es = d.ebin[src];
        const int32_t* ms = d.mag[src];
        uint32_t* ed = d.ebin[src ^ 1u];
        int32_t* md = d.mag[src ^ 1u];
        for (uint32_t j = blockIdx.x * GA_THREADS + threadIdx.x; j < Rn; j += gridDim.x * GA_THREADS) {
            const uint32_t i = min(map[j], last);
            ed[j] = es[i];
            md[j] = ms[i];
        }
    }
}

// Slot permutation of a redistribution: post-exchange slot j in segment q
// (dst[q] <= j < dst[q+1]) takes the source of pre-exchange slot
// src[q] + j - dst[q].
__global__ void __launch_bounds__(256) k_remap(RunDev d, const __grid_constant__ SegList segs) {
    const DevState* st = d.st;
    if (!st->active) return;
    const uint32_t Rn = st->R;
    const uint32_t last = d.cap_alloc - 1;
    for (uint32_t j = blockIdx.x * 256 + threadIdx.x; j < Rn; j += gridDim.x * 256) {
        uint32_t lo = 0, hi = segs.n;  // dst[lo] <= j < dst[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (segs.dst[mid] <= j) lo = mid;
            else hi = mid;
        }
        const uint32_t pre = min(segs.src[lo] + (j - segs.dst[lo]), last);
        d.srcmap2[j] = d.srcmap[pre];
    }
}

// Batched: global tile ids are claimed in increasing order; run r owns ids
// tile_base[r] .. tile_base[r+1]-1, so within a run tiles are claimed in order
// and the lookback only ever waits on tiles already running.
template <int RULE>
__global__ void __launch_bounds__(RS_THREADS) k_resample_batched(BatchDev b) {
    __shared__ ResampleSmem sm;
    __shared__ uint32_t s_run;
#if PA_RS_STAGE
    __shared__ RunDev s_d;
    uint32_t have = 0xffffffffu;
#endif
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t g = atomicAdd(&b.counters[0], 1u);
            if (g >= b.total_tiles) {
                s_run = 0xffffffffu;
            } else {
                uint32_t lo = 0, hi = b.nruns;  // tile_base[lo] <= g < tile_base[hi]
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (b.tile_base[mid] <= g) lo = mid;
                    else hi = mid;
                }
                s_run = lo;
                sm.tile = g - b.tile_base[lo];
            }
        }
        __syncthreads();
        if (s_run == 0xffffffffu) break;
#if PA_RS_STAGE
        if (s_run != have) {
            stage_run(&b.runs[s_run], s_d);
            have = s_run;
            __syncthreads();
        }
        const RunDev& d = s_d;
#else
        const RunDev& d = b.runs[s_run];
#endif
        if (d.st->active) resample_tile<RULE>(d, sm.tile, sm);
        __syncthreads();
    }
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void obs_run(const RunDev& d, int nsweeps) {
    DevState* st = d.st;
    __shared__ long long s_part[3][8];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t step = st->step;
    const long long parity = st->negbonds & 1u;
    const long long dimN = (long long)d.dim * d.N;
    long long cnt = 0, sE = 0, sE2 = 0;
    for (uint32_t k = t; k < (uint32_t)d.bins; k += 256) {
        const long long h = d.hist[k];
        if (!h) continue;
        const long long E = 2 * (2 * (long long)k + parity) - dimN;
        cnt += h;
        sE += h * E;
        sE2 += h * E * E;
    }
    cnt = warp_sum_ll(cnt);
    sE = warp_sum_ll(sE);
    sE2 = warp_sum_ll(sE2);
    if (lane == 0) {
        s_part[0][wid] = cnt;
        s_part[1][wid] = sE;
        s_part[2][wid] = sE2;
    }
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < 8; ++w) {
            cnt += s_part[0][w];
            sE += s_part[1][w];
            sE2 += s_part[2][w];
        }
        const uint32_t R = st->R;
        if (cnt != (long long)R) atomicOr(&st->status, ST_INVARIANT);
        pa_obs o;
        o.step = step;
        o.R = R;
        o.sumE = sE;
        o.sumE2 = sE2;
        o.sumAbsM = (long long)d.accum[0];
        o.sumM2 = (long long)d.accum[1];
        o.beta = d.beta[step];
        o.lnQ = st->lnQ;
        o.lnZ = st->lnZ;
        const double Rd = (double)R, Nd = (double)d.N;
        const double mE = __ddiv_rn((double)o.sumE, Rd);
        const double mE2 = __ddiv_rn((double)o.sumE2, Rd);
        const double mA = __ddiv_rn((double)o.sumAbsM, Rd);
        const double mM2 = __ddiv_rn((double)o.sumM2, Rd);
        o.e = __ddiv_rn(mE, Nd);
        o.cv = __ddiv_rn(__dmul_rn(__dmul_rn(o.beta, o.beta), __dsub_rn(mE2, __dmul_rn(mE, mE))), Nd);
        o.m_abs = __ddiv_rn(mA, Nd);
        o.chi = __ddiv_rn(__dmul_rn(o.beta, __dsub_rn(mM2, __dmul_rn(mA, mA))), Nd);
        d.obs[step] = o;
        st->sweep_base = st->sweep_base + (uint32_t)nsweeps;
        st->sweeps_done = st->sweeps_done + (unsigned long long)nsweeps;
    }
}

__global__ void __launch_bounds__(256) k_obs(RunDev d, int nsweeps) { obs_run(d, nsweeps); }

__global__ void __launch_bounds__(256) k_obs_batched(BatchDev b) {
#if PA_RS_STAGE
    __shared__ RunDev s_d;
    stage_run(&b.runs[blockIdx.x], s_d);
    __syncthreads();
    const RunDev& d = s_d;
#else
    const RunDev& d = b.runs[blockIdx.x];
#endif
    obs_run(d, d.theta);
}

}  // namespace

// CTAs of the plain reweight: one per 256 levels, at most 16 (the tau
// divisions are FP64; each CTA also repeats the sum S, 16 FP64 terms a thread).
cudaError_t launch_tau(const RunDev& d, cudaStream_t s) {
    const int64_t per = ((int64_t)d.bins + 255) / 256;
    const int grid = (int)(per < 16 ? per : 16);
    k_tau<<<grid < 1 ? 1 : grid, 256, 0, s>>>(d);
    return cudaGetLastError();
}

// One wave of resident CTAs (capped by the number of tiles), looked up once
// per device and kernel.
static int resample_wave(const void* fn, int which, uint32_t tiles) {
    static int cache[64][10];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int wave = cache[dev][which];
    if (wave <= 0) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RS_THREADS, 0) != cudaSuccess)
            return 0;
        wave = sms * (per_sm < 1 ? 1 : per_sm);
        cache[dev][which] = wave;
    }
    return (int)((int64_t)tiles < wave ? (int64_t)tiles : wave);
}

// PA_RS_SPLIT = 1: the plain resample is two kernels, counts + scan (with the
// slot -> source map, levels and magnetisations) and then k_gather over the
// whole new population; 0 (the default): one kernel that gathers tile by
// tile.  Measured on GB300 at 2^21 replicas, L = 64, same bits: one kernel
// 0.366 ms with 4 loads in flight per thread in its gather (0.361 ms with 6,
// the default); two kernels 0.374 ms (16 loads in flight per thread, 2 CTAs of
// 256 per SM), 0.380 ms (4 loads, 4 CTAs), 0.385 ms (8 loads, 3 CTAs).  The split
// form serves the redistribution's gather (pa_resample_finish), whose slot
// order is only known after the host has read the scan.
#ifndef PA_RS_SPLIT
#define PA_RS_SPLIT 0
#endif
constexpr bool RS_SPLIT = PA_RS_SPLIT != 0;

static int gather_grid() {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cache[dev] <= 0) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_gather<false>,
                                                          GA_THREADS, 0) != cudaSuccess)
            return 0;
        cache[dev] = sms * (per_sm < 1 ? 1 : per_sm);
    }
    return cache[dev];
}

template <bool SPLIT>
static cudaError_t launch_counts_scan(const RunDev& d, cudaStream_t s) {
    // cache slots: 0/2/4 the one-kernel forms, 7/8/9 the split forms
    const int slot = SPLIT ? 7 : 0;
    if (d.resample == PA_RESAMPLE_POISSON) {
        const int grid = resample_wave((const void*)k_resample<1, SPLIT>, SPLIT ? 8 : 2, d.tiles);
        if (grid <= 0) return cudaErrorInvalidValue;
        k_resample<1, SPLIT><<<grid, RS_THREADS, 0, s>>>(d);
    } else if (d.resample == PA_RESAMPLE_MULTINOMIAL) {
        const int grid = resample_wave((const void*)k_resample<2, SPLIT>, SPLIT ? 9 : 4, d.tiles);
        if (grid <= 0) return cudaErrorInvalidValue;
        k_resample<2, SPLIT><<<grid, RS_THREADS, 0, s>>>(d);
    } else {
        const int grid = resample_wave((const void*)k_resample<0, SPLIT>, slot, d.tiles);
        if (grid <= 0) return cudaErrorInvalidValue;
        k_resample<0, SPLIT><<<grid, RS_THREADS, 0, s>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_resample(const RunDev& d, cudaStream_t s) {
    cudaError_t e = launch_counts_scan<RS_SPLIT>(d, s);
    if (e != cudaSuccess || !RS_SPLIT) return e;
    const int g = gather_grid();
    if (g <= 0) return cudaErrorInvalidValue;
    k_gather<false><<<g, GA_THREADS, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_resample_scan(const RunDev& d, cudaStream_t s) {
    return launch_counts_scan<true>(d, s);
}

cudaError_t launch_remap_gather(const RunDev& d, const SegList& segs, cudaStream_t s) {
    const int g = gather_grid();
    if (g <= 0) return cudaErrorInvalidValue;
    k_remap<<<g, 256, 0, s>>>(d, segs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RunDev dm = d;
    dm.srcmap = d.srcmap2;
    k_gather<true><<<g, GA_THREADS, 0, s>>>(dm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Multinomial resampling: the copy counts of all replicas come from R0
// independent draws.  Replica i weighs t_i = n_k 2^32 + F_k (k = its level);
// C_i = t_0 + ... + t_i are exact 64-bit integers, built by a three-pass scan
// over tiles of RS_TILE replicas (tile sums, one-CTA scan of the tile sums,
// per-tile prefix).  Draw j: v = words 2(j & 1) (low) and 2(j & 1) + 1 (high)
// of Philox block (j >> 1, step, 0, MULTINOMIAL|id), x = floor(v C_{R-1} /
// 2^64), one copy (atomic add) to the first replica with C_i > x.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mn_weight(const RunDev& d, uint32_t k) {
    return ((unsigned long long)d.tab_n[k] << 32) + (unsigned long long)d.tab_F[k];
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sw) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sw[wid] = v;
    __syncthreads();
    unsigned long long tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sw[w];
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(RS_THREADS) k_mn_tile_sums(RunDev d) {
    __shared__ unsigned long long sw[RS_THREADS / 32];
    const DevState* st = d.st;
    if (!st->active) return;
    const uint32_t R = st->R_prev, src = st->src;
    const uint32_t ntiles = (R + RS_TILE - 1) / RS_TILE;
    const uint32_t* eb = d.ebin[src];
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        unsigned long long part = 0;
        for (uint32_t j = threadIdx.x; j < (uint32_t)RS_TILE; j += RS_THREADS) {
            const uint32_t i = tile * RS_TILE + j;
            if (i < R) part += mn_weight(d, eb[i]);
        }
        const unsigned long long tot = block_sum_u64(part, sw);
        if (threadIdx.x == 0) d.mn_tiles[tile] = tot;
    }
}

// Exclusive scan of the tile sums in place; mn_tiles[ntiles] = the total.
__global__ void __launch_bounds__(1024) k_mn_scan(RunDev d) {
    __shared__ unsigned long long s[1024];
    const DevState* st = d.st;
    if (!st->active) return;
    const uint32_t R = st->R_prev;
    const uint32_t ntiles = (R + RS_TILE - 1) / RS_TILE;
    const uint32_t t = threadIdx.x;
    const uint32_t per = (ntiles + 1023) / 1024;
    const uint32_t lo = t * per, hi = min(ntiles, lo + per);
    unsigned long long part = 0;
    for (uint32_t k = lo; k < hi; ++k) part += d.mn_tiles[k];
    s[t] = part;
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
        const unsigned long long v = t >= o ? s[t - o] : 0ull;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    unsigned long long run = s[t] - part;
    for (uint32_t k = lo; k < hi; ++k) {
        const unsigned long long v = d.mn_tiles[k];
        d.mn_tiles[k] = run;
        run += v;
    }
    if (t == 1023) d.mn_tiles[ntiles] = s[1023];
}

// C_i per replica (inclusive), and the copy counts cleared for the draws.
__global__ void __launch_bounds__(RS_THREADS) k_mn_cum(RunDev d) {
    __shared__ unsigned long long sw[RS_THREADS / 32];
    const DevState* st = d.st;
    if (!st->active) return;
    const uint32_t R = st->R_prev, src = st->src;
    const uint32_t ntiles = (R + RS_TILE - 1) / RS_TILE;
    const uint32_t* eb = d.ebin[src];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i0 = tile * RS_TILE + threadIdx.x * RS_ITEMS;
        unsigned long long w[RS_ITEMS], part = 0;
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) {
            w[j] = i0 + j < R ? mn_weight(d, eb[i0 + j]) : 0ull;
            part += w[j];
        }
        unsigned long long incl = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) sw[wid] = incl;
        __syncthreads();
        unsigned long long before = d.mn_tiles[tile];
        for (int k = 0; k < wid; ++k) before += sw[k];
        unsigned long long run = before + incl - part;
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) {
            if (i0 + j < R) {
                run += w[j];
                d.mn_cum[i0 + j] = run;
                d.counts[i0 + j] = 0u;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_mn_draw(RunDev d) {
    const DevState* st = d.st;
    if (!st->active) return;
    const uint32_t R = st->R_prev, step = st->step;
    const uint32_t ntiles = (R + RS_TILE - 1) / RS_TILE;
    const unsigned long long total = d.mn_tiles[ntiles];
    if (total == 0ull) return;
    const uint32_t ctr3 = (TAG_MULTINOMIAL << 28) | d.instance;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    const uint32_t pairs = (d.R0 + 1u) / 2u;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < pairs;
         p += gridDim.x * blockDim.x) {
        const uint4 u = philox(p, step, 0u, ctr3, k0, k1);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t j = 2u * p + (uint32_t)e;
            if (j >= d.R0) break;
            const unsigned long long v = e == 0 ? (((unsigned long long)u.y << 32) | u.x)
                                                : (((unsigned long long)u.w << 32) | u.z);
            const unsigned long long x = __umul64hi(v, total);
            uint32_t lo = 0, hi = R - 1;  // first i with C_i > x
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if (d.mn_cum[mid] > x) hi = mid;
                else lo = mid + 1;
            }
            atomicAdd(&d.counts[lo], 1u);
        }
    }
}

cudaError_t launch_multinomial(const RunDev& d, cudaStream_t s) {
    if (!d.mn_cum || !d.mn_tiles) return cudaErrorInvalidValue;
    const int wave = resample_wave((const void*)k_mn_cum, 5, d.tiles);
    if (wave <= 0) return cudaErrorInvalidValue;
    k_mn_tile_sums<<<wave, RS_THREADS, 0, s>>>(d);
    k_mn_scan<<<1, 1024, 0, s>>>(d);
    k_mn_cum<<<wave, RS_THREADS, 0, s>>>(d);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidValue;
    const uint32_t pairs = (d.R0 + 1u) / 2u;
    const uint32_t want = (pairs + 255u) / 256u;
    const uint32_t cap = (uint32_t)sms * 8u;
    k_mn_draw<<<want < cap ? (want ? want : 1u) : cap, 256, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_obs(const RunDev& d, int nsweeps, cudaStream_t s) {
    k_obs<<<1, 256, 0, s>>>(d, nsweeps);
    return cudaGetLastError();
}

cudaError_t launch_tau_batched(const BatchDev& b, cudaStream_t s) {
    k_tau_batched<<<b.nruns, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_resample_batched(const BatchDev& b, cudaStream_t s) {
    if (b.any_multinomial) {
        const int grid = resample_wave((const void*)k_resample_batched<3>, 6, b.total_tiles);
        if (grid <= 0) return cudaErrorInvalidValue;
        k_resample_batched<3><<<grid, RS_THREADS, 0, s>>>(b);
    } else if (b.any_poisson) {
        const int grid = resample_wave((const void*)k_resample_batched<1>, 3, b.total_tiles);
        if (grid <= 0) return cudaErrorInvalidValue;
        k_resample_batched<1><<<grid, RS_THREADS, 0, s>>>(b);
    } else {
        const int grid = resample_wave((const void*)k_resample_batched<0>, 1, b.total_tiles);
        if (grid <= 0) return cudaErrorInvalidValue;
        k_resample_batched<0><<<grid, RS_THREADS, 0, s>>>(b);
    }
    return cudaGetLastError();
}

cudaError_t launch_obs_batched(const BatchDev& b, cudaStream_t s) {
    k_obs_batched<<<b.nruns, 256, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace pa
