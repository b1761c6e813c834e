// pa_static_scan.cu -- copy counts and their exclusive scan without any
// device allocation (pa_copy_counts_scan_noalloc in include/pa.h).
//
// Some callers cannot allocate device memory at all, not even through a
// caller-side allocator: code that runs while a CUDA graph is being captured,
// plugins whose host process owns every allocation, and embedded callers with
// a fixed memory budget.  For them this entry point computes the
// nearest-integer copy counts and their exclusive scan from buffers the
// caller already has, and keeps the only scratch it needs (the lookback
// descriptors of the single-pass scan, a tile counter and a call counter) in
// the file-scope array below.  That array is part of the library's image:
// every GPU that loads the library holds it until the process exits.
#include <mutex>

#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr int SS_THREADS = 256;
constexpr int SS_ITEMS = 8;
constexpr int SS_TILE = SS_THREADS * SS_ITEMS;  // replicas per tile
constexpr int SS_MAX_TILES = PA_NOALLOC_MAX_REPLICAS / SS_TILE;
static_assert(SS_MAX_TILES * SS_TILE == PA_NOALLOC_MAX_REPLICAS, "whole tiles");
constexpr unsigned SS_SPIN_LIMIT = 1u << 22;

struct StaticScanScratch {
    unsigned long long desc[SS_MAX_TILES];  // (flag << 62) | (epoch << 32) | value
    uint32_t tile_counter;                  // dynamic tile ids, cleared per call
    uint32_t epoch;                         // bumped per call; tags the descriptors
    uint32_t status;                        // bit 0: bad energy level, bit 1: wait gave up
    uint32_t pad[61];
};

// The scratch.  Zero at load time; shared by every call in the process.
static __device__ __align__(256) StaticScanScratch g_scan_scratch;

// Clears the scratch a call reads before writing it: the tile counter, the
// status bits and the descriptors of the call's tiles.  With every descriptor
// cleared, a value left by an earlier call can never be taken as ready, even
// once the 30-bit epoch tag has wrapped.
__global__ void k_static_prepare(StaticScanScratch* s, uint32_t tiles, uint32_t* total) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < tiles;
         i += gridDim.x * blockDim.x)
        s->desc[i] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->tile_counter = 0;
        s->epoch = s->epoch + 1;
        s->status = 0;
        *total = 0;
    }
}

__device__ __forceinline__ void ss_store(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ss_load(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(SS_THREADS)
    k_static_counts_scan(StaticScanScratch* s, const uint32_t* __restrict__ ebin, uint32_t R,
                         const uint32_t* __restrict__ tab_n, const uint32_t* __restrict__ tab_F,
                         uint32_t bins, uint32_t step, uint32_t ctr3, uint32_t k0, uint32_t k1,
                         uint32_t* __restrict__ counts, uint32_t* __restrict__ offsets,
                         uint32_t* __restrict__ total) {
    __shared__ uint32_t s_warp[SS_THREADS / 32];
    __shared__ uint32_t s_tile, s_excl;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t epoch = s->epoch;
    if (t == 0) s_tile = atomicAdd(&s->tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t base = tile * SS_TILE;
    if (base >= R) return;

    uint32_t r[SS_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int j0 = 0; j0 < SS_ITEMS; j0 += 4) {
        const uint32_t i0 = base + (uint32_t)t * SS_ITEMS + j0;
        uint4 u = make_uint4(0, 0, 0, 0);
        if (i0 < R) u = philox(i0 >> 2, step, 0u, ctr3, k0, k1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t i = i0 + j;
            uint32_t v = 0;
            if (i < R) {
                const uint32_t k = ebin[i];
                if (k < bins) {
                    v = tab_n[k] + (pick(u, (uint32_t)j) < tab_F[k] ? 1u : 0u);
                } else {
                    atomicOr(&s->status, 1u);
                }
            }
            r[j0 + j] = v;
            sum += v;
        }
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const uint32_t w = lane < SS_THREADS / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SS_THREADS / 32) s_warp[lane] = wi - w;
        const uint32_t agg = __shfl_sync(0xffffffffu, wi, SS_THREADS / 32 - 1);
        if (lane == 0) {
            const unsigned long long tag = (unsigned long long)(epoch & 0x3fffffffu) << 32;
            uint32_t excl = 0;
            if (tile == 0) {
                ss_store(&s->desc[0], (2ull << 62) | tag | agg);
            } else {
                ss_store(&s->desc[tile], (1ull << 62) | tag | agg);
                int p = (int)tile - 1;
                for (;;) {
                    unsigned long long v = 0;
                    unsigned spins = 0;
                    bool ok = false;
                    for (;;) {
                        v = ss_load(&s->desc[p]);
                        if ((v >> 62) != 0 && ((v >> 32) & 0x3fffffffu) == (epoch & 0x3fffffffu)) {
                            ok = true;
                            break;
                        }
                        if (++spins >= SS_SPIN_LIMIT) break;
                        if (spins > 64) __nanosleep(64);
                    }
                    if (!ok) {
                        atomicOr(&s->status, 2u);
                        break;
                    }
                    excl += (uint32_t)(v & 0xffffffffu);
                    if ((v >> 62) == 2ull || p == 0) break;
                    --p;
                }
                ss_store(&s->desc[tile], (2ull << 62) | tag | (excl + agg));
            }
            s_excl = excl;
        }
    }
    __syncthreads();
    uint32_t o = s_excl + s_warp[wid] + (incl - sum);
#pragma unroll
    for (int j = 0; j < SS_ITEMS; ++j) {
        const uint32_t i = base + (uint32_t)t * SS_ITEMS + j;
        if (i < R) {
            counts[i] = r[j];
            offsets[i] = o;
            if (i == R - 1) {
                const uint32_t bad = atomicOr(&s->status, 0u);
                *total = bad ? 0xffffffffu : o + r[j];
            }
        }
        o += r[j];
    }
}

// Device address of the scratch in the current context.  Host code may not use
// the symbol itself as a pointer: on the host it only names the array.  The
// address belongs to the context that loaded the module, so it is cached per
// context, keyed by the driver's context id, which is unique for the life of
// the process: a caller running in its own (non-primary) context, or a
// primary context re-created after cudaDeviceReset, gets a fresh lookup.
// The two driver calls are reached through the runtime's entry-point query,
// so the library does not link libcuda itself.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

struct ScratchCacheEntry {
    unsigned long long ctx_id;
    void* addr;
};
constexpr int SCRATCH_CACHE = 16;
std::mutex g_mu;
ScratchCacheEntry g_cache[SCRATCH_CACHE];
int g_cache_used = 0, g_cache_next = 0;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

cudaError_t current_context_id(unsigned long long* id) {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000,
                                                         cudaEnableDefault, &q0);
        if (e != cudaSuccess || q0 != cudaDriverEntryPointSuccess || !f0)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f1)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    void* ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return cudaErrorDeviceUninitialized;
    if (g_ctx_get_id(ctx, id) != 0) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

cudaError_t scratch_address(void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e == cudaErrorDeviceUninitialized) {
        // no context is current yet: the symbol lookup makes the runtime bind
        // the device's primary context, after which the id can be read
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scan_scratch);
        if (e != cudaSuccess) return e;
        e = current_context_id(&id);
    }
    if (e != cudaSuccess) return e;
    for (int i = 0; i < g_cache_used; ++i) {
        if (g_cache[i].ctx_id == id) {
            *out = g_cache[i].addr;
            return cudaSuccess;
        }
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scan_scratch);
    if (e != cudaSuccess) return e;
    int slot;
    if (g_cache_used < SCRATCH_CACHE) {
        slot = g_cache_used++;
    } else {  // evict the oldest entry
        slot = g_cache_next;
        g_cache_next = (g_cache_next + 1) % SCRATCH_CACHE;
    }
    g_cache[slot].ctx_id = id;
    g_cache[slot].addr = p;
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace pa

extern "C" int pa_copy_counts_scan_noalloc(const uint32_t* d_ebin, int64_t R,
                                           const uint32_t* d_tab_n, const uint32_t* d_tab_F,
                                           int64_t bins, uint64_t seed, int32_t step,
                                           int32_t instance_id, uint32_t* d_counts,
                                           uint32_t* d_offsets, uint32_t* d_total,
                                           void* stream) {
    if (R < 0 || R > PA_NOALLOC_MAX_REPLICAS) return PA_ERR_INVALID_ARG;
    if (bins < 1 || bins > 0xffffffffll || step < 0 || instance_id < 0 ||
        instance_id >= (1 << 28))
        return PA_ERR_INVALID_ARG;
    if (!d_total || (R > 0 && (!d_ebin || !d_tab_n || !d_tab_F || !d_counts || !d_offsets)))
        return PA_ERR_INVALID_ARG;
    void* addr = nullptr;
    if (pa::scratch_address(&addr) != cudaSuccess) return PA_ERR_CUDA;
    auto* s = static_cast<pa::StaticScanScratch*>(addr);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t tiles = (uint32_t)((R + pa::SS_TILE - 1) / pa::SS_TILE);
    pa::k_static_prepare<<<(tiles + 1023) / 1024 > 0 ? (tiles + 1023) / 1024 : 1, 1024, 0, st>>>(
        s, tiles, d_total);
    if (cudaGetLastError() != cudaSuccess) return PA_ERR_CUDA;
    if (R == 0) return PA_OK;
    const uint32_t ctr3 = (pa::TAG_RESAMPLE << 28) | (uint32_t)instance_id;
    pa::k_static_counts_scan<<<tiles, pa::SS_THREADS, 0, st>>>(
        s, d_ebin, (uint32_t)R, d_tab_n, d_tab_F, (uint32_t)bins, (uint32_t)step, ctr3,
        (uint32_t)seed, (uint32_t)(seed >> 32), d_counts, d_offsets, d_total);
    if (cudaGetLastError() != cudaSuccess) return PA_ERR_CUDA;
    return PA_OK;
}
