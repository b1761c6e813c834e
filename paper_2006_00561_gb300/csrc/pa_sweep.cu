// pa_sweep.cu -- initial population, couplings, and the Metropolis sweep with
// its fused measurement epilogue (energy, magnetisation, energy histogram).
//
// Model: Eq. 6 (H = -sum_<ij> J_ij s_i s_j over the bonds of a periodic L^dim
// lattice; J = +1 for the ferromagnet, +-1 for the Edwards-Anderson variant).
// Equilibration (Sec. 2, theta MCMC sweeps at the new temperature): one sweep
// updates the sites of colour 0 (even coordinate sum), then colour 1; sites of
// one colour have no bond between them, so they are updated together.  A site
// with c_u unsatisfied bonds has dE = 4 (dim - c_u); it flips if dE <= 0, or
// if its uniform u (word h & 3 of the Philox block (h >> 2, 2 g + colour,
// slot, SWEEP | instance), h = s >> 1, g = global sweep index) is below the
// threshold T(beta_i, dE) = floor(2^32 exp(-beta_i dE)).
//
// One warp owns one replica at a time; the replica is staged whole in shared
// memory for all sweeps and written back once.  Grid-stride over replicas, the
// population size is read from device memory.
#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr int WARPS = 4;  // warps per block of the generic sweep kernels

template <int DIM, int L>
struct Geo {
    static constexpr int N = DIM == 2 ? L * L : L * L * L;
    static constexpr int NROWS = DIM == 2 ? L : L * L;
    static constexpr int NW = (L + 31) / 32;
    static constexpr int NWORDS = NROWS * NW;
    static constexpr int HALF = N / 2;
    static constexpr int NCALLS = (HALF + 3) / 4;
    static constexpr uint32_t LASTMASK = (L % 32 == 0) ? 0xffffffffu : ((1u << (L % 32)) - 1u);
    static constexpr int I8BYTES = (N + 15) / 16 * 16;
};

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Histogram of up to 32 energy levels, one per lane, with one atomic per
// distinct level (warp-aggregated: lanes holding the same level elect one).
__device__ __forceinline__ void hist_flush(uint32_t* hist, uint32_t level, int n, int lane) {
    if (n <= 0) return;
    const unsigned valid = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
    if (lane < n) {
        const unsigned peers = __match_any_sync(valid, level);
        if (lane == __ffs(peers) - 1) atomicAdd(&hist[level], (uint32_t)__popc(peers));
    }
}

// Lowest-level site of colour c with colour index h (h = s >> 1).  For even L
// the pair {2h, 2h+1} lies in one row; the row's parity decides which member
// has colour c.
template <int DIM, int L>
__device__ __forceinline__ void site_of(int h, int c, int& row, int& x) {
    const int e = 2 * h;
    row = e / L;
    const int x0 = e - row * L;
    const int rowpar = DIM == 2 ? (row & 1) : ((row % L + row / L) & 1);
    x = x0 + ((c + rowpar) & 1);
}

// --------------------------------------------------------------------------
// Packed layout: bit x of row r (r = y, or y + L z) at word r*NW + x/32.
// --------------------------------------------------------------------------
template <int DIM, int L>
__device__ __forceinline__ uint32_t xplus(const uint32_t* row, int k) {  // bit x <- site x+1
    using G = Geo<DIM, L>;
    if constexpr (G::NW == 1) {
        const uint32_t v = row[0];
        if constexpr (L == 32) return (v >> 1) | (v << 31);
        else return ((v >> 1) | (v << (L - 1))) & G::LASTMASK;
    } else {
        return (row[k] >> 1) | (row[(k + 1) % G::NW] << 31);
    }
}

template <int DIM, int L>
__device__ __forceinline__ uint32_t xminus(const uint32_t* row, int k) {  // bit x <- site x-1
    using G = Geo<DIM, L>;
    if constexpr (G::NW == 1) {
        const uint32_t v = row[0];
        if constexpr (L == 32) return (v << 1) | (v >> 31);
        else return ((v << 1) | (v >> (L - 1))) & G::LASTMASK;
    } else {
        return (row[k] << 1) | (row[(k + G::NW - 1) % G::NW] >> 31);
    }
}

template <int DIM, int L>
__device__ __forceinline__ void row_nbrs(int r, int& yp, int& ym, int& zp, int& zm) {
    if constexpr (DIM == 2) {
        yp = (r + 1) % L;
        ym = (r + L - 1) % L;
        zp = zm = 0;
    } else {
        const int y = r % L, z = r / L;
        yp = (y + 1) % L + L * z;
        ym = (y + L - 1) % L + L * z;
        zp = y + L * ((z + 1) % L);
        zm = y + L * ((z + L - 1) % L);
    }
}

__device__ __forceinline__ void count_add(uint32_t& b0, uint32_t& b1, uint32_t& b2, uint32_t a) {
    const uint32_t c0 = b0 & a;
    b0 ^= a;
    const uint32_t c1 = b1 & c0;
    b1 ^= c0;
    b2 |= c1;
}

template <int DIM, int L, bool PMJ>
__global__ void __launch_bounds__(WARPS * 32) k_sweep_packed(RunDev d, int nsweeps) {
    using G = Geo<DIM, L>;
    constexpr int NW = G::NW, NWORDS = G::NWORDS;
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* S = smem + wib * 5 * NWORDS;
    uint32_t* ALW = S + NWORDS;
    uint32_t* CB0 = ALW + NWORDS;
    uint32_t* CB1 = CB0 + NWORDS;
    uint32_t* FLIP = CB1 + NWORDS;

    DevState* st = d.st;
    const uint32_t R = st->R;
    const uint32_t cur = st->cur;
    const uint32_t step = st->step;
    const uint32_t g0 = st->sweep_base;
    const uint32_t parity = st->negbonds & 1u;
    const uint32_t T0 = d.thr[step * 4 + 0], T1 = d.thr[step * 4 + 1], T2 = d.thr[step * 4 + 2];
    const uint32_t full = d.thr[step * 4 + 3];
    const uint32_t ctr3 = (TAG_SWEEP << 28) | d.instance;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    const uint32_t* Jp = d.jpk;  // plane dd at Jp + dd*NWORDS

    uint8_t* spins = d.spins[cur];
    uint32_t* ebin = d.ebin[cur];
    int32_t* mag = d.mag[cur];

    for (int w = lane; w < NWORDS; w += 32) FLIP[w] = 0u;

    long long sumAbsM = 0, sumM2 = 0;
    uint32_t mylevel = 0;
    int nlev = 0;
    const uint32_t nwarps = gridDim.x * WARPS;
    for (uint32_t slot = blockIdx.x * WARPS + wib; slot < R; slot += nwarps) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(spins + (size_t)slot * d.stride);
        for (int w = lane; w < NWORDS; w += 32) S[w] = src[w];
        __syncwarp();
        for (int t = 0; t < nsweeps; ++t) {
            const uint32_t g = g0 + (uint32_t)t;
            for (int c = 0; c < 2; ++c) {
                // phase A: classify every site of colour c (bit-sliced, 32 sites per word)
                for (int w = lane; w < NWORDS; w += 32) {
                    const int r = w / NW, k = w % NW;
                    int yp, ym, zp, zm;
                    row_nbrs<DIM, L>(r, yp, ym, zp, zm);
                    const uint32_t own = S[w];
                    uint32_t jx = 0, jxm = 0, jyp = 0, jym = 0, jzp = 0, jzm = 0;
                    if constexpr (PMJ) {
                        jx = __ldg(Jp + w);
                        jxm = xminus<DIM, L>(Jp + r * NW, k);
                        jyp = __ldg(Jp + NWORDS + w);
                        jym = __ldg(Jp + NWORDS + ym * NW + k);
                        if constexpr (DIM == 3) {
                            jzp = __ldg(Jp + 2 * NWORDS + w);
                            jzm = __ldg(Jp + 2 * NWORDS + zm * NW + k);
                        }
                    }
                    uint32_t b0 = 0, b1 = 0, b2 = 0;
                    count_add(b0, b1, b2, own ^ xplus<DIM, L>(S + r * NW, k) ^ jx);
                    count_add(b0, b1, b2, own ^ xminus<DIM, L>(S + r * NW, k) ^ jxm);
                    count_add(b0, b1, b2, own ^ S[yp * NW + k] ^ jyp);
                    count_add(b0, b1, b2, own ^ S[ym * NW + k] ^ jym);
                    if constexpr (DIM == 3) {
                        count_add(b0, b1, b2, own ^ S[zp * NW + k] ^ jzp);
                        count_add(b0, b1, b2, own ^ S[zm * NW + k] ^ jzm);
                    }
                    const int rowpar = DIM == 2 ? (r & 1) : ((r % L + r / L) & 1);
                    uint32_t cm = ((c + rowpar) & 1) ? 0xAAAAAAAAu : 0x55555555u;
                    if (k == NW - 1) cm &= G::LASTMASK;
                    const uint32_t zero = ~(b0 | b1 | b2);
                    if constexpr (DIM == 2) {
                        ALW[w] = (b1 | b2) & cm;  // c_u >= 2: dE <= 0
                        CB0[w] = zero;            // c_u = 0: dE = 8 (class 1)
                        CB1[w] = 0u;
                    } else {
                        ALW[w] = (b2 | (b1 & b0)) & cm;  // c_u >= 3
                        CB0[w] = b0 & ~b1 & ~b2;         // c_u = 1: dE = 8 (class 1)
                        CB1[w] = zero;                   // c_u = 0: dE = 12 (class 2)
                    }
                }
                __syncwarp();
                // phase B: one Philox block per 4 colour sites
                for (int q = lane; q < G::NCALLS; q += 32) {
                    const uint4 u = philox((uint32_t)q, 2u * g + (uint32_t)c, slot, ctr3, k0, k1);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int h = 4 * q + j;
                        if (h >= G::HALF) break;
                        int r, x;
                        site_of<DIM, L>(h, c, r, x);
                        const int w = r * NW + (x >> 5);
                        const uint32_t bit = 1u << (x & 31);
                        if (ALW[w] & bit) continue;
                        const uint32_t idx = ((CB0[w] & bit) ? 1u : 0u) | ((CB1[w] & bit) ? 2u : 0u);
                        const uint32_t T = idx == 0 ? T0 : (idx == 1 ? T1 : T2);
                        if (((full >> idx) & 1u) || pick(u, (uint32_t)j) < T) atomicOr(&FLIP[w], bit);
                    }
                }
                __syncwarp();
                // phase C: apply
                for (int w = lane; w < NWORDS; w += 32) {
                    S[w] ^= ALW[w] | FLIP[w];
                    FLIP[w] = 0u;
                }
                __syncwarp();
            }
        }
        // measurement: U = unsatisfied bonds, M = N - 2 * (number of -1 spins)
        uint32_t U = 0, down = 0;
        for (int w = lane; w < NWORDS; w += 32) {
            const int r = w / NW, k = w % NW;
            int yp, ym, zp, zm;
            row_nbrs<DIM, L>(r, yp, ym, zp, zm);
            const uint32_t vm = (k == NW - 1) ? G::LASTMASK : 0xffffffffu;
            const uint32_t own = S[w];
            uint32_t jx = 0, jy = 0, jz = 0;
            if constexpr (PMJ) {
                jx = __ldg(Jp + w);
                jy = __ldg(Jp + NWORDS + w);
                if constexpr (DIM == 3) jz = __ldg(Jp + 2 * NWORDS + w);
            }
            U += __popc((own ^ xplus<DIM, L>(S + r * NW, k) ^ jx) & vm);
            U += __popc((own ^ S[yp * NW + k] ^ jy) & vm);
            if constexpr (DIM == 3) U += __popc((own ^ S[zp * NW + k] ^ jz) & vm);
            down += __popc(own & vm);
        }
        U = warp_sum_u32(U);
        down = warp_sum_u32(down);
        const int M = G::N - 2 * (int)down;
        uint32_t* dst = reinterpret_cast<uint32_t*>(spins + (size_t)slot * d.stride);
        for (int w = lane; w < NWORDS; w += 32) dst[w] = S[w];
        if (lane == 0) {
            ebin[slot] = U >> 1;
            mag[slot] = M;
            if ((U & 1u) != parity) atomicOr(&st->status, ST_INVARIANT);
            sumAbsM += M < 0 ? -M : M;
            sumM2 += (long long)M * M;
        }
        if (lane == nlev) mylevel = U >> 1;
        if (++nlev == 32) {
            hist_flush(d.hist, mylevel, 32, lane);
            nlev = 0;
        }
        __syncwarp();
    }
    hist_flush(d.hist, mylevel, nlev, lane);
    if (lane == 0 && (sumAbsM | sumM2)) {
        atomicAdd(&d.accum[0], (unsigned long long)sumAbsM);
        atomicAdd(&d.accum[1], (unsigned long long)sumM2);
    }
}

// --------------------------------------------------------------------------
// int8 layout: one byte (+1 / -1) per site, site s = x + L y (+ L^2 z).
// --------------------------------------------------------------------------
template <int DIM, int L>
__device__ __forceinline__ int nbr(int s, int dd, int dir) {
    int stride = dd == 0 ? 1 : (dd == 1 ? L : L * L);
    const int xcoord = (s / stride) % L;
    const int xn = (xcoord + dir + L) % L;
    return s + (xn - xcoord) * stride;
}

template <int DIM, int L, bool PMJ>
__global__ void __launch_bounds__(WARPS * 32) k_sweep_i8(RunDev d, int nsweeps) {
    using G = Geo<DIM, L>;
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int8_t* S = reinterpret_cast<int8_t*>(smem) + wib * G::I8BYTES;

    DevState* st = d.st;
    const uint32_t R = st->R;
    const uint32_t cur = st->cur;
    const uint32_t step = st->step;
    const uint32_t g0 = st->sweep_base;
    const uint32_t parity = st->negbonds & 1u;
    const uint32_t T0 = d.thr[step * 4 + 0], T1 = d.thr[step * 4 + 1], T2 = d.thr[step * 4 + 2];
    const uint32_t full = d.thr[step * 4 + 3];
    const uint32_t ctr3 = (TAG_SWEEP << 28) | d.instance;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    const int8_t* J = d.j8;

    uint8_t* spins = d.spins[cur];
    uint32_t* ebin = d.ebin[cur];
    int32_t* mag = d.mag[cur];

    long long sumAbsM = 0, sumM2 = 0;
    uint32_t mylevel = 0;
    int nlev = 0;
    const uint32_t nwarps = gridDim.x * WARPS;
    for (uint32_t slot = blockIdx.x * WARPS + wib; slot < R; slot += nwarps) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(spins + (size_t)slot * d.stride);
        uint32_t* S32 = reinterpret_cast<uint32_t*>(S);
        for (int w = lane; w < G::I8BYTES / 4; w += 32) S32[w] = src[w];
        __syncwarp();
        for (int t = 0; t < nsweeps; ++t) {
            const uint32_t g = g0 + (uint32_t)t;
            for (int c = 0; c < 2; ++c) {
                for (int q = lane; q < G::NCALLS; q += 32) {
                    const uint4 u = philox((uint32_t)q, 2u * g + (uint32_t)c, slot, ctr3, k0, k1);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int h = 4 * q + j;
                        if (h >= G::HALF) break;
                        int r, x;
                        site_of<DIM, L>(h, c, r, x);
                        const int s = x + L * r;
                        int local = 0;
#pragma unroll
                        for (int dd = 0; dd < DIM; ++dd) {
                            const int up = nbr<DIM, L>(s, dd, +1), dn = nbr<DIM, L>(s, dd, -1);
                            if constexpr (PMJ) {
                                local += __ldg(J + s * DIM + dd) * S[up];
                                local += __ldg(J + dn * DIM + dd) * S[dn];
                            } else {
                                local += S[up] + S[dn];
                            }
                        }
                        const int dE = 2 * S[s] * local;
                        bool acc = dE <= 0;
                        if (!acc) {
                            const uint32_t idx = (uint32_t)(dE / 4 - 1);
                            const uint32_t T = idx == 0 ? T0 : (idx == 1 ? T1 : T2);
                            acc = ((full >> idx) & 1u) || pick(u, (uint32_t)j) < T;
                        }
                        if (acc) S[s] = (int8_t)-S[s];
                    }
                }
                __syncwarp();
            }
        }
        uint32_t U = 0, down = 0;
        for (int s = lane; s < G::N; s += 32) {
            const int sv = S[s];
            down += sv < 0;
#pragma unroll
            for (int dd = 0; dd < DIM; ++dd) {
                const int up = nbr<DIM, L>(s, dd, +1);
                int prod = sv * S[up];
                if constexpr (PMJ) prod *= __ldg(J + s * DIM + dd);
                U += prod < 0;
            }
        }
        U = warp_sum_u32(U);
        down = warp_sum_u32(down);
        const int M = G::N - 2 * (int)down;
        uint32_t* dst = reinterpret_cast<uint32_t*>(spins + (size_t)slot * d.stride);
        for (int w = lane; w < G::I8BYTES / 4; w += 32) dst[w] = S32[w];
        if (lane == 0) {
            ebin[slot] = U >> 1;
            mag[slot] = M;
            if ((U & 1u) != parity) atomicOr(&st->status, ST_INVARIANT);
            sumAbsM += M < 0 ? -M : M;
            sumM2 += (long long)M * M;
        }
        if (lane == nlev) mylevel = U >> 1;
        if (++nlev == 32) {
            hist_flush(d.hist, mylevel, 32, lane);
            nlev = 0;
        }
        __syncwarp();
    }
    hist_flush(d.hist, mylevel, nlev, lane);
    if (lane == 0 && (sumAbsM | sumM2)) {
        atomicAdd(&d.accum[0], (unsigned long long)sumAbsM);
        atomicAdd(&d.accum[1], (unsigned long long)sumM2);
    }
}

// --------------------------------------------------------------------------
// Initial population (Sec. 2: uniform states at beta0 = 0) and couplings.
// Site s of replica `slot` takes the top bit of word s & 3 of the Philox
// block (s >> 2, 0, slot, INIT | instance); set means spin -1.  Coupling of
// bond (s, d): top bit of word s & 3 of (s >> 2, d, 0, COUPLING | instance)
// under the coupling key; set means J = -1.
// --------------------------------------------------------------------------
__global__ void k_init_packed(RunDev d, int nrows, int NW) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)d.R0 * d.nwords;
    if (gid >= total) return;
    const uint32_t slot = (uint32_t)(gid / d.nwords);
    const uint32_t w = (uint32_t)(gid % d.nwords);
    const int r = (int)(w / NW), k = (int)(w % NW);
    const uint32_t ctr3 = (TAG_INIT << 28) | d.instance;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    uint32_t bits = 0;
    int64_t cached = -1;
    uint4 u = make_uint4(0, 0, 0, 0);
    for (int b = 0; b < 32; ++b) {
        const int x = 32 * k + b;
        if (x >= d.L) break;
        const int64_t s = x + (int64_t)d.L * r;
        if ((s >> 2) != cached) {
            cached = s >> 2;
            u = philox((uint32_t)(s >> 2), 0u, slot, ctr3, k0, k1);
        }
        bits |= (pick(u, (uint32_t)(s & 3)) >> 31) << b;
    }
    reinterpret_cast<uint32_t*>(d.spins[0] + (size_t)slot * d.stride)[w] = bits;
    (void)nrows;
}

__global__ void k_init_i8(RunDev d) {
    const uint64_t calls = (uint64_t)(d.N + 3) / 4;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)d.R0 * calls) return;
    const uint32_t slot = (uint32_t)(gid / calls);
    const uint32_t q = (uint32_t)(gid % calls);
    const uint4 u = philox(q, 0u, slot, (TAG_INIT << 28) | d.instance, (uint32_t)d.seed,
                           (uint32_t)(d.seed >> 32));
    int8_t* dst = reinterpret_cast<int8_t*>(d.spins[0] + (size_t)slot * d.stride);
    for (int j = 0; j < 4; ++j) {
        const int64_t s = 4 * (int64_t)q + j;
        if (s < d.N) dst[s] = (pick(u, (uint32_t)j) >> 31) ? (int8_t)-1 : (int8_t)1;
    }
}

__global__ void k_init_couplings(RunDev d, int NW) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t ctr3 = (TAG_COUPLING << 28) | d.instance;
    const uint32_t k0 = (uint32_t)d.coupling_seed, k1 = (uint32_t)(d.coupling_seed >> 32);
    uint32_t neg = 0;
    if (d.layout == PA_LAYOUT_PACKED) {
        if (gid < (uint64_t)d.dim * d.nwords) {
            const int dd = (int)(gid / d.nwords);
            const uint32_t w = (uint32_t)(gid % d.nwords);
            const int r = (int)(w / NW), k = (int)(w % NW);
            uint32_t bits = 0;
            for (int b = 0; b < 32; ++b) {
                const int x = 32 * k + b;
                if (x >= d.L) break;
                const int64_t s = x + (int64_t)d.L * r;
                const uint4 u = philox((uint32_t)(s >> 2), (uint32_t)dd, 0u, ctr3, k0, k1);
                bits |= (pick(u, (uint32_t)(s & 3)) >> 31) << b;
            }
            d.jpk[gid] = bits;
            neg = __popc(bits);
        }
    } else {
        if (gid < (uint64_t)d.N * d.dim) {
            const int64_t s = (int64_t)(gid / d.dim);
            const int dd = (int)(gid % d.dim);
            const uint4 u = philox((uint32_t)(s >> 2), (uint32_t)dd, 0u, ctr3, k0, k1);
            const uint32_t bit = pick(u, (uint32_t)(s & 3)) >> 31;
            d.j8[gid] = bit ? (int8_t)-1 : (int8_t)1;
            neg = bit;
        }
    }
    neg = warp_sum_u32(neg);
    if ((threadIdx.x & 31) == 0 && neg) atomicAdd(&d.st->negbonds, neg);
}

// --------------------------------------------------------------------------
// dispatch
// --------------------------------------------------------------------------
struct KInfo {
    const void* fn;
    int smem;
};

template <int DIM, int L>
KInfo pick_kernel(int layout, bool pmj) {
    using G = Geo<DIM, L>;
    if (layout == PA_LAYOUT_PACKED) {
        const int smem = WARPS * 5 * G::NWORDS * 4;
        return {pmj ? (const void*)k_sweep_packed<DIM, L, true>
                    : (const void*)k_sweep_packed<DIM, L, false>,
                smem};
    }
    const int smem = WARPS * G::I8BYTES;
    return {pmj ? (const void*)k_sweep_i8<DIM, L, true> : (const void*)k_sweep_i8<DIM, L, false>,
            smem};
}

KInfo find_kernel(int layout, int dim, int L, bool pmj) {
#define PA_CASE(D_, L_) \
    if (dim == D_ && L == L_) return pick_kernel<D_, L_>(layout, pmj);
    PA_CASE(2, 4) PA_CASE(2, 8) PA_CASE(2, 16) PA_CASE(2, 32) PA_CASE(2, 64) PA_CASE(2, 128)
    PA_CASE(3, 2) PA_CASE(3, 4) PA_CASE(3, 6) PA_CASE(3, 8) PA_CASE(3, 10) PA_CASE(3, 12)
    PA_CASE(3, 16)
#undef PA_CASE
    return {nullptr, 0};
}

}  // namespace

bool sweep_supported(int layout, int dim, int L) {
    if (layout != PA_LAYOUT_INT8 && layout != PA_LAYOUT_PACKED) return false;
    return find_kernel(layout, dim, L, false).fn != nullptr;
}

int sweep_grid(const RunDev& d) {
    if (l64_applies(d)) return l64_grid(d);
    const KInfo k = find_kernel(d.layout, d.dim, d.L, d.model == PA_MODEL_PMJ);
    if (!k.fn) return 0;
    if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) !=
        cudaSuccess)
        return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, WARPS * 32, k.smem) !=
        cudaSuccess)
        return 0;
    if (per_sm < 1) return 0;
    const int64_t need = ((int64_t)d.cap + WARPS - 1) / WARPS;
    const int64_t full = (int64_t)sms * per_sm;
    return (int)(need < full ? need : full);
}

cudaError_t launch_sweep(const RunDev& d, int nsweeps, int grid, cudaStream_t s) {
    if (l64_applies(d)) return launch_sweep_l64(d, nsweeps, grid, s);
    const KInfo k = find_kernel(d.layout, d.dim, d.L, d.model == PA_MODEL_PMJ);
    if (!k.fn) return cudaErrorInvalidValue;
    RunDev dd = d;
    int n = nsweeps;
    void* args[] = {&dd, &n};
    return cudaLaunchKernel(k.fn, dim3(grid), dim3(WARPS * 32), args, (size_t)k.smem, s);
}

cudaError_t launch_init(const RunDev& d, cudaStream_t s) {
    const int NW = (d.L + 31) / 32;
    if (d.model == PA_MODEL_PMJ) {
        const uint64_t n = d.layout == PA_LAYOUT_PACKED ? (uint64_t)d.dim * d.nwords
                                                        : (uint64_t)d.N * d.dim;
        k_init_couplings<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d, NW);
    }
    if (d.layout == PA_LAYOUT_PACKED) {
        const uint64_t n = (uint64_t)d.R0 * d.nwords;
        const int nrows = d.dim == 2 ? d.L : d.L * d.L;
        k_init_packed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d, nrows, NW);
    } else {
        const uint64_t n = (uint64_t)d.R0 * ((d.N + 3) / 4);
        k_init_i8<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d);
    }
    return cudaGetLastError();
}

}  // namespace pa
