// pa_sweep.cu -- initial population, couplings, and the Metropolis sweep with
// its fused measurement epilogue (energy, magnetisation, energy histogram).
//
// Model: Eq. 6 (H = -sum_<ij> J_ij s_i s_j over the bonds of a periodic L^dim
// lattice; J = +1 for the ferromagnet, +-1 for the Edwards-Anderson variant).
// Equilibration (Sec. 2, theta MCMC sweeps at the new temperature): one sweep
// updates the sites of colour 0 (even coordinate sum), then colour 1; sites of
// one colour have no bond between them, so they are updated together.  A site
// with c_u unsatisfied bonds has dE = 4 (dim - c_u); it flips if dE <= 0, or
// if its uniform u (word h & 3 of the Philox block with counter (2 g + colour,
// h >> 2, SWEEP | instance, slot), h = s >> 1, g = global sweep index) is below the
// threshold T(beta_i, dE) = floor(2^32 exp(-beta_i dE)).
//
// One warp owns one replica at a time; the replica is staged whole in shared
// memory for all sweeps and written back once.  The plain kernels grid-stride
// over the replicas of one run; the batched kernels claim chunks of 32
// replicas of one run at a time from the global slot space of a batch class.
// Both call the same per-replica device functions, so they give the same bits.
#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr int WARPS = 4;  // warps per block of the plain generic sweep kernels

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


// Per-run scalars of one sweep launch, read from the run's device state.
struct SweepCtx {
    uint32_t R, cur, step, g0, parity, T0, T1, T2, full, ctag, k0, k1;
    uint32_t nT0, nT1, nT2, one, four;  // 2^32 - T_c, and opaque 1 and 4 (carry-chain tests)
};

// Which thresholds of the row kernel run their test as a carry chain (bit c
// for class c), in 2D and in 3D.  Measured on GB300: 2D L = 32 gains 10 %
// with both classes on the chain; 3D (L = 8, 10) is not bound by the tests
// and keeps the dE = 4 class on the chain only.
#ifndef PA_ROWS_CARRY2
#define PA_ROWS_CARRY2 3
#endif
#ifndef PA_ROWS_CARRY3
#define PA_ROWS_CARRY3 1
#endif

// acc * 4 + [u >= T] on the FMA pipe: the carry out of u * 1 + (2^32 - T)
// feeds the multiply-add that shifts the accumulator (valid for T > 0).
__device__ __forceinline__ uint32_t carry_ge4(uint32_t acc, uint32_t u, uint32_t one,
                                              uint32_t negT, uint32_t four) {
    uint32_t out;
    asm("{\n\t.reg .u32 t;\n\tmad.lo.cc.u32 t, %1, %2, %3;\n\tmadc.lo.u32 %0, %4, %5, 0;\n\t}"
        : "=r"(out)
        : "r"(u), "r"(one), "r"(negT), "r"(acc), "r"(four));
    return out;
}

__device__ __forceinline__ SweepCtx sweep_ctx(const RunDev& d) {
    SweepCtx x;
    const DevState* st = d.st;
    x.R = st->R;
    x.cur = st->cur;
    x.step = st->step;
    x.g0 = st->sweep_base;
    x.parity = st->negbonds & 1u;
    x.T0 = d.thr[x.step * 4 + 0];
    x.T1 = d.thr[x.step * 4 + 1];
    x.T2 = d.thr[x.step * 4 + 2];
    x.full = d.thr[x.step * 4 + 3];
    x.ctag = (TAG_SWEEP << 28) | d.instance;  // counter word 2 of the sweep
    x.k0 = (uint32_t)d.seed;
    x.k1 = (uint32_t)(d.seed >> 32);
    x.nT0 = 0u - x.T0;
    x.nT1 = 0u - x.T1;
    x.nT2 = 0u - x.T2;
    x.one = d.one;
    x.four = d.one << 2;
    return x;
}

// Per-warp bookkeeping of the measurement: energy levels of up to 32
// replicas (one per lane) for one warp-aggregated histogram flush, and the
// magnetisation sums.
struct Tally {
    long long sumAbsM = 0, sumM2 = 0;
    uint32_t level = 0;
    int n = 0;

    __device__ __forceinline__ void add(uint32_t* hist, uint32_t U, int M, int lane) {
        if (lane == 0) {
            sumAbsM += M < 0 ? -M : M;
            sumM2 += (long long)M * M;
        }
        if (lane == n) level = U >> 1;
        if (++n == 32) {
            hist_flush(hist, level, 32, lane);
            n = 0;
        }
    }
    __device__ __forceinline__ void finish(uint32_t* hist, unsigned long long* accum, int lane) {
        hist_flush(hist, level, n, lane);
        n = 0;
        if (lane == 0 && (sumAbsM | sumM2)) {
            atomicAdd(&accum[0], (unsigned long long)sumAbsM);
            atomicAdd(&accum[1], (unsigned long long)sumM2);
        }
        sumAbsM = sumM2 = 0;
    }
};

// Stores the measured level and magnetisation of a replica (lane 0) and
// checks that U has the instance's parity.
__device__ __forceinline__ void record(const RunDev& d, const SweepCtx& x, uint32_t slot,
                                       uint32_t U, int M, int lane) {
    if (lane == 0) {
        d.ebin[x.cur][slot] = U >> 1;
        d.mag[x.cur][slot] = M;
        if ((U & 1u) != x.parity) atomicOr(&d.st->status, ST_INVARIANT);
    }
}

// --------------------------------------------------------------------------
// One replica, packed layout: theta sweeps in shared memory (S and the four
// class / flip arrays of NWORDS words each), then the measurement.  Returns
// U; M through the reference.  FLIP must be zero on entry and is on exit.
// --------------------------------------------------------------------------
template <int DIM, int L, bool PMJ>
__device__ __forceinline__ uint32_t packed_replica(const RunDev& d, const SweepCtx& x,
                                                   uint32_t slot, int nsweeps, uint32_t* S,
                                                   int lane, int& M) {
    using G = Geo<DIM, L>;
    constexpr int NW = G::NW, NWORDS = G::NWORDS;
    uint32_t* ALW = S + NWORDS;
    uint32_t* CB0 = ALW + NWORDS;
    uint32_t* CB1 = CB0 + NWORDS;
    uint32_t* FLIP = CB1 + NWORDS;
    const uint32_t* Jp = d.jpk;  // plane dd at Jp + dd*NWORDS
    uint8_t* spins = d.spins[x.cur];

    const uint32_t* src = reinterpret_cast<const uint32_t*>(spins + (size_t)slot * d.stride);
    for (int w = lane; w < NWORDS; w += 32) S[w] = src[w];
    __syncwarp();
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t g = x.g0 + (uint32_t)t;
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
                const uint4 u = philox(2u * g + (uint32_t)c, (uint32_t)q, x.ctag, slot, x.k0, x.k1);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int h = 4 * q + j;
                    if (h >= G::HALF) break;
                    int r, xx;
                    site_of<DIM, L>(h, c, r, xx);
                    const int w = r * NW + (xx >> 5);
                    const uint32_t bit = 1u << (xx & 31);
                    if (ALW[w] & bit) continue;
                    const uint32_t idx = ((CB0[w] & bit) ? 1u : 0u) | ((CB1[w] & bit) ? 2u : 0u);
                    const uint32_t T = idx == 0 ? x.T0 : (idx == 1 ? x.T1 : x.T2);
                    if (((x.full >> idx) & 1u) || pick(u, (uint32_t)j) < T) atomicOr(&FLIP[w], bit);
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
    M = G::N - 2 * (int)down;
    uint32_t* dst = reinterpret_cast<uint32_t*>(spins + (size_t)slot * d.stride);
    for (int w = lane; w < NWORDS; w += 32) dst[w] = S[w];
    __syncwarp();
    return U;
}

// --------------------------------------------------------------------------
// One replica, int8 layout: one byte (+1 / -1) per site, s = x + L y (+L^2 z).
// Same-colour sites are independent, so a lane flips its site in place.
// --------------------------------------------------------------------------
template <int DIM, int L>
__device__ __forceinline__ int nbr(int s, int dd, int dir) {
    int stride = dd == 0 ? 1 : (dd == 1 ? L : L * L);
    const int xcoord = (s / stride) % L;
    const int xn = (xcoord + dir + L) % L;
    return s + (xn - xcoord) * stride;
}

template <int DIM, int L, bool PMJ>
__device__ __forceinline__ uint32_t i8_replica(const RunDev& d, const SweepCtx& x, uint32_t slot,
                                               int nsweeps, int8_t* S, int lane, int& M) {
    using G = Geo<DIM, L>;
    const int8_t* J = d.j8;
    uint8_t* spins = d.spins[x.cur];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(spins + (size_t)slot * d.stride);
    uint32_t* S32 = reinterpret_cast<uint32_t*>(S);
    for (int w = lane; w < G::I8BYTES / 4; w += 32) S32[w] = src[w];
    __syncwarp();
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t g = x.g0 + (uint32_t)t;
        for (int c = 0; c < 2; ++c) {
            for (int q = lane; q < G::NCALLS; q += 32) {
                const uint4 u = philox(2u * g + (uint32_t)c, (uint32_t)q, x.ctag, slot, x.k0, x.k1);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int h = 4 * q + j;
                    if (h >= G::HALF) break;
                    int r, xx;
                    site_of<DIM, L>(h, c, r, xx);
                    const int s = xx + L * r;
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
                        const uint32_t T = idx == 0 ? x.T0 : (idx == 1 ? x.T1 : x.T2);
                        acc = ((x.full >> idx) & 1u) || pick(u, (uint32_t)j) < T;
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
    M = G::N - 2 * (int)down;
    uint32_t* dst = reinterpret_cast<uint32_t*>(spins + (size_t)slot * d.stride);
    for (int w = lane; w < G::I8BYTES / 4; w += 32) dst[w] = S32[w];
    __syncwarp();
    return U;
}

// --------------------------------------------------------------------------
// One replica, packed layout with one 32-bit word per row (L <= 32) and at
// most 128 rows (2D L <= 32, 3D L <= 10): rows resident in registers.
// Lane l owns rows l, l + 32, ... and keeps their spins and couplings in
// registers; the rows are also published in shared memory (S) for the
// neighbours.  Per half-sweep: (1) Philox blocks in counter order into U
// (shared), (2) every owned row takes the uniforms of its L/2 colour sites
// from U at compile-time offsets, tests them against all class thresholds at
// once (bit j of mask t set iff u_j < T_t) and combines them with the row's
// bit-sliced classes, (3) the rows are flipped and re-published.  Same
// counters and thresholds as packed_replica(), hence the same bits.
// --------------------------------------------------------------------------
template <int DIM, int L>
struct RowGeo {
    static constexpr int NROWS = DIM == 2 ? L : L * L;
    static constexpr int RPL = (NROWS + 31) / 32;
    static constexpr int HR = L / 2;  // colour sites per row
    static constexpr uint32_t MASK = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
    static constexpr bool OK = L <= 32 && NROWS <= 128;
};

template <int DIM, int L>
__device__ __forceinline__ uint32_t rot_plus(uint32_t v) {  // bit x <- bit x+1 (mod L)
    if constexpr (L == 32) return (v >> 1) | (v << 31);
    else return ((v >> 1) | (v << (L - 1))) & RowGeo<DIM, L>::MASK;
}
template <int DIM, int L>
__device__ __forceinline__ uint32_t rot_minus(uint32_t v) {  // bit x <- bit x-1 (mod L)
    if constexpr (L == 32) return (v << 1) | (v >> 31);
    else return ((v << 1) | (v >> (L - 1))) & RowGeo<DIM, L>::MASK;
}

template <int DIM, int L, bool PMJ>
__device__ __forceinline__ uint32_t rows_replica(const RunDev& d, const SweepCtx& x, uint32_t slot,
                                                 int nsweeps, uint32_t* S, int lane, int& M) {
    using RG = RowGeo<DIM, L>;
    using G = Geo<DIM, L>;
    constexpr int NROWS = RG::NROWS, RPL = RG::RPL, HR = RG::HR;
    uint32_t* U = S + ((NROWS + 3) & ~3);  // uniforms of the half-sweep, in counter order
    const uint32_t* Jp = d.jpk;
    uint8_t* spins = d.spins[x.cur];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(spins + (size_t)slot * d.stride);

    uint32_t own[RPL], jx[RPL], jxm[RPL], jyp[RPL], jym[RPL], jzp[RPL], jzm[RPL];
    int yp[RPL], ym[RPL], zp[RPL], zm[RPL], par[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
        const int r = lane + 32 * k;
        own[k] = 0u;
        jx[k] = jxm[k] = jyp[k] = jym[k] = jzp[k] = jzm[k] = 0u;
        yp[k] = ym[k] = zp[k] = zm[k] = par[k] = 0;
        if (r < NROWS) {
            row_nbrs<DIM, L>(r, yp[k], ym[k], zp[k], zm[k]);
            par[k] = DIM == 2 ? (r & 1) : ((r % L + r / L) & 1);
            own[k] = src[r];
            S[r] = own[k];
            if constexpr (PMJ) {
                jx[k] = __ldg(Jp + r);
                jxm[k] = rot_minus<DIM, L>(jx[k]);
                jyp[k] = __ldg(Jp + NROWS + r);
                jym[k] = __ldg(Jp + NROWS + ym[k]);
                if constexpr (DIM == 3) {
                    jzp[k] = __ldg(Jp + 2 * NROWS + r);
                    jzm[k] = __ldg(Jp + 2 * NROWS + zm[k]);
                }
            }
        }
    }
    __syncwarp();
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t g = x.g0 + (uint32_t)t;
        for (int c = 0; c < 2; ++c) {
            for (int q = lane; q < G::NCALLS; q += 32) {
                const uint4 u = philox(2u * g + (uint32_t)c, (uint32_t)q, x.ctag, slot, x.k0, x.k1);
                reinterpret_cast<uint4*>(U)[q] = u;
            }
            __syncwarp();
            uint32_t flip[RPL];
#pragma unroll
            for (int k = 0; k < RPL; ++k) {
                flip[k] = 0u;
                const int r = lane + 32 * k;
                if (r >= NROWS) continue;
                const uint32_t o = own[k];
                uint32_t b0 = 0, b1 = 0, b2 = 0;
                count_add(b0, b1, b2, o ^ rot_plus<DIM, L>(o) ^ jx[k]);
                count_add(b0, b1, b2, o ^ rot_minus<DIM, L>(o) ^ jxm[k]);
                count_add(b0, b1, b2, o ^ S[yp[k]] ^ jyp[k]);
                count_add(b0, b1, b2, o ^ S[ym[k]] ^ jym[k]);
                if constexpr (DIM == 3) {
                    count_add(b0, b1, b2, o ^ S[zp[k]] ^ jzp[k]);
                    count_add(b0, b1, b2, o ^ S[zm[k]] ^ jzm[k]);
                }
                const uint32_t zero = ~(b0 | b1 | b2);
                uint32_t alw, m0, m1, m2;
                if constexpr (DIM == 2) {
                    alw = b1 | b2;            // c_u >= 2: dE <= 0
                    m1 = zero;                // c_u = 0: dE = 8
                    m0 = b0 & ~b1 & ~b2;      // c_u = 1: dE = 4
                    m2 = 0u;
                } else {
                    alw = b2 | (b1 & b0);     // c_u >= 3
                    m2 = zero;                // c_u = 0: dE = 12
                    m1 = b0 & ~b1 & ~b2;      // c_u = 1: dE = 8
                    m0 = b1 & ~b0 & ~b2;      // c_u = 2: dE = 4
                }
                // site frame: bit 2j <-> colour site j of the row (x = 2j + p)
                const int p = (c + par[k]) & 1;
                const uint32_t* ur = U + HR * r;
                uint32_t a0 = 0, a1 = 0, a2 = 0;
                constexpr uint32_t EVEN = 0x55555555u;
                constexpr uint32_t SITES = (HR >= 16 ? 0xffffffffu : ((1u << (2 * HR)) - 1u)) & EVEN;
                // thresholds whose test runs as a carry chain on the FMA pipe
                // (acc * 4 + [u >= T], sites in decreasing j so site j ends at
                // bit 2j), the others as compare and select on the ALU
                constexpr int CM = DIM == 2 ? PA_ROWS_CARRY2 : PA_ROWS_CARRY3;
#pragma unroll
                for (int j = HR - 1; j >= 0; --j) {
                    const uint32_t u = ur[j];
                    const uint32_t bit = 1u << (2 * j);
                    if constexpr (CM & 1) a0 = carry_ge4(a0, u, x.one, x.nT0, x.four);
                    else if (u < x.T0) a0 |= bit;
                    if constexpr (CM & 2) a1 = carry_ge4(a1, u, x.one, x.nT1, x.four);
                    else if (u < x.T1) a1 |= bit;
                    if constexpr (DIM == 3) {
                        if constexpr (CM & 4) a2 = carry_ge4(a2, u, x.one, x.nT2, x.four);
                        else if (u < x.T2) a2 |= bit;
                    }
                }
                if constexpr (CM & 1) a0 = x.T0 ? (~a0 & SITES) : 0u;
                if constexpr (CM & 2) a1 = x.T1 ? (~a1 & SITES) : 0u;
                if constexpr (DIM == 3 && (CM & 4)) a2 = x.T2 ? (~a2 & SITES) : 0u;
                if (x.full & 1u) a0 = ~0u;
                if (x.full & 2u) a1 = ~0u;
                if (x.full & 4u) a2 = ~0u;
                const uint32_t acc = ((alw >> p) | ((m0 >> p) & a0) | ((m1 >> p) & a1) |
                                      ((m2 >> p) & a2)) & EVEN;
                flip[k] = (acc << p) & RG::MASK;
            }
            __syncwarp();  // every lane is done reading S and U
#pragma unroll
            for (int k = 0; k < RPL; ++k) {
                const int r = lane + 32 * k;
                if (r < NROWS) {
                    own[k] ^= flip[k];
                    S[r] = own[k];
                }
            }
            __syncwarp();
        }
    }
    uint32_t Uc = 0, down = 0;
    uint32_t* dst = reinterpret_cast<uint32_t*>(spins + (size_t)slot * d.stride);
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
        const int r = lane + 32 * k;
        if (r >= NROWS) continue;
        const uint32_t o = own[k];
        Uc += __popc((o ^ rot_plus<DIM, L>(o) ^ jx[k]) & RG::MASK);
        Uc += __popc((o ^ S[yp[k]] ^ jyp[k]) & RG::MASK);
        if constexpr (DIM == 3) Uc += __popc((o ^ S[zp[k]] ^ jzp[k]) & RG::MASK);
        down += __popc(o & RG::MASK);
        dst[r] = o;
    }
    Uc = warp_sum_u32(Uc);
    down = warp_sum_u32(down);
    M = G::N - 2 * (int)down;
    __syncwarp();
    return Uc;
}

// Shared memory per warp of each layout, in 32-bit words.
template <int DIM, int L, int LAYOUT>
__host__ __device__ constexpr int warp_words() {
    if constexpr (LAYOUT != PA_LAYOUT_PACKED) return Geo<DIM, L>::I8BYTES / 4;
    else if constexpr (RowGeo<DIM, L>::OK)
        return ((RowGeo<DIM, L>::NROWS + 3) & ~3) + 4 * Geo<DIM, L>::NCALLS;
    else return 5 * Geo<DIM, L>::NWORDS;
}

template <int DIM, int L, int LAYOUT, bool PMJ>
__device__ __forceinline__ uint32_t one_replica(const RunDev& d, const SweepCtx& x, uint32_t slot,
                                                int nsweeps, uint32_t* wsmem, int lane, int& M) {
    if constexpr (LAYOUT == PA_LAYOUT_PACKED && RowGeo<DIM, L>::OK)
        return rows_replica<DIM, L, PMJ>(d, x, slot, nsweeps, wsmem, lane, M);
    else if constexpr (LAYOUT == PA_LAYOUT_PACKED)
        return packed_replica<DIM, L, PMJ>(d, x, slot, nsweeps, wsmem, lane, M);
    else
        return i8_replica<DIM, L, PMJ>(d, x, slot, nsweeps, reinterpret_cast<int8_t*>(wsmem), lane,
                                       M);
}

// Plain: every replica of one run, grid-stride.
template <int DIM, int L, int LAYOUT, bool PMJ>
__global__ void __launch_bounds__(WARPS * 32) k_sweep(RunDev d, int nsweeps) {
    extern __shared__ uint32_t smem[];
    constexpr int WW = warp_words<DIM, L, LAYOUT>();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* ws = smem + wib * WW;
    if constexpr (LAYOUT == PA_LAYOUT_PACKED && !RowGeo<DIM, L>::OK)
        for (int w = lane; w < Geo<DIM, L>::NWORDS; w += 32) ws[4 * Geo<DIM, L>::NWORDS + w] = 0u;
    __syncwarp();
    const SweepCtx x = sweep_ctx(d);
    Tally tally;
    const uint32_t nwarps = gridDim.x * WARPS;
    const uint32_t end = min(x.R, d.slot_hi);
    for (uint32_t slot = d.slot_lo + blockIdx.x * WARPS + wib; slot < end; slot += nwarps) {
        int M = 0;
        const uint32_t U = one_replica<DIM, L, LAYOUT, PMJ>(d, x, slot, nsweeps, ws, lane, M);
        record(d, x, slot, U, M, lane);
        tally.add(d.hist, U, M, lane);
    }
    tally.finish(d.hist, d.accum, lane);
}

// Batched: chunks of a.chunk slots of one run, claimed from the class's slot space.
template <int DIM, int L, int LAYOUT, bool PMJ, int BW>
__global__ void __launch_bounds__(BW * 32) k_sweep_batched(BatchSweepArgs a) {
    extern __shared__ uint32_t smem[];
    constexpr int WW = warp_words<DIM, L, LAYOUT>();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* ws = smem + wib * WW;
    if constexpr (LAYOUT == PA_LAYOUT_PACKED && !RowGeo<DIM, L>::OK)
        for (int w = lane; w < Geo<DIM, L>::NWORDS; w += 32) ws[4 * Geo<DIM, L>::NWORDS + w] = 0u;
    __syncwarp();
    Tally tally;
    for (;;) {
        uint32_t chunk = 0;
        if (lane == 0) chunk = atomicAdd(a.counter, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint32_t g = chunk * a.chunk;
        if (g >= a.total_slots) break;
        uint32_t lo = 0, hi = a.n;  // slot_base[lo] <= g < slot_base[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.slot_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        const RunDev& d = a.runs[a.run_ids[lo]];
        const SweepCtx x = sweep_ctx(d);
        const uint32_t first = g - a.slot_base[lo];
        for (uint32_t slot = first; slot < first + a.chunk && slot < x.R; ++slot) {
            int M = 0;
            const uint32_t U = one_replica<DIM, L, LAYOUT, PMJ>(d, x, slot, d.theta, ws, lane, M);
            record(d, x, slot, U, M, lane);
            tally.add(d.hist, U, M, lane);
        }
        tally.finish(d.hist, d.accum, lane);
    }
}

// --------------------------------------------------------------------------
// Replica-sliced sweeps (packed layout, L <= 32): a warp takes 32 replicas of
// one run, slots b0 .. b0 + 31, and keeps in shared memory one 32-bit word
// per lattice site whose bit r is the spin of replica b0 + r (set = -1).
// All bit logic (bond states, the bit-sliced count of unsatisfied bonds, the
// energy classes, the flips) then runs on 32 replicas at once, whatever L and
// the dimension, and no lane idles on a short row.
//
// Random numbers and update rule are those of the other kernels: in a
// half-sweep of colour c, lane k of the work takes the group of the four
// colour-c sites with h = s >> 1 in 4k .. 4k + 3 (Philox counter
// (2g + c, k, SWEEP | instance, slot), word h & 3), draws the 32 replicas'
// blocks and folds every uniform into carry chains, one per (site, class):
// acc = 2 acc + [u >= T_class], replica r ending at bit r.  A site flips in
// replica r if its class has dE <= 0, or if bit r of the chain of its class
// is clear (u < T).
// --------------------------------------------------------------------------
// Shared-memory index of site word s.  The lanes of a half-sweep touch sites
// about 8 apart (four pairs each), so one padding word per 32 sites spreads
// them over all banks.
#ifndef PA_RS_PAD
#define PA_RS_PAD 1
#endif
// Classes whose chain runs on the FMA pipe (multiply-add with carry-out and a
// multiply-add with carry-in by 2) instead of the ALU (bit c for class c).
#ifndef PA_RS_FMA
#define PA_RS_FMA 0
#endif
__device__ __forceinline__ int rs_ix(int s) { return PA_RS_PAD ? s + (s >> 5) : s; }

template <int DIM, int L, bool PMJ>
struct RSGeo {
    static constexpr int N = DIM == 2 ? L * L : L * L * L;
    static constexpr int NS = PA_RS_PAD ? N + (N + 31) / 32 : N;  // site words with padding
    static constexpr int HALF = N / 2;
    static constexpr int NGROUPS = HALF / 4;
    static constexpr int NROWS = DIM == 2 ? L : L * L;
    static constexpr int NCLS = DIM == 2 ? 2 : 3;
    static constexpr int JWORDS = PMJ ? (N + 3) / 4 : 0;  // coupling pattern, one byte per site
    static constexpr int WORDS = NS + JWORDS + 20;        // + round keys (batched form)
    static constexpr int SPL = (N + 31) / 32;             // sites per lane in the measurement
    static constexpr int bits(int v) { return v <= 1 ? 1 : 1 + bits(v >> 1); }
    static constexpr int KU = bits(DIM * SPL);
    static constexpr int KM = bits(SPL);
    static constexpr bool OK = L <= 32 && (HALF % 4) == 0 && N >= 8;
};

template <int DIM, int L, int RSW>
__host__ __device__ constexpr int rs_words(bool pmj) {
    return pmj ? RSGeo<DIM, L, true>::WORDS : RSGeo<DIM, L, false>::WORDS;
}

// Neighbours of site s in the order +x, -x, +y, -y (, +z, -z), periodic.
template <int DIM, int L>
__device__ __forceinline__ void rs_nbrs(int s, int (&nb)[2 * DIM]) {
    const int x = s % L, row = s / L, y = row % L;
    nb[0] = x == L - 1 ? s - (L - 1) : s + 1;
    nb[1] = x == 0 ? s + (L - 1) : s - 1;
    nb[2] = y == L - 1 ? s - (L - 1) * L : s + L;
    nb[3] = y == 0 ? s + (L - 1) * L : s - L;
    if constexpr (DIM == 3) {
        const int z = row / L;
        nb[4] = z == L - 1 ? s - (L - 1) * L * L : s + L * L;
        nb[5] = z == 0 ? s + (L - 1) * L * L : s - L * L;
    }
}

// Colour-c site of pair h = s >> 1.
template <int DIM, int L>
__device__ __forceinline__ int rs_site(int h, int c) {
    const int row = h / (L / 2), m = h % (L / 2);
    const int par = DIM == 2 ? (row & 1) : ((row % L + row / L) & 1);
    return row * L + 2 * m + ((c + par) & 1);
}

// acc = 2 acc + [u >= T]: the carry of u - T, shifted in with the add.
__device__ __forceinline__ uint32_t rs_chain(uint32_t acc, uint32_t u, uint32_t T) {
    uint32_t out;
    asm("{\n\t.reg .u32 t;\n\tsub.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
        : "=r"(out) : "r"(u), "r"(T), "r"(acc));
    return out;
}

// The same on the FMA pipe: u * 1 + (2^32 - T) carries iff u >= T (T > 0;
// T = 0 never carries and is handled by the caller), then acc * 2 + carry.
__device__ __forceinline__ uint32_t rs_chain_fma(uint32_t acc, uint32_t u, uint32_t one,
                                                 uint32_t negT, uint32_t two) {
    uint32_t out;
    asm("{\n\t.reg .u32 t;\n\tmad.lo.cc.u32 t, %1, %2, %3;\n\tmadc.lo.u32 %0, %4, %5, 0;\n\t}"
        : "=r"(out) : "r"(u), "r"(one), "r"(negT), "r"(acc), "r"(two));
    return out;
}

// Bit-sliced counter of 32 lanes' worth of bits: adds word v into C[0..K-1].
template <int K>
__device__ __forceinline__ void rs_count(uint32_t (&C)[K], uint32_t v) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t t = C[k] & v;
        C[k] ^= v;
        v = t;
    }
}

// Sum over the warp of the bit-sliced counters, for replica r = lane: bit r
// of plane k over all lanes, weighted 2^k (a transpose by ballots).
template <int K>
__device__ __forceinline__ uint32_t rs_total(const uint32_t (&C)[K], int lane) {
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const uint32_t b = __ballot_sync(0xffffffffu, (C[k] >> r) & 1u);
            if (lane == r) tot += (uint32_t)__popc(b) << k;
        }
    }
    return tot;
}

// Philox round keys: pointers into the kernel parameters (plain kernel, so
// that the xors take them as constant-bank operands) or into the warp's
// shared-memory copy of the chunk's run (batched kernel).  PA_RS_KEYREG = 1
// copies them into registers instead; on GB300 that ran 1.4 % slower on the
// 3D ensemble (the extra registers cost more than the loads).
struct RSKeys {
    const uint32_t* rk0;
    const uint32_t* rk1;
};
struct RSKeyRegs {
    uint32_t rk0[10], rk1[10];
};
#ifndef PA_RS_KEYREG
#define PA_RS_KEYREG 0
#endif

// How the replica-sliced kernel forms its Philox products: 0 = high and low
// halves from C++ (__umulhi, *), 1 (the default) = one mul.wide.u32 per
// product.  Measured on GB300 (single runs, attempts/ns, same bits), 0 -> 1:
// 3D +-J L = 8 1120 -> 1223, L = 10 1027 -> 1100, L = 6 916 -> 982, 2D L = 32
// 1295 -> 1391, L = 16 1237 -> 1330.
#ifndef PA_RS_MUL_MODE
#define PA_RS_MUL_MODE 1
#endif
// PA_RS_OR_SLOT = 1 (the default): the replica's slot b0 + r (b0 a multiple
// of 32, r < 32) is formed as b0 | r, so that it folds into the xor of its
// Philox word.  With mul.wide products, measured on GB300: 3D L = 10 1100 ->
// 1130, L = 6 982 -> 986, 2D L = 32 1391 -> 1413, L = 16 1330 -> 1354, 3D L = 8
// 1223 -> 1185 attempts/ns.
#ifndef PA_RS_OR_SLOT
#define PA_RS_OR_SLOT 1
#endif
// Replicas of a group whose Philox blocks are unrolled together.  Measured on
// GB300 (attempts/ns, same bits; 1, 2, 4, 8 unrolled): 3D +-J L = 6 941, 965,
// 962, 964; L = 8 1149, 1160, 1199, 1220; L = 10 1033, 1045, 1050, 1059; 2D
// L = 32 1370, 1419, 1427, 1422; batched, 16 3D +-J L = 8 runs 1217, 1245,
// 1243, 1236.  Two stays the default: the batched form, which runs the
// disorder ensembles, is fastest there.
#ifndef PA_RS_RUNROLL
#define PA_RS_RUNROLL 2
#endif
constexpr int RS_RUNROLL = PA_RS_RUNROLL;
__device__ __forceinline__ void rs_mul(uint32_t m, uint32_t a, uint32_t& hi, uint32_t& lo) {
#if PA_RS_MUL_MODE == 1
    uint64_t p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#else
    hi = __umulhi(m, a);
    lo = m * a;
#endif
}

// Groups of a lane that share one pass over the 32 replicas (PA_RS_KG = 1, 2
// or 4, at most what the lattice's group count fills; see rs_kg below).
// Measured on GB300 (attempts/ns, same bits; up to 1, 2, 4 groups per pass):
// 3D +-J L = 8 1157, 1206, 1208 (two groups fill it); L = 10 1042, 1129, 1232;
// 2D L = 32 1416, 1433, 1502; batched, 16 3D +-J L = 8 runs 1242, 1301, 1302,
// 12 runs of L = 6, 8, 10 1120, 1149, 1168; L = 6 (27 groups, one per lane)
// 961 in every form.
#ifndef PA_RS_KG
#define PA_RS_KG 4
#endif

// KG half-sweep groups of one lane: the sites of pairs 4k .. 4k + 3, colour c,
// for k = k0, k0 + 32, .., k0 + 32 (KG - 1) (those below NGROUPS), 32
// replicas.  Philox of the replicas' blocks, counter (2 g + colour, k, SWEEP |
// instance, slot): round 1 multiplies only words that every block of the
// half-sweep shares (the group index enters word 1 and the slot word 3, both
// by xors); round 2 multiplies one group word (shared by the 32 replicas) and
// one replica word (shared by the groups), round 3 again one of each.  The
// group products are formed once per group, the replica products once per
// replica for all KG groups: a block costs 14 + 2 / KG multiplies.
template <int DIM, int L, bool PMJ, typename KT, int KG>
__device__ __forceinline__ void rs_groups(uint32_t* S, const uint8_t* JS, int k0, int c,
                                          uint32_t g, uint32_t b0, uint32_t ctag, const KT& K,
                                          const SweepCtx& x) {
    using G = RSGeo<DIM, L, PMJ>;
    constexpr int NC = G::NCLS;
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t T[3] = {x.T0, x.T1, x.T2};
    const uint32_t nT[3] = {x.nT0, x.nT1, x.nT2};
    const uint32_t two = x.one << 1;
    uint32_t acc[KG][4][NC];
#pragma unroll
    for (int q = 0; q < KG; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int cl = 0; cl < NC; ++cl) acc[q][i][cl] = 0u;
    const uint32_t c0 = 2u * g + (uint32_t)c;
    const uint32_t y0s = __umulhi(M1, ctag) ^ K.rk0[0];  // round 1, before the xor with k
    const uint32_t y1 = M1 * ctag;
    const uint32_t y2s = __umulhi(M0, c0) ^ K.rk1[0];  // word 2 before the xor with the slot
    const uint32_t y3 = M0 * c0;
    uint32_t z3k[KG], w0s[KG], w1[KG];
#pragma unroll
    for (int q = 0; q < KG; ++q) {
        const uint32_t y0 = y0s ^ (uint32_t)(k0 + 32 * q);
        const uint32_t z2 = __umulhi(M0, y0) ^ y3 ^ K.rk1[1];  // round 2, group half
        z3k[q] = (M0 * y0) ^ K.rk1[2];
        w0s[q] = __umulhi(M1, z2) ^ K.rk0[2];  // round 3, group half
        w1[q] = M1 * z2;
    }
#pragma unroll RS_RUNROLL
    for (int r = 31; r >= 0; --r) {
        // b0 is a multiple of 32 and r < 32: b0 | r is the slot b0 + r
        const uint32_t y2 = PA_RS_OR_SLOT ? y2s ^ (b0 | (uint32_t)r) : y2s ^ (b0 + (uint32_t)r);
        uint32_t h2, z1;
        rs_mul(M1, y2, h2, z1);                                 // round 2, replica half
        const uint32_t z0 = h2 ^ y1 ^ K.rk0[1];
        uint32_t h3, c3r;
        rs_mul(M0, z0, h3, c3r);                                // round 3, replica half
#pragma unroll
        for (int q = 0; q < KG; ++q) {
            uint32_t c0w = w0s[q] ^ z1;
            uint32_t c1w = w1[q];
            uint32_t c2w = h3 ^ z3k[q];
            uint32_t c3w = c3r;
#pragma unroll
            for (int rr = 3; rr < 10; ++rr) {
                const uint32_t a = c0w, b = c2w;
                uint32_t hiA, loA, hiB, loB;
                rs_mul(M0, a, hiA, loA);
                rs_mul(M1, b, hiB, loB);
                c0w = hiB ^ c1w ^ K.rk0[rr];
                c1w = loB;
                c2w = hiA ^ c3w ^ K.rk1[rr];
                c3w = loA;
            }
            const uint32_t w[4] = {c0w, c1w, c2w, c3w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int cl = 0; cl < NC; ++cl)
                    acc[q][i][cl] = ((PA_RS_FMA >> cl) & 1)
                                        ? rs_chain_fma(acc[q][i][cl], w[i], x.one, nT[cl], two)
                                        : rs_chain(acc[q][i][cl], w[i], T[cl]);
        }
    }
    // the FMA form reports T = 0 as "below" for every u: nothing is below 0
#pragma unroll
    for (int cl = 0; cl < NC; ++cl)
        if (((PA_RS_FMA >> cl) & 1) && T[cl] == 0u)
#pragma unroll
            for (int q = 0; q < KG; ++q)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[q][i][cl] = 0xffffffffu;
    // flips: count the unsatisfied bonds of every replica bit-sliced
    uint32_t full[3];
#pragma unroll
    for (int cl = 0; cl < 3; ++cl) full[cl] = (x.full >> cl) & 1u ? 0xffffffffu : 0u;
#pragma unroll
    for (int q = 0; q < KG; ++q) {
        const int k = k0 + 32 * q;
        if (KG > 1 && k >= G::NGROUPS) continue;  // a padding group: its draws go unused
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int s = rs_site<DIM, L>(4 * k + i, c);
            int nb[2 * DIM];
            rs_nbrs<DIM, L>(s, nb);
            const uint32_t W = S[rs_ix(s)];
            uint32_t v[2 * DIM];
            const uint32_t jp = PMJ ? (uint32_t)JS[s] : 0u;
#pragma unroll
            for (int d = 0; d < 2 * DIM; ++d) {
                const uint32_t jm = PMJ ? (0u - ((jp >> d) & 1u)) : 0u;
                v[d] = W ^ S[rs_ix(nb[d])] ^ jm;
            }
            uint32_t b0c, b1c, b2c;
            if constexpr (DIM == 2) {
                const uint32_t s1 = v[0] ^ v[1] ^ v[2], k1 = (v[0] & v[1]) | (v[2] & (v[0] ^ v[1]));
                b0c = s1 ^ v[3];
                const uint32_t k2 = s1 & v[3];
                b1c = k1 ^ k2;
                b2c = k1 & k2;
            } else {
                const uint32_t s1 = v[0] ^ v[1] ^ v[2], k1 = (v[0] & v[1]) | (v[2] & (v[0] ^ v[1]));
                const uint32_t s2 = v[3] ^ v[4] ^ v[5], k2 = (v[3] & v[4]) | (v[5] & (v[3] ^ v[4]));
                b0c = s1 ^ s2;
                const uint32_t k3 = s1 & s2;
                b1c = k1 ^ k2 ^ k3;
                b2c = (k1 & k2) | (k3 & (k1 ^ k2));
            }
            uint32_t flip;
            if constexpr (DIM == 2) {
                const uint32_t alw = b1c | b2c;              // c_u >= 2: dE <= 0
                const uint32_t m0 = b0c & ~b1c & ~b2c;       // c_u = 1: dE = 4
                const uint32_t m1 = ~(b0c | b1c | b2c);      // c_u = 0: dE = 8
                flip = alw | (m0 & (~acc[q][i][0] | full[0])) | (m1 & (~acc[q][i][1] | full[1]));
            } else {
                const uint32_t alw = b2c | (b1c & b0c);      // c_u >= 3
                const uint32_t m0 = b1c & ~b0c & ~b2c;       // c_u = 2: dE = 4
                const uint32_t m1 = b0c & ~b1c & ~b2c;       // c_u = 1: dE = 8
                const uint32_t m2 = ~(b0c | b1c | b2c);      // c_u = 0: dE = 12
                flip = alw | (m0 & (~acc[q][i][0] | full[0])) | (m1 & (~acc[q][i][1] | full[1])) |
                       (m2 & (~acc[q][i][NC - 1] | full[2]));
            }
            S[rs_ix(s)] = W ^ flip;
        }
    }
}

// Groups per pass for a lattice: the largest power of two up to PA_RS_KG whose
// passes keep the lanes as busy as one group per pass does (within 2 %): the
// NGROUPS groups fill ceil(NGROUPS / 32 KG) passes of 32 KG slots.
template <int NGROUPS>
__host__ __device__ constexpr int rs_kg() {
    int best = 1;
    const int per1 = 32 * ((NGROUPS + 31) / 32);
    for (int kg = 2; kg <= PA_RS_KG; kg *= 2) {
        const int per = 32 * kg * ((NGROUPS + 32 * kg - 1) / (32 * kg));
        if (100 * per1 >= 98 * per) best = kg;
    }
    return best;
}

// One chunk of 32 replicas (slots b0 .. b0 + 31, those below R valid): load
// and transpose, theta sweeps, measurement, transpose back and store.
template <int DIM, int L, bool PMJ, typename KT>
__device__ __forceinline__ void rs_chunk(const RunDev& d, const SweepCtx& x, uint32_t b0,
                                         int nsweeps, uint32_t* S, const uint8_t* JS,
                                         const KT& K, int lane, long long& sAbsM,
                                         long long& sM2) {
    using G = RSGeo<DIM, L, PMJ>;
    constexpr int N = G::N;
    const uint32_t slot = b0 + (uint32_t)lane;
    const bool valid = slot < x.R;
    const int nvalid = (int)min(32u, x.R - b0);
    uint8_t* spins = d.spins[x.cur];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(spins + (size_t)slot * d.stride);
    // load: row words of each lane's replica, one ballot per site
    uint32_t keep = 0;
    for (int row = 0; row < G::NROWS; ++row) {
        const uint32_t word = valid ? __ldg(src + row) : 0u;
#pragma unroll
        for (int xx = 0; xx < L; ++xx) {
            const int s = row * L + xx;
            const uint32_t bits = __ballot_sync(0xffffffffu, (word >> xx) & 1u);
            if ((s & 31) == lane) keep = bits;
            if ((s & 31) == 31) S[rs_ix(s - 31 + lane)] = keep;
        }
    }
    if (N & 31) {
        if (lane < (N & 31)) S[rs_ix((N & ~31) + lane)] = keep;
    }
    __syncwarp();
    const uint32_t ctag = x.ctag;
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t g = x.g0 + (uint32_t)t;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            constexpr int KG = rs_kg<G::NGROUPS>();
            for (int k = lane; k < G::NGROUPS; k += 32 * KG)
                rs_groups<DIM, L, PMJ, KT, KG>(S, JS, k, c, g, b0, ctag, K, x);
            __syncwarp();
        }
    }
    // measurement: unsatisfied bonds (s, +d) and spins down, bit-sliced per
    // lane over its sites, then summed per replica
    uint32_t CU[G::KU], CM[G::KM];
#pragma unroll
    for (int k = 0; k < G::KU; ++k) CU[k] = 0u;
#pragma unroll
    for (int k = 0; k < G::KM; ++k) CM[k] = 0u;
    for (int s = lane; s < N; s += 32) {
        int nb[2 * DIM];
        rs_nbrs<DIM, L>(s, nb);
        const uint32_t W = S[rs_ix(s)];
        const uint32_t jp = PMJ ? (uint32_t)JS[s] : 0u;
        rs_count<G::KM>(CM, W);
#pragma unroll
        for (int dd = 0; dd < DIM; ++dd) {
            const uint32_t jm = PMJ ? (0u - ((jp >> (2 * dd)) & 1u)) : 0u;
            rs_count<G::KU>(CU, W ^ S[rs_ix(nb[2 * dd])] ^ jm);
        }
    }
    const uint32_t U = rs_total<G::KU>(CU, lane);
    const uint32_t down = rs_total<G::KM>(CM, lane);
    const int M = N - 2 * (int)down;
    // store: each lane gathers its replica's bits back into row words
    if (nsweeps > 0 && valid) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(spins + (size_t)slot * d.stride);
        for (int row = 0; row < G::NROWS; ++row) {
            uint32_t word = 0;
#pragma unroll
            for (int xx = 0; xx < L; ++xx) word |= ((S[rs_ix(row * L + xx)] >> lane) & 1u) << xx;
            dst[row] = word;
        }
    }
    if (valid) {
        d.ebin[x.cur][slot] = U >> 1;
        d.mag[x.cur][slot] = M;
        if ((U & 1u) != x.parity) atomicOr(&d.st->status, ST_INVARIANT);
    }
    hist_flush(d.hist, U >> 1, nvalid, lane);
    long long a = valid ? (long long)(M < 0 ? -M : M) : 0ll;
    long long q = valid ? (long long)M * M : 0ll;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    sAbsM += a;
    sM2 += q;
    __syncwarp();  // S is reused by the next chunk
}

// Coupling pattern of every site, bit d of JS[s] = J(s, dir d) is -1, dirs
// in the order of rs_nbrs.
template <int DIM, int L>
__device__ __forceinline__ void rs_couplings(const RunDev& d, uint8_t* JS, int lane) {
    constexpr int N = DIM == 2 ? L * L : L * L * L;
    const int nw = (int)d.nwords;
    for (int s = lane; s < N; s += 32) {
        int nb[2 * DIM];
        rs_nbrs<DIM, L>(s, nb);
        uint32_t jp = 0;
#pragma unroll
        for (int dd = 0; dd < DIM; ++dd) {
            const int tp = s, tm = nb[2 * dd + 1];  // bond (s, +d) and bond (s - e_d, +d)
            jp |= ((d.jpk[dd * nw + tp / L] >> (tp % L)) & 1u) << (2 * dd);
            jp |= ((d.jpk[dd * nw + tm / L] >> (tm % L)) & 1u) << (2 * dd + 1);
        }
        JS[s] = (uint8_t)jp;
    }
    __syncwarp();
}

template <int DIM, int L, bool PMJ, int RSW>
__global__ void __launch_bounds__(RSW * 32) k_sweep_rs(__grid_constant__ const RunDev d, int nsweeps) {
    extern __shared__ uint32_t smem[];
    using G = RSGeo<DIM, L, PMJ>;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* S = smem + wib * G::WORDS;
    uint8_t* JS = reinterpret_cast<uint8_t*>(S + G::NS);
    if constexpr (PMJ) rs_couplings<DIM, L>(d, JS, lane);
    const SweepCtx x = sweep_ctx(d);
    const RSKeys K{d.rk0, d.rk1};
    long long sAbsM = 0, sM2 = 0;
    const uint32_t end = min(x.R, d.slot_hi);
    for (uint32_t ch = (d.slot_lo >> 5) + blockIdx.x * RSW + wib; ch * 32u < end;
         ch += gridDim.x * RSW)
        rs_chunk<DIM, L, PMJ, RSKeys>(d, x, ch * 32u, nsweeps, S, JS, K, lane, sAbsM, sM2);
    if (lane == 0 && (sAbsM | sM2)) {
        atomicAdd(&d.accum[0], (unsigned long long)sAbsM);
        atomicAdd(&d.accum[1], (unsigned long long)sM2);
    }
}

// Batched: 32-slot chunks claimed from the class's slot space (run capacities
// are rounded up to 32, so a chunk never straddles two runs).
template <int DIM, int L, bool PMJ, int BW>
__global__ void __launch_bounds__(BW * 32) k_sweep_rs_batched(BatchSweepArgs a) {
    extern __shared__ uint32_t smem[];
    using G = RSGeo<DIM, L, PMJ>;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* S = smem + wib * G::WORDS;
    uint8_t* JS = reinterpret_cast<uint8_t*>(S + G::NS);
    uint32_t* keys = S + G::NS + G::JWORDS;
    uint32_t have = 0xffffffffu;  // run whose keys and couplings are staged
    const RunDev* dp = nullptr;
    long long sAbsM = 0, sM2 = 0;
    for (;;) {
        uint32_t chunk = 0;
        if (lane == 0) chunk = atomicAdd(a.counter, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint32_t g = chunk * 32u;
        if (g >= a.total_slots) break;
        uint32_t lo = 0, hi = a.n;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.slot_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        const uint32_t run = a.run_ids[lo];
        const RunDev& d = a.runs[run];
        if (run != have) {
            if (dp && lane == 0 && (sAbsM | sM2)) {
                atomicAdd(&dp->accum[0], (unsigned long long)sAbsM);
                atomicAdd(&dp->accum[1], (unsigned long long)sM2);
            }
            sAbsM = sM2 = 0;
            have = run;
            dp = &d;
            if (lane < 10) {
                keys[lane] = d.rk0[lane];
                keys[10 + lane] = d.rk1[lane];
            }
            if constexpr (PMJ) rs_couplings<DIM, L>(d, JS, lane);
            __syncwarp();
        }
        const SweepCtx x = sweep_ctx(d);
        const uint32_t b0 = g - a.slot_base[lo];
        if (b0 < x.R) {
            if constexpr (PA_RS_KEYREG) {
                RSKeyRegs K;
#pragma unroll
                for (int r = 0; r < 10; ++r) {
                    K.rk0[r] = keys[r];
                    K.rk1[r] = keys[10 + r];
                }
                rs_chunk<DIM, L, PMJ, RSKeyRegs>(d, x, b0, d.theta, S, JS, K, lane, sAbsM, sM2);
            } else {
                const RSKeys K{keys, keys + 10};
                rs_chunk<DIM, L, PMJ, RSKeys>(d, x, b0, d.theta, S, JS, K, lane, sAbsM, sM2);
            }
        }
    }
    if (dp && lane == 0 && (sAbsM | sM2)) {
        atomicAdd(&dp->accum[0], (unsigned long long)sAbsM);
        atomicAdd(&dp->accum[1], (unsigned long long)sM2);
    }
}

// --------------------------------------------------------------------------
// Initial population (Sec. 2: uniform states at beta0 = 0, or the ground
// state for heating from near T = 0) and couplings.
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
    if (d.init == PA_INIT_GROUND) {  // all spins +1
        reinterpret_cast<uint32_t*>(d.spins[0] + (size_t)slot * d.stride)[w] = 0u;
        return;
    }
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
    int8_t* dst = reinterpret_cast<int8_t*>(d.spins[0] + (size_t)slot * d.stride);
    if (d.init == PA_INIT_GROUND) {  // all spins +1
        for (int j = 0; j < 4; ++j) {
            const int64_t s = 4 * (int64_t)q + j;
            if (s < d.N) dst[s] = 1;
        }
        return;
    }
    const uint4 u = philox(q, 0u, slot, (TAG_INIT << 28) | d.instance, (uint32_t)d.seed,
                           (uint32_t)(d.seed >> 32));
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

// Replica-sliced kernels for the packed layout where they apply (PA_RS = 0
// keeps the row / word kernels, for comparison).
#ifndef PA_RS
#define PA_RS 1
#endif
constexpr int RSW = 4;  // warps per block of the plain replica-sliced kernel

template <int DIM, int L>
constexpr bool rs_applies() {
    return PA_RS && RSGeo<DIM, L, false>::OK;
}

template <int DIM, int L>
KInfo pick_plain(int layout, bool pmj) {
    if constexpr (rs_applies<DIM, L>()) {
        if (layout == PA_LAYOUT_PACKED)
            return {pmj ? (const void*)k_sweep_rs<DIM, L, true, RSW>
                        : (const void*)k_sweep_rs<DIM, L, false, RSW>,
                    RSW * (pmj ? RSGeo<DIM, L, true>::WORDS : RSGeo<DIM, L, false>::WORDS) * 4};
    }
    if (layout == PA_LAYOUT_PACKED) {
        const int smem = WARPS * warp_words<DIM, L, PA_LAYOUT_PACKED>() * 4;
        return {pmj ? (const void*)k_sweep<DIM, L, PA_LAYOUT_PACKED, true>
                    : (const void*)k_sweep<DIM, L, PA_LAYOUT_PACKED, false>,
                smem};
    }
    const int smem = WARPS * warp_words<DIM, L, PA_LAYOUT_INT8>() * 4;
    return {pmj ? (const void*)k_sweep<DIM, L, PA_LAYOUT_INT8, true>
                : (const void*)k_sweep<DIM, L, PA_LAYOUT_INT8, false>,
            smem};
}

template <int DIM, int L, int LAYOUT, int BW>
KInfo pick_batched_w(bool pmj) {
    const int smem = BW * warp_words<DIM, L, LAYOUT>() * 4;
    return {pmj ? (const void*)k_sweep_batched<DIM, L, LAYOUT, true, BW>
                : (const void*)k_sweep_batched<DIM, L, LAYOUT, false, BW>,
            smem};
}

template <int DIM, int L, int BW>
KInfo pick_rs_batched_w(bool pmj) {
    return {pmj ? (const void*)k_sweep_rs_batched<DIM, L, true, BW>
                : (const void*)k_sweep_rs_batched<DIM, L, false, BW>,
            BW * (pmj ? RSGeo<DIM, L, true>::WORDS : RSGeo<DIM, L, false>::WORDS) * 4};
}

template <int DIM, int L>
KInfo pick_batched(int layout, bool pmj, int warps) {
    if constexpr (rs_applies<DIM, L>()) {
        if (layout == PA_LAYOUT_PACKED) {
            if (warps == 2) return pick_rs_batched_w<DIM, L, 2>(pmj);
            if (warps == 4) return pick_rs_batched_w<DIM, L, 4>(pmj);
            if (warps == 8) return pick_rs_batched_w<DIM, L, 8>(pmj);
            return {nullptr, 0};
        }
    }
    if (layout == PA_LAYOUT_PACKED) {
        if (warps == 2) return pick_batched_w<DIM, L, PA_LAYOUT_PACKED, 2>(pmj);
        if (warps == 4) return pick_batched_w<DIM, L, PA_LAYOUT_PACKED, 4>(pmj);
        if (warps == 8) return pick_batched_w<DIM, L, PA_LAYOUT_PACKED, 8>(pmj);
    } else {
        if (warps == 2) return pick_batched_w<DIM, L, PA_LAYOUT_INT8, 2>(pmj);
        if (warps == 4) return pick_batched_w<DIM, L, PA_LAYOUT_INT8, 4>(pmj);
        if (warps == 8) return pick_batched_w<DIM, L, PA_LAYOUT_INT8, 8>(pmj);
    }
    return {nullptr, 0};
}

#define PA_SIZES(X) X(2, 4) X(2, 8) X(2, 16) X(2, 32) X(2, 64) X(2, 128) \
    X(3, 2) X(3, 4) X(3, 6) X(3, 8) X(3, 10) X(3, 12) X(3, 16)

KInfo find_kernel(int layout, int dim, int L, bool pmj) {
#define PA_CASE(D_, L_) \
    if (dim == D_ && L == L_) return pick_plain<D_, L_>(layout, pmj);
    PA_SIZES(PA_CASE)
#undef PA_CASE
    return {nullptr, 0};
}

KInfo find_batched(int layout, int dim, int L, bool pmj, int warps) {
#define PA_CASE(D_, L_) \
    if (dim == D_ && L == L_) return pick_batched<D_, L_>(layout, pmj, warps);
    PA_SIZES(PA_CASE)
#undef PA_CASE
    return {nullptr, 0};
}

int grid_for(const KInfo& k, int threads, int64_t need_blocks) {
    if (!k.fn) return 0;
    if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) !=
        cudaSuccess)
        return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, threads, k.smem) !=
        cudaSuccess)
        return 0;
    if (per_sm < 1) return 0;
    const int64_t full = (int64_t)sms * per_sm;
    if (need_blocks > 0 && need_blocks < full) return (int)need_blocks;
    return (int)full;
}

}  // namespace

bool sweep_supported(int layout, int dim, int L) {
    if (layout != PA_LAYOUT_INT8 && layout != PA_LAYOUT_PACKED) return false;
    return find_kernel(layout, dim, L, false).fn != nullptr;
}

// Replica-sliced kernels take 32 replicas per warp.
bool rs_kernel(const RunDev& d) {
    if (d.layout != PA_LAYOUT_PACKED) return false;
#define PA_CASE(D_, L_) \
    if (d.dim == D_ && d.L == L_) return rs_applies<D_, L_>();
    PA_SIZES(PA_CASE)
#undef PA_CASE
    return false;
}

int sweep_grid(const RunDev& d) {
    if (l64_applies(d)) return l64_grid(d);
    const KInfo k = find_kernel(d.layout, d.dim, d.L, d.model == PA_MODEL_PMJ);
    const int64_t per_block = rs_kernel(d) ? 32 * RSW : WARPS;
    return grid_for(k, WARPS * 32, ((int64_t)d.cap + per_block - 1) / per_block);
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

bool batched_warps_valid(const RunDev& proto, int warps) {
    if (l64_batched_applies(proto)) return true;
    return find_batched(proto.layout, proto.dim, proto.L, proto.model == PA_MODEL_PMJ, warps).fn !=
           nullptr;
}

int batched_sweep_grid(const RunDev& proto, int warps) {
    if (l64_batched_applies(proto)) return l64_batched_grid(proto);
    const KInfo k = find_batched(proto.layout, proto.dim, proto.L, proto.model == PA_MODEL_PMJ, warps);
    return grid_for(k, warps * 32, 0);
}

cudaError_t launch_sweep_batched(const BatchSweepArgs& a, const RunDev& proto, int warps, int grid,
                                 cudaStream_t s) {
    if (l64_batched_applies(proto)) return launch_sweep_l64_batched(a, proto, grid, s);
    const KInfo k = find_batched(proto.layout, proto.dim, proto.L, proto.model == PA_MODEL_PMJ, warps);
    if (!k.fn) return cudaErrorInvalidValue;
    BatchSweepArgs aa = a;
    void* args[] = {&aa};
    return cudaLaunchKernel(k.fn, dim3(grid), dim3(warps * 32), args, (size_t)k.smem, s);
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
