// pa_sweep_l64.cu -- Metropolis sweeps of the 2D Ising ferromagnet (Eq. 6) at
// L = 64, the workload of the paper's tests (Sec. 3 and 4), bit-packed one
// 64-site row per 64-bit word.
//
// Same update rule and random numbers as the generic kernels of pa_sweep.cu
// (checkerboard order, dE = 4 (2 - c_u), u = word h & 3 of the Philox block
// with counter (2 g + colour, h >> 2, SWEEP | instance, slot), h = s >> 1, accept iff
// dE <= 0 or u < T(beta_i, dE)), mapped for throughput:
//   * one warp holds one replica for all theta sweeps, entirely in registers:
//     lane l owns rows 2l and 2l+1 (one 16-byte load per lane, coalesced);
//   * vertical neighbours come from the adjacent lanes by warp shuffle,
//     horizontal ones by a 64-bit rotate; the unsatisfied-bond count of all
//     64 sites of a row is evaluated bit-sliced (a handful of word ops);
//   * a row holds 32 sites of each colour = 8 Philox blocks, each block
//     covering 4 sites of that row, and both acceptance tests (dE = 4 and 8)
//     are folded into two bit masks in registers, with no atomics;
//   * each test is a carry chain: the carry out of u - T is [u >= T], and an
//     add with carry-in shifts it into an accumulator that holds both tests
//     of 16 sites (two instructions per test, no predicates or selects; the
//     FMA pipe is left to the Philox multiplies);
//   * the Philox round keys come from the kernel parameters; the products
//     shared by all blocks of a half-sweep are formed once per half-sweep; the
//     round-2 block products, which depend only on the run and the block
//     index, and the round-3 block products, which depend only on the run,
//     the block index and the half-sweep, once per CTA into shared-memory
//     tables: a block costs 14 of Philox's 20 multiplies.
// Grid-stride (persistent) over replicas; the population size is read from
// device memory.  The measurement epilogue is the one of the generic kernel.
#include "pa_internal.cuh"

namespace pa {
namespace {

// Tuning knobs (compile time): warps per block and the resident blocks per SM
// the register budget is sized for; the forms of the threshold tests are the
// PA_L64_CHAIN and PA_L64_SEL_BLOCKS knobs further down.
#ifndef PA_L64_MIN_BLOCKS
#define PA_L64_MIN_BLOCKS 1
#endif

// How the Philox products are formed: 0 = high and low halves from C++
// (__umulhi, *), 1 = one mul.wide.u32, 2 = separate mul.hi.u32 / mul.lo.u32.
#ifndef PA_L64_MUL_MODE
#define PA_L64_MUL_MODE 1
#endif

// Warps per block (one block per SM).  With both groups of a row unrolled,
// measured on GB300 (attempts/ns, same bits): 16 warps (125 registers) 1671,
// 12 warps (152) 1686, 8 warps (212) 1653 (ferromagnet, 2^21 replicas); +-J
// 2^20: 1626, 1636, 1611; batched, 8 +-J runs of 2^17: 1597, 1632, 1604.
// With the Philox tables (fewer registers) 16 warps ran at 1755 against 1749
// (ferromagnet) and 1704 against 1712 (+-J): 12 stays.
#ifndef PA_L64_WARPS
#define PA_L64_WARPS 12
#endif
constexpr int WARPS64 = PA_L64_WARPS;

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Threshold of one energy class for the current step: u < T accepts.
struct Thr {
    uint32_t T;
};

// Philox4x32-10 of the blocks (c0, c1, ctag, slot) of one half-sweep of one
// replica, with c0 = 2 g + colour, c1 = h >> 2 the block index and ctag =
// SWEEP | instance.  Round 1 multiplies c0 and ctag (both shared); c1 enters
// word 0 by an xor, so round 2 multiplies one block word (M0 * word 0) and one
// shared word, round 3 again one of each (M1 * word 2, M0 * word 0 shared),
// and rounds 4..10 are the plain rounds.  The shared products are formed once
// per half-sweep (HalfSweepGen), the round-2 block product once per run and
// the round-3 block product once per launch (cta_tables): 14 multiplies per
// block; 15 in the batched kernel, whose warps serve several runs and keep
// per-warp round-2 tables (round2_table).  Same bits as philox().
constexpr uint32_t PM0 = 0xD2511F53u, PM1 = 0xCD9E8D57u;

// Round keys of the run's seed and the opaque 1 of the multiply-add tests:
// kernel parameters in the plain kernel, a per-warp shared-memory copy of the
// chunk's run in the batched one.
struct Keys {
    const uint32_t* rk0;
    const uint32_t* rk1;
    uint32_t one;
    const uint2* r2;  // the lane's column of the run's round-2 table (entry j at r2[32 j])
    const uint2* t3;  // the lane's column of the step's round-3 table, or null (entry
                      // (hs, j) at t3[512 hs + 32 j] for half-sweep hs of the launch)
};

__device__ __forceinline__ void mul_hilo(uint32_t m, uint32_t a, uint32_t& hi, uint32_t& lo) {
#if PA_L64_MUL_MODE == 1
    uint64_t p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#elif PA_L64_MUL_MODE == 2
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(hi) : "r"(a), "r"(m));
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(lo) : "r"(a), "r"(m));
#else
    hi = __umulhi(m, a);
    lo = m * a;
#endif
}

struct HalfSweepGen {
    const uint2* t3;  // this half-sweep's slice of the lane's round-3 table column (or null)
    uint32_t y0k;  // round-1 word 0 before the xor with c1: high half of M1 * ctag ^ key 0
    uint32_t y3k;  // round-1 word 3 (low half of M0 * c0) ^ round-2 key 1
    uint32_t z1k;  // round-2 word 1 ^ round-3 key 0
    uint32_t e2k;  // high half of M0 * (round-2 word 0) ^ round-3 key 1
    uint32_t e3;   // low half of M0 * (round-2 word 0): round-3 word 3
};

__device__ __forceinline__ HalfSweepGen half_sweep_gen(const Keys& d, uint32_t c0, uint32_t slot,
                                                      uint32_t ctag) {
    HalfSweepGen g;
    g.t3 = nullptr;
    uint32_t ht, lt, hc, lc;
    mul_hilo(PM1, ctag, ht, lt);  // round 1
    mul_hilo(PM0, c0, hc, lc);
    g.y0k = ht ^ d.rk0[0];
    g.y3k = lc ^ d.rk1[1];
    const uint32_t y2 = hc ^ slot ^ d.rk1[0];
    uint32_t h2, l2;
    mul_hilo(PM1, y2, h2, l2);  // round 2, shared half
    const uint32_t z0 = h2 ^ lt ^ d.rk0[1];
    g.z1k = l2 ^ d.rk0[2];
    uint32_t h3, l3;
    mul_hilo(PM0, z0, h3, l3);  // round 3, shared half
    g.e2k = h3 ^ d.rk1[2];
    g.e3 = l3;
    return g;
}

// The round-2 block product M0 * (hi(M1 * ctag) ^ key0 ^ c1) depends only on
// the run (its tag, instance and key) and the block index c1, not on the
// half-sweep or the replica: each lane forms those of its NB blocks
// c1 = NB * lane + j once per run, into its column of a shared-memory table
// (entry j at col[32 j], so the lanes of a warp touch consecutive words), and
// a block then costs 15 of Philox's 20 multiplies.
template <uint32_t NB>
__device__ __forceinline__ void round2_table(uint2* col, uint32_t lane, uint32_t ctag,
                                             const uint32_t* rk0) {
    uint32_t ht, lt;
    mul_hilo(PM1, ctag, ht, lt);  // round 1
    const uint32_t y0k = ht ^ rk0[0];
#pragma unroll 1
    for (uint32_t j = 0; j < NB; ++j) {
        uint32_t h, l;
        mul_hilo(PM0, y0k ^ (NB * lane + j), h, l);  // round 2, block half
        col[32u * j] = make_uint2(h, l);
    }
}

// The round-3 block product M1 * (h2(c1) ^ lo(M0 * c0) ^ key) depends only on
// the run, the block index and the half-sweep, not on the replica: the plain
// L = 64 kernel forms those of every block and half-sweep of its launch once
// per CTA into a second table (T3), and a block then costs 14 multiplies.

// Block c1 of the half-sweep: with NB > 0 c1 is one of the lane's NB table
// blocks and its round-2 product comes from the table (NB = 0 forms it); with
// T3 its round-3 product comes from the half-sweep's slice of the step table.
template <uint32_t NB, bool T3 = false>
__device__ __forceinline__ uint4 philox_block(const Keys& d, const HalfSweepGen& g, uint32_t c1) {
    uint32_t l2, h3, l3;
    if constexpr (T3) {
        static_assert(NB > 0, "the step table needs the round-2 table");
        const uint32_t j = c1 & (NB - 1u);
        const uint2 w = g.t3[32u * j];  // round 3, block half (step table)
        h3 = w.x;
        l3 = w.y;
        l2 = d.r2[32u * j].y;  // round 2, block half (run table)
    } else {
        uint2 r2;
        if constexpr (NB > 0) {
            r2 = d.r2[32u * (c1 & (NB - 1u))];  // round 2, block half (table)
        } else {
            mul_hilo(PM0, g.y0k ^ c1, r2.x, r2.y);  // round 2, block half
        }
        l2 = r2.y;
        mul_hilo(PM1, r2.x ^ g.y3k, h3, l3);  // round 3, block half
    }
    uint32_t c0 = h3 ^ g.z1k;
    uint32_t c1w = l3;
    uint32_t c2 = l2 ^ g.e2k;
    uint32_t c3 = g.e3;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint32_t a = c0, b = c2;
        uint32_t hiA, loA, hiB, loB;
        mul_hilo(PM0, a, hiA, loA);
        mul_hilo(PM1, b, hiB, loB);
        c0 = hiB ^ c1w ^ d.rk0[r];
        c1w = loB;
        c2 = hiA ^ c3 ^ d.rk1[r];
        c3 = loA;
    }
    return make_uint4(c0, c1w, c2, c3);
}

// Both tests of one site into a shared accumulator, two bits per site:
// acc = 4 acc + 2 c4 + c8, where c is the carry of the compare, written by
// mad.lo.cc (FMA pipe: u * 1 + (2^32 - T) carries iff u >= T, for T > 0) or
// by sub.cc (ALU pipe: u + ~T + 1 carries iff u >= T, for every T), and
// shifted in by addc (ALU pipe).
template <bool F4, bool F8>
__device__ __forceinline__ uint32_t site_chain(uint32_t acc, uint32_t u, uint32_t one,
                                               uint32_t c4, uint32_t c8) {
    uint32_t out;
    if constexpr (F4 && F8)
        asm("{\n\t.reg .u32 t, a;\n\tmad.lo.cc.u32 t, %1, %2, %3;\n\taddc.u32 a, %4, %4;"
            "\n\tmad.lo.cc.u32 t, %1, %2, %5;\n\taddc.u32 %0, a, a;\n\t}"
            : "=r"(out) : "r"(u), "r"(one), "r"(c4), "r"(acc), "r"(c8));
    else if constexpr (F4)
        asm("{\n\t.reg .u32 t, a;\n\tmad.lo.cc.u32 t, %1, %2, %3;\n\taddc.u32 a, %4, %4;"
            "\n\tsub.cc.u32 t, %1, %5;\n\taddc.u32 %0, a, a;\n\t}"
            : "=r"(out) : "r"(u), "r"(one), "r"(c4), "r"(acc), "r"(c8));
    else if constexpr (F8)
        asm("{\n\t.reg .u32 t, a;\n\tsub.cc.u32 t, %1, %3;\n\taddc.u32 a, %4, %4;"
            "\n\tmad.lo.cc.u32 t, %1, %2, %5;\n\taddc.u32 %0, a, a;\n\t}"
            : "=r"(out) : "r"(u), "r"(one), "r"(c4), "r"(acc), "r"(c8));
    else
        asm("{\n\t.reg .u32 t, a;\n\tsub.cc.u32 t, %1, %3;\n\taddc.u32 a, %4, %4;"
            "\n\tsub.cc.u32 t, %1, %5;\n\taddc.u32 %0, a, a;\n\t}"
            : "=r"(out) : "r"(u), "r"(one), "r"(c4), "r"(acc), "r"(c8));
    return out;
}

// PA_L64_CHAIN (1..4): both tests of a site go into one accumulator
// (site_chain), each compare on the FMA or the ALU pipe.  3 (both on the ALU,
// the default) ran 7.5 % faster on GB300 than separate accumulators per test
// with FMA-pipe chains, and 17 % faster than compare and select.
#ifndef PA_L64_CHAIN
#define PA_L64_CHAIN 3
#endif
static_assert(PA_L64_CHAIN >= 1 && PA_L64_CHAIN <= 4, "PA_L64_CHAIN: 1 .. 4");

// PA_L64_SEL_BLOCKS (0..3): with the chains of PA_L64_CHAIN, the tests of
// the last that many blocks of every group of four (h < PA_L64_SEL_BLOCKS)
// run as compare and select instead, instructions that only the ALU pipe
// executes; the carry chains are integer adds, which the compiler may move
// to the FMA pipe.
// PA_L64_OR_INDEX = 1: the block index base + h (base a multiple of 4, h =
// 0 .. 3) is formed as base | h, the same value, so that it folds into the
// xor of the round-2 word as one three-input logic op on the ALU pipe.
#ifndef PA_L64_OR_INDEX
#define PA_L64_OR_INDEX 0
#endif
#if PA_L64_OR_INDEX
#define PA_L64_BLOCK(base, h) ((base) | (uint32_t)(h))
#else
#define PA_L64_BLOCK(base, h) ((base) + (uint32_t)(h))
#endif

// Philox blocks of a group of four unrolled together in the L = 64 kernel.
#ifndef PA_L64_HUNROLL
#define PA_L64_HUNROLL 4
#endif
// Groups of four blocks unrolled together (a row's colour sites are two groups
// at L = 64 and four at L = 128).  Measured on GB300, same bits: at L = 64
// both groups together (125 registers, no spills) run at 1674 attempts/ns
// against 1606 one at a time (ferromagnet, 2^21 replicas), 1631 against 1575
// (+-J, 2^20) and 1601 against 1557 (batched, 8 +-J runs of 2^17); with two
// Philox blocks per group unrolled instead of four, 1573.  At L = 128 two of
// the four groups together run at 1484 against 1437 (ferromagnet, 12 warps,
// 166 registers) and 1497 against 1361 (+-J, 8 warps); all four spill.  All
// four groups with two blocks each unrolled (125 registers) run at 1462, 1491
// and 1509 with 8, 12 and 16 warps (+-J 1420 at every width), against 1512 to
// 1520 for two groups of four blocks at 8 warps.
#ifndef PA_L64_QUNROLL
#define PA_L64_QUNROLL 2
#endif
#ifndef PA_L128_QUNROLL
#define PA_L128_QUNROLL 2
#endif
constexpr int L64_QUNROLL = PA_L64_QUNROLL, L128_QUNROLL = PA_L128_QUNROLL;

#ifndef PA_L64_SEL_BLOCKS
#define PA_L64_SEL_BLOCKS 0
#endif
static_assert(PA_L64_SEL_BLOCKS >= 0 && PA_L64_SEL_BLOCKS < 4, "PA_L64_SEL_BLOCKS: 0 .. 3");

// The tests of one group of four Philox blocks (block(h), h = 3 .. 0): the
// carries [u >= T4], [u >= T8] of site j = 4h + m end at bits 2j + 1, 2j.
// Chain blocks come first (the chain shifts its accumulator by two bits per
// site), then the compare-and-select blocks OR their bits in place.
template <bool F4, bool F8, int UNROLL, typename Block>
__device__ __forceinline__ uint32_t group_tests(const Block& block, uint32_t one, uint32_t c4,
                                                uint32_t c8, uint32_t T4, uint32_t T8) {
    constexpr int XS = PA_L64_SEL_BLOCKS;
    uint32_t kc = 0;
#pragma unroll UNROLL
    for (int h = 3; h >= XS; --h) {
        const uint4 u = block(h);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int m = 3; m >= 0; --m) kc = site_chain<F4, F8>(kc, w[m], one, c4, c8);
    }
    if constexpr (XS > 0) {
        kc <<= 8 * XS;
#pragma unroll
        for (int h = XS - 1; h >= 0; --h) {
            const uint4 u = block(h);
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * h + m;
                kc |= (w[m] >= T4 ? 2u << (2 * j) : 0u) | (w[m] >= T8 ? 1u << (2 * j) : 0u);
            }
        }
    }
    return kc;
}

// Acceptance masks of the 32 colour-c sites of row y, P = (y + c) & 1: sites
// x = 8j + 2m + P take word m of Philox block 8y + j; bit x of a4 / a8 is set
// when that uniform is below T4 / T8.  Four blocks per iteration fill one
// 32-bit half of each mask.
template <int P, bool T3>
__device__ __forceinline__ void row_accepts(const Keys& d, const HalfSweepGen& gen, uint32_t y,
                                            const Thr& t4, const Thr& t8, uint64_t& a4,
                                            uint64_t& a8) {
    const uint32_t one = d.one;
    // PA_L64_CHAIN: 1 both compares on the FMA pipe, 2 dE = 4 on the FMA pipe
    // and dE = 8 on the ALU, 3 both on the ALU, 4 the reverse of 2
    constexpr bool F4 = PA_L64_CHAIN == 1 || PA_L64_CHAIN == 2;
    constexpr bool F8 = PA_L64_CHAIN == 1 || PA_L64_CHAIN == 4;
    const uint32_t c4 = F4 ? 0u - t4.T : t4.T, c8 = F8 ? 0u - t8.T : t8.T;
    uint32_t h4[2], h8[2];
#pragma unroll L64_QUNROLL
    for (uint32_t q = 0; q < 2; ++q) {
        const uint32_t base = 8u * y + 4u * q;
        const uint32_t kc = group_tests<F4, F8, PA_L64_HUNROLL>(
            [&](int h) { return philox_block<16, T3>(d, gen, PA_L64_BLOCK(base, h)); }, one, c4, c8, t4.T,
            t8.T);
        // site j = 4h + m: dE = 4 carry at bit 2j + 1, dE = 8 carry at bit 2j
        constexpr uint32_t EV = 0x55555555u;
        const uint32_t r4 = (kc >> 1) & EV, r8 = kc & EV;
        // a carry is [u >= T]; below is its complement (T = 0 on the FMA
        // form carries never, and nothing is below it)
        const uint32_t b4 = (F4 && !t4.T) ? 0u : (~r4 & EV);
        const uint32_t b8 = (F8 && !t8.T) ? 0u : (~r8 & EV);
        if (q == 0) {
            h4[0] = b4 << P;
            h8[0] = b8 << P;
        } else {
            h4[1] = b4 << P;
            h8[1] = b8 << P;
        }
    }
    a4 = ((uint64_t)h4[1] << 32) | h4[0];
    a8 = ((uint64_t)h8[1] << 32) | h8[0];
}

// +-J couplings of one row (bit x set: J = -1) for its four bonds: to x + 1,
// to x - 1, to y - 1 and to y + 1.  All zero for the ferromagnet.
struct RowJ {
    uint64_t xp, xm, up, dn;
};

// Flip mask of the colour sites (parity P) of one row, given the rows above
// and below.  c_u >= 2 flips outright (dE <= 0); c_u = 1 needs u < T4; c_u = 0
// needs u < T8.  full bit 0 / 1: T4 / T8 equal 2^32 (beta = 0), always accept.
// A bond is unsatisfied when the spins' xor differs from its coupling bit.
template <int P, bool PMJ, bool T3>
__device__ __forceinline__ uint64_t row_flips(const Keys& d, const HalfSweepGen& gen,
                                              uint64_t own, uint64_t up, uint64_t dn, uint32_t y,
                                              const Thr& t4, const Thr& t8, uint32_t full,
                                              const RowJ& j) {
    constexpr uint64_t cm = P ? 0xAAAAAAAAAAAAAAAAull : 0x5555555555555555ull;
    uint64_t a4, a8;
    row_accepts<P, T3>(d, gen, y, t4, t8, a4, a8);
    uint64_t a = own ^ ((own >> 1) | (own << 63));  // bond to x + 1
    uint64_t b = own ^ ((own << 1) | (own >> 63));  // bond to x - 1
    uint64_t e = own ^ up;
    uint64_t f = own ^ dn;
    if constexpr (PMJ) {
        a ^= j.xp;
        b ^= j.xm;
        e ^= j.up;
        f ^= j.dn;
    }
    const uint64_t s1 = a ^ b, s2 = e ^ f;
    const uint64_t ge2 = (a & b) | (e & f) | (s1 & s2);
    const uint64_t zero = ~(a | b | e | f);
    const uint64_t one = (s1 ^ s2) & ~ge2;
    if (full & 1u) a4 = ~0ull;
    if (full & 2u) a8 = ~0ull;
    return (ge2 | (one & a4) | (zero & a8)) & cm;
}

__device__ __forceinline__ void hist_flush(uint32_t* hist, uint32_t level, int n, int lane) {
    if (n <= 0) return;
    const unsigned valid = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
    if (lane < n) {
        const unsigned peers = __match_any_sync(valid, level);
        if (lane == __ffs(peers) - 1) atomicAdd(&hist[level], (uint32_t)__popc(peers));
    }
}

// Couplings of lane l's rows 2l and 2l + 1 from the packed tables (J(+x) and
// J(+y) bit-planes, two 32-bit words per row).
__device__ __forceinline__ void l64_couplings(const RunDev& d, int lane, RowJ& ja, RowJ& jb) {
    const uint32_t* jx = d.jpk;
    const uint32_t* jy = d.jpk + d.nwords;
    auto row = [](const uint32_t* t, int y) { return ((uint64_t)t[2 * y + 1] << 32) | t[2 * y]; };
    auto rot_m = [](uint64_t v) { return (v << 1) | (v >> 63); };  // bit x <- bit x - 1
    const int ya = 2 * lane, yb = ya + 1;
    const uint64_t xa = row(jx, ya), xb = row(jx, yb);
    ja = RowJ{xa, rot_m(xa), row(jy, (ya + 63) & 63), row(jy, ya)};
    jb = RowJ{xb, rot_m(xb), row(jy, ya), row(jy, yb)};
}

// One replica: theta sweeps in registers, then the measurement.  Returns U
// (all lanes), M through the reference; writes the replica back.
template <bool PMJ, bool T3>
__device__ __forceinline__ uint32_t l64_replica(const Keys& K, uint4* spins, uint32_t slot,
                                                int nsweeps, uint32_t g0, uint32_t ctag,
                                                const Thr& t4, const Thr& t8, uint32_t full,
                                                int lane, int& M, const RowJ& ja, const RowJ& jb) {
    const uint32_t ya = 2u * (uint32_t)lane, yb = ya + 1u;
    const int lup = (lane + 31) & 31, ldn = (lane + 1) & 31;
    const uint4 v = spins[(size_t)slot * 32 + lane];
    uint64_t ra = ((uint64_t)v.y << 32) | v.x;  // row ya
    uint64_t rb = ((uint64_t)v.w << 32) | v.z;  // row yb
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t g = g0 + (uint32_t)t;
        {  // colour 0: even rows have parity 0, odd rows parity 1
            const uint64_t up = shfl64(rb, lup);  // row ya - 1
            const uint64_t dn = shfl64(ra, ldn);  // row yb + 1
            HalfSweepGen gen = half_sweep_gen(K, 2u * g, slot, ctag);
            if constexpr (T3) gen.t3 = K.t3 + (size_t)(2 * t) * 512;
            const uint64_t fa = row_flips<0, PMJ, T3>(K, gen, ra, up, rb, ya, t4, t8, full, ja);
            const uint64_t fb = row_flips<1, PMJ, T3>(K, gen, rb, ra, dn, yb, t4, t8, full, jb);
            ra ^= fa;
            rb ^= fb;
        }
        {  // colour 1
            const uint64_t up = shfl64(rb, lup);
            const uint64_t dn = shfl64(ra, ldn);
            HalfSweepGen gen = half_sweep_gen(K, 2u * g + 1u, slot, ctag);
            if constexpr (T3) gen.t3 = K.t3 + (size_t)(2 * t + 1) * 512;
            const uint64_t fa = row_flips<1, PMJ, T3>(K, gen, ra, up, rb, ya, t4, t8, full, ja);
            const uint64_t fb = row_flips<0, PMJ, T3>(K, gen, rb, ra, dn, yb, t4, t8, full, jb);
            ra ^= fa;
            rb ^= fb;
        }
    }
    // measurement: bonds to x + 1 and to y + 1 of both rows
    const uint64_t dn = shfl64(ra, ldn);
    uint32_t U = __popcll(ra ^ ((ra >> 1) | (ra << 63)) ^ ja.xp) + __popcll(ra ^ rb ^ ja.dn) +
                 __popcll(rb ^ ((rb >> 1) | (rb << 63)) ^ jb.xp) + __popcll(rb ^ dn ^ jb.dn);
    uint32_t down = __popcll(ra) + __popcll(rb);
    U = warp_sum(U);
    down = warp_sum(down);
    M = 4096 - 2 * (int)down;
    if (nsweeps > 0)  // a measurement alone leaves the replica as it is
        spins[(size_t)slot * 32 + lane] =
            make_uint4((uint32_t)ra, (uint32_t)(ra >> 32), (uint32_t)rb, (uint32_t)(rb >> 32));
    return U;
}

struct L64Tally {
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

__device__ __forceinline__ void thresholds(const RunDev& d, uint32_t step, Thr& t4, Thr& t8,
                                           uint32_t& full) {
    t4.T = d.thr[step * 4 + 0];
    t8.T = d.thr[step * 4 + 1];
    full = d.thr[step * 4 + 3];
}

// The run's round-2 table of a CTA, entry j * 32 + l for block 16 l + j, and
// with T3 the launch's round-3 table after it, entry (hs * 16 + j) * 32 + l for
// block 16 l + j in half-sweep hs = 2 t + colour of sweep g0 + t (c0 = 2 g0 + hs),
// formed by all threads of the CTA (which all serve one run).
template <bool T3>
__device__ __forceinline__ void cta_tables(uint2* tab, uint32_t ctag, uint32_t g0, int nsweeps,
                                           const uint32_t* rk0, const uint32_t* rk1) {
    uint32_t ht, lt;
    mul_hilo(PM1, ctag, ht, lt);  // round 1
    const uint32_t y0k = ht ^ rk0[0];
    for (uint32_t e = threadIdx.x; e < 512u; e += blockDim.x) {
        uint32_t h, l;
        mul_hilo(PM0, y0k ^ (16u * (e & 31u) + (e >> 5)), h, l);  // round 2, block half
        tab[e] = make_uint2(h, l);
    }
    if constexpr (T3) {
        __syncthreads();
        const uint32_t n = 2u * (uint32_t)nsweeps * 512u;
        for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
            uint32_t hc, lc, h, l;
            mul_hilo(PM0, 2u * g0 + (e >> 9), hc, lc);  // round 1: M0 * c0
            mul_hilo(PM1, tab[e & 511u].x ^ lc ^ rk1[1], h, l);  // round 3, block half
            tab[512u + e] = make_uint2(h, l);
        }
    }
    __syncthreads();
}

template <bool PMJ, bool T3>
__global__ void __launch_bounds__(WARPS64 * 32, PA_L64_MIN_BLOCKS)
    k_sweep_l64(__grid_constant__ const RunDev d, int nsweeps) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    DevState* st = d.st;
    const uint32_t R = st->R;
    const uint32_t cur = st->cur;
    const uint32_t g0 = st->sweep_base;
    Thr t4, t8;
    uint32_t full;
    thresholds(d, st->step, t4, t8, full);
    const uint32_t ctag = (TAG_SWEEP << 28) | d.instance;
    extern __shared__ uint2 s_tab[];  // 512 round-2 products, then (T3) 2 nsweeps x 512 round-3
    cta_tables<T3>(s_tab, ctag, g0, nsweeps, d.rk0, d.rk1);
    const Keys K{d.rk0, d.rk1, d.one, s_tab + lane, T3 ? s_tab + 512 + lane : nullptr};
    uint4* spins = reinterpret_cast<uint4*>(d.spins[cur]);
    RowJ ja{0, 0, 0, 0}, jb{0, 0, 0, 0};
    if constexpr (PMJ) l64_couplings(d, lane, ja, jb);
    const uint32_t parity = st->negbonds & 1u;
    L64Tally tally;
    const uint32_t nwarps = gridDim.x * WARPS64;
    const uint32_t end = min(R, d.slot_hi);
    for (uint32_t slot = d.slot_lo + blockIdx.x * WARPS64 + wib; slot < end; slot += nwarps) {
        int M = 0;
        const uint32_t U =
            l64_replica<PMJ, T3>(K, spins, slot, nsweeps, g0, ctag, t4, t8, full, lane, M, ja, jb);
        if (lane == 0) {
            d.ebin[cur][slot] = U >> 1;
            d.mag[cur][slot] = M;
            if ((U & 1u) != parity) atomicOr(&st->status, ST_INVARIANT);
        }
        tally.add(d.hist, U, M, lane);
    }
    tally.finish(d.hist, d.accum, lane);
}

// Batched: chunks of a.chunk slots of one run from a class's slot space.
template <bool PMJ>
__global__ void __launch_bounds__(WARPS64 * 32, PA_L64_MIN_BLOCKS) k_sweep_l64_batched(BatchSweepArgs a) {
    __shared__ uint32_t s_keys[WARPS64][24];
    extern __shared__ uint2 s_r2[];  // WARPS64 x 16 x 32 round-2 products
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint2* col = s_r2 + (size_t)wib * 16 * 32 + lane;
    uint32_t have = 0xffffffffu;  // run whose round-2 table the warp holds
    L64Tally tally;
    for (;;) {
        uint32_t chunk = 0;
        if (lane == 0) chunk = atomicAdd(a.counter, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint32_t g = chunk * a.chunk;
        if (g >= a.total_slots) break;
        uint32_t lo = 0, hi = a.n;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.slot_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        const RunDev& d = a.runs[a.run_ids[lo]];
        DevState* st = d.st;
        const uint32_t R = st->R, cur = st->cur, g0 = st->sweep_base;
        Thr t4, t8;
        uint32_t full;
        thresholds(d, st->step, t4, t8, full);
        if (lane < 10) {
            s_keys[wib][lane] = d.rk0[lane];
            s_keys[wib][10 + lane] = d.rk1[lane];
        }
        __syncwarp();
        const uint32_t ctag = (TAG_SWEEP << 28) | d.instance;
        if (a.run_ids[lo] != have) {
            round2_table<16>(col, (uint32_t)lane, ctag, &s_keys[wib][0]);
            have = a.run_ids[lo];
        }
        const Keys K{&s_keys[wib][0], &s_keys[wib][10], d.one, col};
        uint4* spins = reinterpret_cast<uint4*>(d.spins[cur]);
        const uint32_t first = g - a.slot_base[lo];
        RowJ ja{0, 0, 0, 0}, jb{0, 0, 0, 0};
        if constexpr (PMJ) l64_couplings(d, lane, ja, jb);
        const uint32_t parity = st->negbonds & 1u;
        for (uint32_t slot = first; slot < first + a.chunk && slot < R; ++slot) {
            int M = 0;
            const uint32_t U =
                l64_replica<PMJ, false>(K, spins, slot, d.theta, g0, ctag, t4, t8, full, lane, M, ja,
                                        jb);
            if (lane == 0) {
                d.ebin[cur][slot] = U >> 1;
                d.mag[cur][slot] = M;
                if ((U & 1u) != parity) atomicOr(&st->status, ST_INVARIANT);
            }
            tally.add(d.hist, U, M, lane);
        }
        tally.finish(d.hist, d.accum, lane);
        __syncwarp();
    }
}

// --------------------------------------------------------------------------
// L = 128: the same scheme with a row of two 64-bit words (lo: x = 0..63,
// hi: x = 64..127) and four rows per lane (rows 4l .. 4l + 3, one coalesced
// 64-byte span per lane).  A row has 64 sites of each colour = 16 Philox
// blocks (16y .. 16y + 15), taken in four groups of four blocks, each group
// filling one 32-bit quarter of the row's masks.  Rows are updated in place
// one after the other: the sites a half-sweep flips have the active colour,
// and the classes of active-colour sites depend only on the other colour.
// Each block forms its round-2 product (16 multiplies per block).  Tables of
// them as in the L = 64 kernel ran slower on GB300: per warp (128 KB per
// block) 1490 against 1508 attempts/ns, and one per CTA (16 KB) 1504-1507
// (ferromagnet) and 1476-1479 against 1495-1497 (+-J).
// --------------------------------------------------------------------------
// Block warps: with two groups unrolled, the ferromagnet runs at 1508 to 1517
// attempts/ns with 8 warps (183 registers) against 1484 with 12 (166
// registers) on GB300, 2^19 replicas; the +-J kernel holds eight rows of
// couplings more and keeps 8 warps (12 spill).
#ifndef PA_L128_WARPS
#define PA_L128_WARPS 8
#endif
#ifndef PA_L128_WARPS_PMJ
#define PA_L128_WARPS_PMJ 8
#endif
// Philox blocks of a group unrolled together (registers against latency).
#ifndef PA_L128_HUNROLL
#define PA_L128_HUNROLL 4
#endif
constexpr int L128_HUNROLL = PA_L128_HUNROLL;
template <bool PMJ>
__host__ __device__ constexpr int warps128() {
    return PMJ ? PA_L128_WARPS_PMJ : PA_L128_WARPS;
}

struct Row2 {
    uint64_t lo, hi;
};

__device__ __forceinline__ Row2 shfl_row(const Row2& r, int src) {
    return Row2{shfl64(r.lo, src), shfl64(r.hi, src)};
}

// Acceptance masks of the 64 colour-c sites of row y, P = (y + c) & 1: site
// x = 32q + 8j + 2m + P takes word m of Philox block 16y + 4q + j.
template <int P>
__device__ __forceinline__ void row_accepts128(const Keys& d, const HalfSweepGen& gen, uint32_t y,
                                               const Thr& t4, const Thr& t8, Row2& a4, Row2& a8) {
    const uint32_t one = d.one;
    constexpr uint32_t EV = 0x55555555u;
    uint32_t h4[4], h8[4];
#pragma unroll L128_QUNROLL
    for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t base = 16u * y + 4u * q;
        const uint32_t kc = group_tests<false, false, L128_HUNROLL>(
            [&](int h) { return philox_block<0>(d, gen, PA_L64_BLOCK(base, h)); }, one, t4.T, t8.T, t4.T,
            t8.T);
        const uint32_t b4 = (~(kc >> 1) & EV) << P, b8 = (~kc & EV) << P;
        if (q == 0) {
            h4[0] = b4;
            h8[0] = b8;
        } else if (q == 1) {
            h4[1] = b4;
            h8[1] = b8;
        } else if (q == 2) {
            h4[2] = b4;
            h8[2] = b8;
        } else {
            h4[3] = b4;
            h8[3] = b8;
        }
    }
    a4.lo = ((uint64_t)h4[1] << 32) | h4[0];
    a4.hi = ((uint64_t)h4[3] << 32) | h4[2];
    a8.lo = ((uint64_t)h8[1] << 32) | h8[0];
    a8.hi = ((uint64_t)h8[3] << 32) | h8[2];
}

// Flip mask of one 64-bit word of a row, from its bonds to x + 1 (a), x - 1
// (b), y - 1 (e) and y + 1 (f).
__device__ __forceinline__ uint64_t word_flips(uint64_t a, uint64_t b, uint64_t e, uint64_t f,
                                               uint64_t a4, uint64_t a8, uint64_t cm) {
    const uint64_t s1 = a ^ b, s2 = e ^ f;
    const uint64_t ge2 = (a & b) | (e & f) | (s1 & s2);
    const uint64_t zero = ~(a | b | e | f);
    const uint64_t one = (s1 ^ s2) & ~ge2;
    return (ge2 | (one & a4) | (zero & a8)) & cm;
}

// +-J couplings of one L = 128 row (bit x set: J = -1): bonds to x + 1, x - 1,
// y - 1, y + 1, two words each.
struct RowJ2 {
    Row2 xp, xm, up, dn;
};

// Flips the colour sites (parity P) of row y in place.
template <int P, bool PMJ>
__device__ __forceinline__ void row_update128(const Keys& d, const HalfSweepGen& gen, Row2& own,
                                              const Row2& up, const Row2& dn, uint32_t y,
                                              const Thr& t4, const Thr& t8, uint32_t full,
                                              const RowJ2& j) {
    constexpr uint64_t cm = P ? 0xAAAAAAAAAAAAAAAAull : 0x5555555555555555ull;
    Row2 a4, a8;
    row_accepts128<P>(d, gen, y, t4, t8, a4, a8);
    if (full & 1u) a4.lo = a4.hi = ~0ull;
    if (full & 2u) a8.lo = a8.hi = ~0ull;
    // bit x of the rotations: own bit x + 1 (rp) and x - 1 (rm), mod 128
    const uint64_t rp_lo = (own.lo >> 1) | (own.hi << 63), rp_hi = (own.hi >> 1) | (own.lo << 63);
    const uint64_t rm_lo = (own.lo << 1) | (own.hi >> 63), rm_hi = (own.hi << 1) | (own.lo >> 63);
    uint64_t a_lo = own.lo ^ rp_lo, b_lo = own.lo ^ rm_lo, e_lo = own.lo ^ up.lo, f_lo = own.lo ^ dn.lo;
    uint64_t a_hi = own.hi ^ rp_hi, b_hi = own.hi ^ rm_hi, e_hi = own.hi ^ up.hi, f_hi = own.hi ^ dn.hi;
    if constexpr (PMJ) {
        a_lo ^= j.xp.lo, b_lo ^= j.xm.lo, e_lo ^= j.up.lo, f_lo ^= j.dn.lo;
        a_hi ^= j.xp.hi, b_hi ^= j.xm.hi, e_hi ^= j.up.hi, f_hi ^= j.dn.hi;
    }
    const uint64_t fl_lo = word_flips(a_lo, b_lo, e_lo, f_lo, a4.lo, a8.lo, cm);
    const uint64_t fl_hi = word_flips(a_hi, b_hi, e_hi, f_hi, a4.hi, a8.hi, cm);
    own.lo ^= fl_lo;
    own.hi ^= fl_hi;
}

__device__ __forceinline__ uint32_t bonds_x128(const Row2& r, const Row2& jx) {
    return __popcll(r.lo ^ ((r.lo >> 1) | (r.hi << 63)) ^ jx.lo) +
           __popcll(r.hi ^ ((r.hi >> 1) | (r.lo << 63)) ^ jx.hi);
}

// Couplings of lane l's rows 4l .. 4l + 3 (four 32-bit words per row).
__device__ __forceinline__ void l128_couplings(const RunDev& d, int lane, RowJ2 (&j)[4]) {
    const uint32_t* jx = d.jpk;
    const uint32_t* jy = d.jpk + d.nwords;
    auto row = [](const uint32_t* t, int y) {
        return Row2{((uint64_t)t[4 * y + 1] << 32) | t[4 * y], ((uint64_t)t[4 * y + 3] << 32) | t[4 * y + 2]};
    };
    const int y0 = 4 * lane;
    Row2 prev = row(jy, (y0 + 127) & 127);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const Row2 x = row(jx, y0 + k), y = row(jy, y0 + k);
        // bit x of xm: the bond to x - 1, i.e. J(+x) of site x - 1 (mod 128)
        const Row2 xm{(x.lo << 1) | (x.hi >> 63), (x.hi << 1) | (x.lo >> 63)};
        j[k] = RowJ2{x, xm, prev, y};
        prev = y;
    }
}

// One replica at L = 128: theta sweeps in registers, then the measurement.
template <bool PMJ>
__device__ __forceinline__ uint32_t l128_replica(const Keys& K, uint4* spins, uint32_t slot,
                                                 int nsweeps, uint32_t g0, uint32_t ctag,
                                                 const Thr& t4, const Thr& t8, uint32_t full,
                                                 int lane, int& M, const RowJ2 (&j)[4]) {
    const uint32_t y0 = 4u * (uint32_t)lane;
    const int lup = (lane + 31) & 31, ldn = (lane + 1) & 31;
    uint4* p = spins + (size_t)slot * 128 + 4 * lane;  // 2048 bytes per replica
    Row2 r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint4 v = p[k];
        r[k].lo = ((uint64_t)v.y << 32) | v.x;
        r[k].hi = ((uint64_t)v.w << 32) | v.z;
    }
    for (int t = 0; t < nsweeps; ++t) {
        const uint32_t g = g0 + (uint32_t)t;
        {  // colour 0: rows 4l and 4l + 2 have parity 0
            const Row2 up = shfl_row(r[3], lup), dn = shfl_row(r[0], ldn);
            const HalfSweepGen gen = half_sweep_gen(K, 2u * g, slot, ctag);
            row_update128<0, PMJ>(K, gen, r[0], up, r[1], y0, t4, t8, full, j[0]);
            row_update128<1, PMJ>(K, gen, r[1], r[0], r[2], y0 + 1u, t4, t8, full, j[1]);
            row_update128<0, PMJ>(K, gen, r[2], r[1], r[3], y0 + 2u, t4, t8, full, j[2]);
            row_update128<1, PMJ>(K, gen, r[3], r[2], dn, y0 + 3u, t4, t8, full, j[3]);
        }
        {  // colour 1
            const Row2 up = shfl_row(r[3], lup), dn = shfl_row(r[0], ldn);
            const HalfSweepGen gen = half_sweep_gen(K, 2u * g + 1u, slot, ctag);
            row_update128<1, PMJ>(K, gen, r[0], up, r[1], y0, t4, t8, full, j[0]);
            row_update128<0, PMJ>(K, gen, r[1], r[0], r[2], y0 + 1u, t4, t8, full, j[1]);
            row_update128<1, PMJ>(K, gen, r[2], r[1], r[3], y0 + 2u, t4, t8, full, j[2]);
            row_update128<0, PMJ>(K, gen, r[3], r[2], dn, y0 + 3u, t4, t8, full, j[3]);
        }
    }
    // measurement: bonds to x + 1 and to y + 1 of the four rows
    const Row2 dn = shfl_row(r[0], ldn);
    uint32_t U = 0, down = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const Row2& nx = k < 3 ? r[k + 1] : dn;
        U += bonds_x128(r[k], j[k].xp) + __popcll(r[k].lo ^ nx.lo ^ j[k].dn.lo) +
             __popcll(r[k].hi ^ nx.hi ^ j[k].dn.hi);
        down += __popcll(r[k].lo) + __popcll(r[k].hi);
    }
    U = warp_sum(U);
    down = warp_sum(down);
    M = 16384 - 2 * (int)down;
    if (nsweeps > 0)  // a measurement alone leaves the replica as it is
#pragma unroll
        for (int k = 0; k < 4; ++k)
            p[k] = make_uint4((uint32_t)r[k].lo, (uint32_t)(r[k].lo >> 32), (uint32_t)r[k].hi,
                              (uint32_t)(r[k].hi >> 32));
    return U;
}

template <bool PMJ>
__global__ void __launch_bounds__(warps128<PMJ>() * 32, 1)
    k_sweep_l128(__grid_constant__ const RunDev d, int nsweeps) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    DevState* st = d.st;
    const uint32_t R = st->R;
    const uint32_t cur = st->cur;
    const uint32_t g0 = st->sweep_base;
    Thr t4, t8;
    uint32_t full;
    thresholds(d, st->step, t4, t8, full);
    const uint32_t ctag = (TAG_SWEEP << 28) | d.instance;
    const Keys K{d.rk0, d.rk1, d.one, nullptr};
    uint4* spins = reinterpret_cast<uint4*>(d.spins[cur]);
    RowJ2 j[4] = {};
    if constexpr (PMJ) l128_couplings(d, lane, j);
    const uint32_t parity = st->negbonds & 1u;
    L64Tally tally;
    constexpr int W = warps128<PMJ>();
    const uint32_t nwarps = gridDim.x * W;
    const uint32_t end = min(R, d.slot_hi);
    for (uint32_t slot = d.slot_lo + blockIdx.x * W + wib; slot < end; slot += nwarps) {
        int M = 0;
        const uint32_t U =
            l128_replica<PMJ>(K, spins, slot, nsweeps, g0, ctag, t4, t8, full, lane, M, j);
        if (lane == 0) {
            d.ebin[cur][slot] = U >> 1;
            d.mag[cur][slot] = M;
            if ((U & 1u) != parity) atomicOr(&st->status, ST_INVARIANT);
        }
        tally.add(d.hist, U, M, lane);
    }
    tally.finish(d.hist, d.accum, lane);
}

template <bool PMJ>
__global__ void __launch_bounds__(warps128<PMJ>() * 32, 1) k_sweep_l128_batched(BatchSweepArgs a) {
    __shared__ uint32_t s_keys[warps128<PMJ>()][24];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    L64Tally tally;
    for (;;) {
        uint32_t chunk = 0;
        if (lane == 0) chunk = atomicAdd(a.counter, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint32_t g = chunk * a.chunk;
        if (g >= a.total_slots) break;
        uint32_t lo = 0, hi = a.n;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.slot_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        const RunDev& d = a.runs[a.run_ids[lo]];
        DevState* st = d.st;
        const uint32_t R = st->R, cur = st->cur, g0 = st->sweep_base;
        Thr t4, t8;
        uint32_t full;
        thresholds(d, st->step, t4, t8, full);
        if (lane < 10) {
            s_keys[wib][lane] = d.rk0[lane];
            s_keys[wib][10 + lane] = d.rk1[lane];
        }
        __syncwarp();
        const uint32_t ctag = (TAG_SWEEP << 28) | d.instance;
        const Keys K{&s_keys[wib][0], &s_keys[wib][10], d.one, nullptr};
        uint4* spins = reinterpret_cast<uint4*>(d.spins[cur]);
        const uint32_t first = g - a.slot_base[lo];
        RowJ2 j[4] = {};
        if constexpr (PMJ) l128_couplings(d, lane, j);
        const uint32_t parity = st->negbonds & 1u;
        for (uint32_t slot = first; slot < first + a.chunk && slot < R; ++slot) {
            int M = 0;
            const uint32_t U =
                l128_replica<PMJ>(K, spins, slot, d.theta, g0, ctag, t4, t8, full, lane, M, j);
            if (lane == 0) {
                d.ebin[cur][slot] = U >> 1;
                d.mag[cur][slot] = M;
                if ((U & 1u) != parity) atomicOr(&st->status, ST_INVARIANT);
            }
            tally.add(d.hist, U, M, lane);
        }
        tally.finish(d.hist, d.accum, lane);
        __syncwarp();
    }
}

bool is_l128(const RunDev& d) {
    return d.layout == PA_LAYOUT_PACKED && d.dim == 2 && d.L == 128 && d.stride == 2048;
}

}  // namespace

// The register-resident row kernels: 2D ferromagnet, packed, L = 64 or 128.
bool l64_applies(const RunDev& d) {
    return (d.layout == PA_LAYOUT_PACKED && d.dim == 2 && d.L == 64 && d.stride == 512) ||
           is_l128(d);
}

int l64_block_warps(const RunDev& d) {
    if (!is_l128(d)) return WARPS64;
    return d.model == PA_MODEL_PMJ ? warps128<true>() : warps128<false>();
}

// --------------------------------------------------------------------------
// The generator's own ceiling in the register kernels' launch shape: the
// Philox blocks of k_sweep_l64 (half-sweep products shared, round-2 and
// round-3 block products from the tables: 14 multiplies per block; 16 blocks
// per half-sweep and lane) with nothing else done to the
// uniforms but an xor into one word per thread.  One warp stands for one
// replica (slot = global warp index); half-sweep g of lane l draws blocks
// 16 l .. 16 l + 15 of counter (2 g, block, SWEEP, slot).
struct PhiloxRateArgs {
    uint32_t rk0[10], rk1[10];
    uint32_t one;
    uint32_t halfsweeps;
    uint32_t* out;
};

// The generator alone runs one block of PHILOX_RATE_WARPS warps per SM: on
// GB300 16 warps draw 2135 uniforms/ns, 12 warps 2119, 8 warps 2058.
#ifndef PA_PHILOX_RATE_WARPS
#define PA_PHILOX_RATE_WARPS 16
#endif
constexpr int PHILOX_RATE_WARPS = PA_PHILOX_RATE_WARPS;

// Half-sweeps of one round-3 table window of the generator alone.
constexpr uint32_t PHILOX_RATE_WIN = 48;

__global__ void __launch_bounds__(PHILOX_RATE_WARPS * 32, 1)
    k_philox_rate(__grid_constant__ const PhiloxRateArgs a) {
    // the sweep kernel's tables: the run's round-2 products, then a window of
    // PHILOX_RATE_WIN half-sweeps' round-3 products, rebuilt per window
    extern __shared__ uint2 s_tab[];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t ctag = TAG_SWEEP << 28;
    cta_tables<false>(s_tab, ctag, 0u, 0, a.rk0, a.rk1);
    const Keys K{a.rk0, a.rk1, a.one, s_tab + lane, s_tab + 512 + lane};
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t slot = tid >> 5, base = lane * 16u;
    uint32_t acc = 0;
    for (uint32_t gb = 0; gb < a.halfsweeps; gb += PHILOX_RATE_WIN) {
        const uint32_t nw = min(PHILOX_RATE_WIN, a.halfsweeps - gb);
        __syncthreads();  // the previous window is read by no one any more
        for (uint32_t e = threadIdx.x; e < nw * 512u; e += blockDim.x) {
            uint32_t hc, lc, h, l;
            mul_hilo(PM0, 2u * (gb + (e >> 9)), hc, lc);  // round 1: M0 * c0, c0 = 2 g
            mul_hilo(PM1, s_tab[e & 511u].x ^ lc ^ a.rk1[1], h, l);  // round 3, block half
            s_tab[512u + e] = make_uint2(h, l);
        }
        __syncthreads();
        for (uint32_t w = 0; w < nw; ++w) {
            HalfSweepGen gen = half_sweep_gen(K, 2u * (gb + w), slot, ctag);
            gen.t3 = K.t3 + (size_t)w * 512;
#pragma unroll 4
            for (uint32_t h = 0; h < 16u; ++h) {
                const uint4 u = philox_block<16, true>(K, gen, base + h);
                acc ^= u.x ^ u.y ^ u.z ^ u.w;
            }
        }
    }
    a.out[tid] = acc;
}

// Dynamic shared memory of the L = 64 kernels: the plain kernel's CTA-wide
// round-2 table (512 entries) and, for launches of up to L64_T3_MAX sweeps,
// the round-3 table after it (2 nsweeps x 512 entries); the batched kernel's
// per-warp round-2 tables (its warps may serve different runs); the
// generator's round-2 table and one window of round-3 products.
constexpr int L64_T3_MAX = 26;
constexpr size_t TAB_ROW = 512 * sizeof(uint2);
static size_t l64_plain_smem(bool t3, int nsweeps) {
    return t3 ? (size_t)(1 + 2 * nsweeps) * TAB_ROW : TAB_ROW;
}
constexpr size_t L64_BATCHED_SMEM = (size_t)WARPS64 * 16 * 32 * sizeof(uint2);
constexpr size_t PHILOX_RATE_SMEM = (size_t)(1 + PHILOX_RATE_WIN) * TAB_ROW;

// Tables above the default 48 KB need the kernel's opt-in, once per device
// (set at the first launch, which pa_init makes outside any stream capture).
static cudaError_t ensure_smem_optin() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int t3max = (int)l64_plain_smem(true, L64_T3_MAX);
    if ((e = cudaFuncSetAttribute(k_sweep_l64<false, true>, A, t3max)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_sweep_l64<true, true>, A, t3max)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_sweep_l64_batched<false>, A, (int)L64_BATCHED_SMEM)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_sweep_l64_batched<true>, A, (int)L64_BATCHED_SMEM)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_philox_rate, A, (int)PHILOX_RATE_SMEM)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

// The L = 128 kernels form their round-2 products: a 128 KB table per block
// ran 0.5-1.3 % slower there on GB300 (it takes that much of the L1).
static size_t l64_batched_smem(const RunDev& d) { return is_l128(d) ? 0 : L64_BATCHED_SMEM; }

static int wave(const void* fn, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (ensure_smem_optin() != cudaSuccess) return 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess)
        return 0;
    return per_sm < 1 ? 0 : sms * per_sm;
}

template <typename K64, typename K128>
static const void* pick(const RunDev& d, K64 f64f, K64 f64j, K128 f128f, K128 f128j) {
    const bool pmj = d.model == PA_MODEL_PMJ;
    if (is_l128(d)) return pmj ? (const void*)f128j : (const void*)f128f;
    return pmj ? (const void*)f64j : (const void*)f64f;
}

int l64_grid(const RunDev& d) {
    const int w = l64_block_warps(d);
    // one CTA per SM in either form (the register budget of 12 warps)
    const int full = wave(pick(d, k_sweep_l64<false, false>, k_sweep_l64<true, false>,
                               k_sweep_l128<false>, k_sweep_l128<true>),
                          w * 32, is_l128(d) ? 0 : l64_plain_smem(false, 0));
    if (full <= 0) return 0;
    const int64_t need = ((int64_t)d.cap + w - 1) / w;
    return (int)(need < full ? need : full);
}

cudaError_t launch_sweep_l64(const RunDev& d, int nsweeps, int grid, cudaStream_t s) {
    const cudaError_t e = ensure_smem_optin();
    if (e != cudaSuccess) return e;
    const bool pmj = d.model == PA_MODEL_PMJ;
    if (is_l128(d)) {
        if (pmj) k_sweep_l128<true><<<grid, warps128<true>() * 32, 0, s>>>(d, nsweeps);
        else k_sweep_l128<false><<<grid, warps128<false>() * 32, 0, s>>>(d, nsweeps);
    } else if (nsweeps >= 1 && nsweeps <= L64_T3_MAX) {
        const size_t sm = l64_plain_smem(true, nsweeps);
        if (pmj) k_sweep_l64<true, true><<<grid, WARPS64 * 32, sm, s>>>(d, nsweeps);
        else k_sweep_l64<false, true><<<grid, WARPS64 * 32, sm, s>>>(d, nsweeps);
    } else {
        const size_t sm = l64_plain_smem(false, nsweeps);
        if (pmj) k_sweep_l64<true, false><<<grid, WARPS64 * 32, sm, s>>>(d, nsweeps);
        else k_sweep_l64<false, false><<<grid, WARPS64 * 32, sm, s>>>(d, nsweeps);
    }
    return cudaGetLastError();
}

// One block per SM.
static int philox_rate_grid() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

int philox_rate_threads() { return philox_rate_grid() * PHILOX_RATE_WARPS * 32; }

cudaError_t launch_philox_rate(uint64_t seed, uint32_t halfsweeps, uint32_t* out, cudaStream_t s) {
    const int grid = philox_rate_grid();
    if (grid <= 0) return cudaErrorInvalidValue;
    PhiloxRateArgs a;
    for (int k = 0; k < 10; ++k) {
        a.rk0[k] = (uint32_t)seed + (uint32_t)k * 0x9E3779B9u;
        a.rk1[k] = (uint32_t)(seed >> 32) + (uint32_t)k * 0xBB67AE85u;
    }
    a.one = 1u;
    a.halfsweeps = halfsweeps;
    a.out = out;
    const cudaError_t e = ensure_smem_optin();
    if (e != cudaSuccess) return e;
    k_philox_rate<<<grid, PHILOX_RATE_WARPS * 32, PHILOX_RATE_SMEM, s>>>(a);
    return cudaGetLastError();
}

bool l64_batched_applies(const RunDev& proto) { return l64_applies(proto); }

int l64_batched_grid(const RunDev& proto) {
    return wave(pick(proto, k_sweep_l64_batched<false>, k_sweep_l64_batched<true>,
                     k_sweep_l128_batched<false>, k_sweep_l128_batched<true>),
                l64_block_warps(proto) * 32, l64_batched_smem(proto));
}

cudaError_t launch_sweep_l64_batched(const BatchSweepArgs& a, const RunDev& proto, int grid,
                                     cudaStream_t s) {
    const cudaError_t e = ensure_smem_optin();
    if (e != cudaSuccess) return e;
    const bool pmj = proto.model == PA_MODEL_PMJ;
    const size_t sm = l64_batched_smem(proto);
    if (is_l128(proto)) {
        if (pmj) k_sweep_l128_batched<true><<<grid, warps128<true>() * 32, sm, s>>>(a);
        else k_sweep_l128_batched<false><<<grid, warps128<false>() * 32, sm, s>>>(a);
    } else {
        if (pmj) k_sweep_l64_batched<true><<<grid, WARPS64 * 32, sm, s>>>(a);
        else k_sweep_l64_batched<false><<<grid, WARPS64 * 32, sm, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace pa
