// pa_bench.cu -- integer-pipe throughput of this GPU (pa_bench_intops in
// include/pa.h).  A measurement, not part of a run: it gives the peak against
// which the sweep kernels' integer work is reported.
//
// Every thread runs `iters` iterations of IO_CHAINS independent dependency
// chains, one step per chain and iteration, written as inline PTX so that
// each chain step is one instruction of the chosen kind (two for the
// multiply-xor step):
//   PA_INTOPS_LOP3       lop3.b32 (three-input logic; the ALU pipe)
//   PA_INTOPS_IMAD       mad.lo.u32 (32-bit multiply-add)
//   PA_INTOPS_WIDE       mad.wide.u32 (32 x 32 -> 64 multiply with a 64-bit add)
//   PA_INTOPS_LOP3_IMAD  lop3 on even chains, mad.lo on odd ones
//   PA_INTOPS_LOP3_WIDE  lop3 on even chains, mad.wide on odd ones
//   PA_INTOPS_MULWIDE_XOR  x <- hi(x b) xor lo(x b): a mul.wide.u32 and a
//                        two-input xor per chain step, both halves of the
//                        product consumed -- one multiply of a Philox4x32
//                        round with its xor
// The grid fills every SM with resident threads, so independent chains
// cover the instruction latencies and the count of instructions over the
// kernel's time is the pipe throughput.  The chains are folded into one word
// per thread at the end, so nothing is dead code.
#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr int IO_THREADS = 256;
constexpr int IO_BLOCKS_PER_SM = 8;  // 2048 threads: a full SM
constexpr int IO_CHAINS = 8;

__device__ __forceinline__ void op_lop3(uint32_t& a, uint32_t b, uint32_t c) {
    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a) : "r"(b), "r"(c));
}

__device__ __forceinline__ void op_imad(uint32_t& a, uint32_t b, uint32_t c) {
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a) : "r"(b), "r"(c));
}

__device__ __forceinline__ void op_mulwide_xor(uint32_t& a, uint32_t b) {
    asm volatile(
        "{\n\t.reg .u64 t;\n\t.reg .u32 lo, hi;\n\t"
        "mul.wide.u32 t, %0, %1;\n\t"
        "mov.b64 {lo, hi}, t;\n\t"
        "xor.b32 %0, lo, hi;\n\t}"
        : "+r"(a)
        : "r"(b));
}

__device__ __forceinline__ void op_wide(unsigned long long& w, uint32_t b) {
    asm volatile(
        "{\n\t.reg .u32 lo, hi;\n\t"
        "mov.b64 {lo, hi}, %0;\n\t"
        "mad.wide.u32 %0, lo, %1, %0;\n\t}"
        : "+l"(w)
        : "r"(b));
}

template <int KIND>
__global__ void __launch_bounds__(IO_THREADS) k_intops(uint32_t iters, uint32_t seed,
                                                       uint32_t* __restrict__ out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[IO_CHAINS];
    unsigned long long w[IO_CHAINS];
#pragma unroll
    for (int j = 0; j < IO_CHAINS; ++j) {
        a[j] = tid * 0x9E3779B9u + (uint32_t)j * 0x85EBCA6Bu + seed;
        w[j] = ((unsigned long long)a[j] << 32) | (a[j] ^ 0x5bd1e995u);
    }
    const uint32_t b = seed | 1u, c = seed ^ 0x27d4eb2fu;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < IO_CHAINS; ++j) {
            if (KIND == PA_INTOPS_LOP3) {
                op_lop3(a[j], b, c);
            } else if (KIND == PA_INTOPS_IMAD) {
                op_imad(a[j], b, c);
            } else if (KIND == PA_INTOPS_WIDE) {
                op_wide(w[j], b);
            } else if (KIND == PA_INTOPS_LOP3_IMAD) {
                if (j & 1) op_imad(a[j], b, c);
                else op_lop3(a[j], b, c);
            } else if (KIND == PA_INTOPS_MULWIDE_XOR) {
                op_mulwide_xor(a[j], b);
            } else {
                if (j & 1) op_wide(w[j], b);
                else op_lop3(a[j], b, c);
            }
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < IO_CHAINS; ++j) r ^= a[j] ^ (uint32_t)w[j] ^ (uint32_t)(w[j] >> 32);
    out[tid] = r;
}

int intops_grid() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms * IO_BLOCKS_PER_SM;
}

}  // namespace
}  // namespace pa

extern "C" int64_t pa_bench_intops_threads(void) {
    return (int64_t)pa::intops_grid() * pa::IO_THREADS;
}

extern "C" int64_t pa_bench_intops_per_iter(void) { return pa::IO_CHAINS; }

extern "C" int pa_bench_intops(int32_t kind, int32_t iters, void* out_dev, int64_t out_words,
                               void* stream) {
    const int grid = pa::intops_grid();
    if (grid <= 0) return PA_ERR_CUDA;
    if (!out_dev || iters < 1 || out_words < (int64_t)grid * pa::IO_THREADS)
        return PA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* out = static_cast<uint32_t*>(out_dev);
    const uint32_t seed = 0x2006u;
    switch (kind) {
        case PA_INTOPS_LOP3:
            pa::k_intops<PA_INTOPS_LOP3><<<grid, pa::IO_THREADS, 0, s>>>(iters, seed, out);
            break;
        case PA_INTOPS_IMAD:
            pa::k_intops<PA_INTOPS_IMAD><<<grid, pa::IO_THREADS, 0, s>>>(iters, seed, out);
            break;
        case PA_INTOPS_WIDE:
            pa::k_intops<PA_INTOPS_WIDE><<<grid, pa::IO_THREADS, 0, s>>>(iters, seed, out);
            break;
        case PA_INTOPS_LOP3_IMAD:
            pa::k_intops<PA_INTOPS_LOP3_IMAD><<<grid, pa::IO_THREADS, 0, s>>>(iters, seed, out);
            break;
        case PA_INTOPS_LOP3_WIDE:
            pa::k_intops<PA_INTOPS_LOP3_WIDE><<<grid, pa::IO_THREADS, 0, s>>>(iters, seed, out);
            break;
        case PA_INTOPS_MULWIDE_XOR:
            pa::k_intops<PA_INTOPS_MULWIDE_XOR><<<grid, pa::IO_THREADS, 0, s>>>(iters, seed, out);
            break;
        default:
            return PA_ERR_INVALID_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}
