// chain_latency.cu -- dependent-latency microbenchmark of the operation
// classes on one lineage's event chain (measurement tool of the test side;
// not part of the library).
//
// Each kernel runs one dependent chain of STEPS operations of one class in
// one warp (lane 0's clock), every lane from a different value (a chain of
// warp-uniform values may run on the uniform datapath instead of the
// per-lane pipes the kernels use), and writes the chain's result, so
// nothing can be dropped; the cycle count comes from clock64() around the chain.  The
// chains are built so that no step can start before the previous one ends
// and no algebra can shorten them: every step feeds a nonlinear operation
// (a high product, a table index, a shuffle lane, a compare) or is measured
// as the difference of two such chains.
//
//   imad_hi     x = mulhi32(x, y)                       32-bit high product
//   philox      one Philox4x32 round (two high/low product pairs, xors and
//               the key schedule): the round's dependent path
//   philox_split the same with the low products from run-time multipliers
//   philox_m1   the same with each low product as c (M - 1) + c
//   hi_xor      x = mulhi32(x, y) ^ z                   high product + xor
//   umul64hi    x = mulhi64(x, y)                       64-bit high product
//   imad_wide   x = lo64(lo32(x) * y + x)               32x32 -> 64 multiply-add
//   add64_sel   x = (x + a < b) ? x + a : x + c         64-bit add, compare, select
//   clz_norm    x = (x << clz64(x)) ^ a                 normalise: leading-zero count, shift
//   lds         i = s[i]                                shared-memory load
//   ldg_l1      i = g[i] (4 KB ring, L1-resident)       global load, L1 hit
//   ldg_dram    i = g[i] (random ring >> L2)            global load from DRAM
//   ballot      x = ballot(x & bit) ^ x                  warp vote + xor
//   redux_min   x = redux.min(x) ^ lane-independent    warp reduction
//   shfl_add    x = shfl(x, lane x & 31) + z            shuffle and add
//   bulk_row    one 6.4 KB bulk copy (TMA) of a random row into shared
//               memory, issue to mbarrier completion
//
// and one throughput kernel: independent Philox blocks on every SM, the
// integer peak of the library's op mix (k_philox_tput).
#include <cstdint>
#include <cuda_runtime.h>

constexpr int STEPS = 2048;

struct Out {
    unsigned long long cycles;
    unsigned long long sink;
};

__device__ __forceinline__ unsigned long long clk() { return clock64(); }

// the clock read after a value is known (its data dependence keeps it last)
__device__ __forceinline__ unsigned long long clk_after_u32(uint32_t x) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(t) : "r"(x) : "memory");
    return t;
}

#define CHAIN_KERNEL(NAME, TYPE, INIT, STEP)                                              \
    __global__ void k_##NAME(const uint64_t* __restrict__ prm, Out* out) {                \
        TYPE x = (TYPE)(INIT) ^ (TYPE)(threadIdx.x * 0x9E3779B9u); /* lane-dependent */  \
        const uint64_t a = prm[0], b = prm[1], c = prm[2];                                \
        const uint32_t y = (uint32_t)prm[3], z = (uint32_t)prm[4];                        \
        (void)a; (void)b; (void)c; (void)y; (void)z;                                       \
        __syncwarp();                                                                     \
        const unsigned long long t0 = clk();                                              \
        _Pragma("unroll 1") for (int it = 0; it < STEPS / 64; ++it) {                      \
            _Pragma("unroll") for (int s = 0; s < 64; ++s) { STEP; }                       \
        }                                                                                 \
        const unsigned long long t1 = clk();                                              \
        if ((threadIdx.x & 31u) == 0u) out->cycles = t1 - t0;                              \
        out->sink += (unsigned long long)x;                                               \
    }

CHAIN_KERNEL(imad_hi, uint32_t, prm[5], x = __umulhi(x, y))
CHAIN_KERNEL(hi_xor, uint32_t, prm[5], x = __umulhi(x, y) ^ z)
CHAIN_KERNEL(umul64hi, uint64_t, prm[5], x = __umul64hi(x, a))
CHAIN_KERNEL(imad_wide, uint64_t, prm[5], x = (uint64_t)(uint32_t)x * y + x)
CHAIN_KERNEL(add64_sel, uint64_t, prm[5], { const uint64_t s0 = x + a; x = s0 < b ? s0 : x + c; })
CHAIN_KERNEL(clz_norm, uint64_t, prm[5], x = (x << __clzll((long long)x)) ^ a)
CHAIN_KERNEL(ballot, uint32_t, prm[5], x = __ballot_sync(0xFFFFFFFFu, (x >> (threadIdx.x & 31u)) & 1u) ^ z)
CHAIN_KERNEL(redux_min, uint32_t, prm[5], x = __reduce_min_sync(0xFFFFFFFFu, x ^ threadIdx.x) + z)

// a 32-bit add whose result indexes nothing: x = (x + z) ^ y is one
// dependent add and one xor per step (measured beside hi_xor and imad_hi)
CHAIN_KERNEL(add_xor, uint32_t, prm[5], x = (x + z) ^ y)

// a shuffle whose source lane comes from the data, then an add (a bare
// shuffle chain is not kept intact by the compiler)
CHAIN_KERNEL(shfl_add, uint32_t, prm[5], x = __shfl_sync(0xFFFFFFFFu, x, (int)(x & 31u)) + z)

// one Philox4x32 round per step: the counter words feed the next round,
// the key words advance by the Weyl increments
__global__ void k_philox(const uint64_t* __restrict__ prm, Out* out) {
    // lane-dependent counters: the chain runs on the per-lane pipes, as in
    // the kernels (a warp-uniform chain may run on the uniform datapath)
    uint32_t c0 = (uint32_t)prm[0] ^ threadIdx.x, c1 = (uint32_t)prm[1], c2 = (uint32_t)prm[2] + threadIdx.x,
             c3 = (uint32_t)prm[3];
    uint32_t k0 = (uint32_t)prm[4], k1 = (uint32_t)prm[5];
    __syncwarp();
    const unsigned long long t0 = clk();
#pragma unroll 1
    for (int it = 0; it < STEPS / 64; ++it) {
#pragma unroll
        for (int s = 0; s < 64; ++s) {
            const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
            const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
            c0 = hi1 ^ c1 ^ k0;
            c1 = lo1;
            c2 = hi0 ^ c3 ^ k1;
            c3 = lo0;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    const unsigned long long t1 = clk();
    if ((threadIdx.x & 31u) == 0u) out->cycles = t1 - t0;
    out->sink += (unsigned long long)(c0 ^ c1 ^ c2 ^ c3);
}

// the same round with the low products taken from multipliers read at run
// time (equal to the constants), so that each high product stays a lone
// high-half multiply rather than one wide multiply giving both halves
__constant__ uint32_t c_zero = 0;
__global__ void k_philox_split(const uint64_t* __restrict__ prm, Out* out) {
    // lane-dependent counters: the chain runs on the per-lane pipes, as in
    // the kernels (a warp-uniform chain may run on the uniform datapath)
    uint32_t c0 = (uint32_t)prm[0] ^ threadIdx.x, c1 = (uint32_t)prm[1], c2 = (uint32_t)prm[2] + threadIdx.x,
             c3 = (uint32_t)prm[3];
    uint32_t k0 = (uint32_t)prm[4], k1 = (uint32_t)prm[5];
    const uint32_t m0 = 0xD2511F53u ^ c_zero, m1 = 0xCD9E8D57u ^ c_zero;
    __syncwarp();
    const unsigned long long t0 = clk();
#pragma unroll 1
    for (int it = 0; it < STEPS / 64; ++it) {
#pragma unroll
        for (int s = 0; s < 64; ++s) {
            const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = m0 * c0;
            const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = m1 * c2;
            c0 = hi1 ^ c1 ^ k0;
            c1 = lo1;
            c2 = hi0 ^ c3 ^ k1;
            c3 = lo0;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    const unsigned long long t1 = clk();
    if ((threadIdx.x & 31u) == 0u) out->cycles = t1 - t0;
    out->sink += (unsigned long long)(c0 ^ c1 ^ c2 ^ c3);
}

// the same round with each low product written as c (M - 1) + c: equal to
// c M, but with a multiplier other than the high product's, so that the two
// need not share one wide multiply
__global__ void k_philox_m1(const uint64_t* __restrict__ prm, Out* out) {
    // lane-dependent counters: the chain runs on the per-lane pipes, as in
    // the kernels (a warp-uniform chain may run on the uniform datapath)
    uint32_t c0 = (uint32_t)prm[0] ^ threadIdx.x, c1 = (uint32_t)prm[1], c2 = (uint32_t)prm[2] + threadIdx.x,
             c3 = (uint32_t)prm[3];
    uint32_t k0 = (uint32_t)prm[4], k1 = (uint32_t)prm[5];
    __syncwarp();
    const unsigned long long t0 = clk();
#pragma unroll 1
    for (int it = 0; it < STEPS / 64; ++it) {
#pragma unroll
        for (int s = 0; s < 64; ++s) {
            const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = c0 * (0xD2511F53u - 1u) + c0;
            const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = c2 * (0xCD9E8D57u - 1u) + c2;
            c0 = hi1 ^ c1 ^ k0;
            c1 = lo1;
            c2 = hi0 ^ c3 ^ k1;
            c3 = lo0;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    const unsigned long long t1 = clk();
    if ((threadIdx.x & 31u) == 0u) out->cycles = t1 - t0;
    out->sink += (unsigned long long)(c0 ^ c1 ^ c2 ^ c3);
}

// dependent loads: i = table[i] over a ring laid out by the host
__global__ void k_lds(const uint64_t* __restrict__ prm, Out* out) {
    __shared__ uint32_t s[1024];
    for (uint32_t k = threadIdx.x; k < 1024; k += blockDim.x) s[k] = (k * 7u + 13u) & 1023u;
    __syncthreads();
    uint32_t i = ((uint32_t)prm[5] + threadIdx.x * 37u) & 1023u;
    const unsigned long long t0 = clk();
#pragma unroll 1
    for (int it = 0; it < STEPS / 64; ++it) {
#pragma unroll
        for (int s2 = 0; s2 < 64; ++s2) i = s[i];
    }
    const unsigned long long t1 = clk();
    if ((threadIdx.x & 31u) == 0u) out->cycles = t1 - t0;
    out->sink += i;
}

__global__ void k_ldg(const uint32_t* __restrict__ ring, uint32_t start, int steps, Out* out) {
    uint32_t i = start;
    const unsigned long long t0 = clk();
    for (int s = 0; s < steps; ++s) i = __ldcg(ring + i);  // L2-cached load (L1 bypassed): the gather's path
    const unsigned long long t1 = clk();
    if ((threadIdx.x & 31u) == 0u) out->cycles = t1 - t0;
    out->sink += i;
}

__global__ void k_ldg_l1(const uint32_t* __restrict__ ring, uint32_t start, int steps, Out* out) {
    uint32_t i = start;
    const unsigned long long t0 = clk();
    for (int s = 0; s < steps; ++s) i = __ldg(ring + i);
    const unsigned long long t1 = clk();
    if ((threadIdx.x & 31u) == 0u) out->cycles = t1 - t0;
    out->sink += i;
}

// The map row's copy: bulk copies (cp.async.bulk, TMA) of `bytes` in pieces
// of `piece` bytes from a pseudo-random 16-byte-aligned row of a device buffer of
// `n_rows` rows into shared memory, completing an mbarrier; every lane then
// waits on it (bounded: at most 2^22 probes, else error bit 1 in out->sink's
// high word and the loop stops).  Cycles per copy, issue to completion.
// Every source address lies in the buffer: row < n_rows, row * stride +
// bytes <= n_rows * stride.
__global__ void k_bulk_row(const unsigned char* __restrict__ buf, uint32_t n_rows, uint32_t stride, uint32_t bytes,
                           uint32_t piece, int copies, Out* out) {
    extern __shared__ __align__(16) unsigned char sm[];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t dst = bar + 16u;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    uint32_t row = 12345u % n_rows;
    unsigned long long err = 0;
    const unsigned long long t0 = clk();
    for (int c = 0; c < copies; ++c) {
        const unsigned char* src = buf + (size_t)row * stride;
        __syncwarp();
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        }
        // the row in pieces of `piece` bytes (the last one shorter), issued
        // one per lane side by side, all completing the one barrier
        const uint32_t first = lane * piece;
        if (first < bytes) {
            const uint32_t len = min(piece, bytes - first);
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             dst + first),
                         "l"(src + first), "r"(len), "r"(bar)
                         : "memory");
        }
        uint32_t done = 0;
        for (uint32_t it = 0; it < (1u << 22) && !done; ++it)
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done)
                         : "r"(bar), "r"((uint32_t)c & 1u)
                         : "memory");
        if (!done) {
            err = 1;
            break;
        }
        // the next row depends on the copied data, so copies do not overlap
        const uint32_t v = *(volatile const uint32_t*)(sm + 16);
        row = (uint32_t)(((uint64_t)(row * 2654435761u + v + 1u)) % n_rows);
    }
    const unsigned long long t1 = clk_after_u32(row);
    if (lane == 0) {
        out->cycles = t1 - t0;
        out->sink = (err << 32) | row;
    }
}

// spins for `cycles` SM clock cycles (bounded by the count itself): timed
// with CUDA events on the host, it gives the SM clock during the run
__global__ void k_spin(unsigned long long cycles, Out* out) {
    const unsigned long long t0 = clk();
    unsigned long long t = t0;
    while (t - t0 < cycles) t = clk();
    if (threadIdx.x == 0) out->cycles = t - t0;
}

// Integer throughput on every SM: each thread runs PX_LANES independent
// Philox4x32-10 blocks side by side, block after block, counter-chained so
// that nothing is dropped (one round: two 32x32 products giving high and low
// halves, two three-input xors, two key adds).  Counted as the library's op
// model counts a block: 10 rounds x 10 integer ops.
constexpr int PX_LANES = 4;

__global__ void __launch_bounds__(256) k_philox_tput(uint32_t blocks, uint32_t seed, Out* out) {
    uint32_t c0[PX_LANES], c1[PX_LANES], c2[PX_LANES], c3[PX_LANES];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int l = 0; l < PX_LANES; ++l) {
        c0[l] = tid * 0x9E3779B9u + (uint32_t)l;
        c1[l] = seed;
        c2[l] = (uint32_t)l * 0x85EBCA6Bu;
        c3[l] = tid;
    }
    for (uint32_t b = 0; b < blocks; ++b) {
        uint32_t k0 = seed ^ b, k1 = 0xBB67AE85u ^ b;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
#pragma unroll
            for (int l = 0; l < PX_LANES; ++l) {
                const uint32_t hi0 = __umulhi(0xD2511F53u, c0[l]), lo0 = 0xD2511F53u * c0[l];
                const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2[l]), lo1 = 0xCD9E8D57u * c2[l];
                const uint32_t n0 = hi1 ^ c1[l] ^ k0, n2 = hi0 ^ c3[l] ^ k1;
                c0[l] = n0;
                c1[l] = lo1;
                c2[l] = n2;
                c3[l] = lo0;
            }
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int l = 0; l < PX_LANES; ++l) x ^= c0[l] ^ c1[l] ^ c2[l] ^ c3[l];
    if (x == 0x5A5A5A5Au && seed == 0x12345u) out->sink = x;  // keeps the work; practically never true
}

extern "C" {

// measured integer ops per second of the Philox mix on all SMs (grid: SMs x
// blocks_per_sm blocks of 256 threads); negative: CUDA error
double hwlat_philox_throughput(int sms, int blocks_per_sm, uint32_t blocks, void* out_dev) {
    if (sms < 1 || blocks_per_sm < 1 || blocks < 1) return -1.0;
    Out* o = (Out*)out_dev;
    const int grid = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
    k_philox_tput<<<grid, 256>>>(8, 0x12345u, o);  // warm-up launch
    cudaEventRecord(e0);
    k_philox_tput<<<grid, 256>>>(blocks, 0x12345u, o);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return -(double)e;
    const double ops = (double)grid * 256.0 * PX_LANES * (double)blocks * 100.0;
    return ops / ((double)ms * 1e-3);
}

// SM clock in MHz over a spin of `cycles` cycles (negative: CUDA error)
double hwlat_clock_mhz(unsigned long long cycles, void* out_dev) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
    k_spin<<<1, 32>>>(1000, (Out*)out_dev);  // warm-up launch
    cudaEventRecord(e0);
    k_spin<<<1, 32>>>(cycles, (Out*)out_dev);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return -(double)e;
    return (double)cycles / ((double)ms * 1e3);
}

int hwlat_steps() { return STEPS; }

// class ids: 0 imad_hi, 1 hi_xor, 2 umul64hi, 3 imad_wide, 4 add64_sel,
// 5 clz_norm, 6 add_xor, 8 ballot, 9 redux_min, 10 philox, 11 lds, 12 philox_split, 13 philox_m1, 14 shfl_add
// Runs the chain once in one warp of one block; returns its cycles, or a
// negative CUDA error.  prm: 6 device words of runtime operands.
long long hwlat_run(int cls, const uint64_t* prm, void* out_dev) {
    Out* o = (Out*)out_dev;
    switch (cls) {
        case 0: k_imad_hi<<<1, 32>>>(prm, o); break;
        case 1: k_hi_xor<<<1, 32>>>(prm, o); break;
        case 2: k_umul64hi<<<1, 32>>>(prm, o); break;
        case 3: k_imad_wide<<<1, 32>>>(prm, o); break;
        case 4: k_add64_sel<<<1, 32>>>(prm, o); break;
        case 5: k_clz_norm<<<1, 32>>>(prm, o); break;
        case 6: k_add_xor<<<1, 32>>>(prm, o); break;
        case 8: k_ballot<<<1, 32>>>(prm, o); break;
        case 9: k_redux_min<<<1, 32>>>(prm, o); break;
        case 10: k_philox<<<1, 32>>>(prm, o); break;
        case 11: k_lds<<<1, 32>>>(prm, o); break;
        case 12: k_philox_split<<<1, 32>>>(prm, o); break;
        case 13: k_philox_m1<<<1, 32>>>(prm, o); break;
        case 14: k_shfl_add<<<1, 32>>>(prm, o); break;
        default: return -1;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return -(long long)e;
    Out h;
    e = cudaMemcpy(&h, o, sizeof(Out), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return -(long long)e;
    return (long long)h.cycles;
}

// cycles per bulk row copy (see k_bulk_row); negative: CUDA error, or -1000
// if a wait gave up
long long hwlat_bulk_row(const unsigned char* buf, uint32_t n_rows, uint32_t stride, uint32_t bytes, uint32_t piece,
                         int copies, void* out_dev) {
    if (bytes % 16u || stride % 16u || bytes > stride || bytes > 32768u || n_rows == 0) return -1;
    if (piece % 16u || piece == 0 || (uint64_t)piece * 32u < bytes) return -1;  // at most 32 pieces, 16-byte multiples
    Out* o = (Out*)out_dev;
    cudaFuncSetAttribute(k_bulk_row, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes + 16u));
    k_bulk_row<<<1, 32, bytes + 16u>>>(buf, n_rows, stride, bytes, piece, copies, o);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return -(long long)e;
    Out h;
    e = cudaMemcpy(&h, o, sizeof(Out), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return -(long long)e;
    if (h.sink >> 32) return -1000;
    return (long long)h.cycles;
}

// dependent global loads over a ring of n entries (device array built by the
// caller); l1: 1 for the L1-cached form.  Every index stays below n.
long long hwlat_ring(const uint32_t* ring, uint32_t start, int steps, int l1, void* out_dev) {
    Out* o = (Out*)out_dev;
    if (l1) k_ldg_l1<<<1, 32>>>(ring, start, steps, o);
    else k_ldg<<<1, 32>>>(ring, start, steps, o);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return -(long long)e;
    Out h;
    e = cudaMemcpy(&h, o, sizeof(Out), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return -(long long)e;
    return (long long)h.cycles;
}

}
