// engine.cu -- kernels and C ABI of the Independent-algorithm engine.
//
// One engine serves a single simulation and a batch of uneven simulations
// alike: the lineages of all simulations of a batch share structure-of-arrays
// buffers, each simulation keeps its own horizon (water level, appendix "The
// Independent Water-Level Algorithm"), and one persistent advance kernel per
// round moves every active lineage of every simulation to its simulation's
// horizon.  Per round:
//   advance  -- events (speciation or dispersal) until the next event lies
//               beyond the horizon; then insert the lineage's indexed
//               location into the round's dedup table (min lineage id wins);
//   compact  -- drop finished lineages, cull the losers of the dedup
//               (parent[loser] = winner), write the survivors to the other
//               buffer; its last block advances every simulation's horizon.
// Lineages at the same indexed location at a horizon T are exact duplicates:
// the next event of both is the first point of that location's event
// process after T, and everything after depends only on (location, time).
// Culling either copy is exact, so results do not depend on the dedup, its
// cadence, the tuning or the GPU's execution order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "indep.h"
#include "device.cuh"

namespace indep {
void host_ln_tables(uint64_t* L, uint32_t* R, int n, uint64_t* ln2_q64, int64_t* c3);
int host_gauss_half(double sigma);
std::vector<uint64_t> host_gauss_cdf(double sigma);
std::vector<uint64_t> host_kernel_weights(double sigma, int radius);
int host_poisson_n(double mu);
std::vector<uint64_t> host_poisson_cdf(double mu);
}  // namespace indep

using namespace indep;

// ---------------------------------------------------------------------------
// process state
// ---------------------------------------------------------------------------
static std::atomic<int> g_last_cuda_error{0};
static std::atomic<uint64_t> g_launches{0};
static ind_allocator g_alloc = {nullptr, nullptr, nullptr};

#define CK(expr)                                           \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) {                           \
            g_last_cuda_error.store((int)e_);              \
            return IND_ERR_CUDA;                           \
        }                                                  \
    } while (0)

#define CKL()                                              \
    do {                                                   \
        g_launches.fetch_add(1);                           \
        cudaError_t e_ = cudaGetLastError();               \
        if (e_ != cudaSuccess) {                           \
            g_last_cuda_error.store((int)e_);              \
            return IND_ERR_CUDA;                           \
        }                                                  \
    } while (0)

struct Alloc {
    void* p;
    size_t bytes;
};

static void* dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (g_alloc.alloc) return g_alloc.alloc(bytes, (void*)s, g_alloc.ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dev_free(void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    bytes = (bytes + 255) & ~(size_t)255;
    if (g_alloc.release) {
        g_alloc.release(p, bytes, (void*)s, g_alloc.ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

// owner of a set of device allocations on one stream
struct Pool {
    cudaStream_t stream = nullptr;
    std::vector<Alloc> allocs;
    template <class T>
    T* get(size_t count) {
        size_t bytes = count * sizeof(T);
        void* p = dev_alloc(bytes, stream);
        if (p) allocs.push_back({p, bytes});
        return (T*)p;
    }
    void release_all() {
        for (auto& a : allocs) dev_free(a.p, a.bytes, stream);
        allocs.clear();
    }
    size_t total() const {
        size_t t = 0;
        for (auto& a : allocs) t += a.bytes;
        return t;
    }
};

// ---------------------------------------------------------------------------
// device data
// ---------------------------------------------------------------------------
__device__ LnTables g_ln;  // read-only tables of the inverse-transform logarithm
static std::mutex g_ln_mutex;
static std::vector<int> g_ln_ready;  // per device

static ind_status ensure_ln_tables(cudaStream_t s) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_ln_mutex);
    if ((int)g_ln_ready.size() <= dev) g_ln_ready.resize(dev + 1, 0);
    if (g_ln_ready[dev]) return IND_OK;
    static LnTables host;
    host_ln_tables(host.L, host.R, (int)LN_N, &host.ln2_q64, &host.c3);
    CK(cudaMemcpyToSymbolAsync(g_ln, &host, sizeof(LnTables), 0, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    g_ln_ready[dev] = 1;
    return IND_OK;
}

constexpr uint32_t DONE_BIT = 0x80000000u;
constexpr uint64_t EMPTY_KEY = ~0ull;
constexpr uint32_t INTERVAL_BLOCK_LIMIT = 1u << 19;  // 2^20 draws per re-prime interval
constexpr uint32_t INTERVAL_LIMIT = 1u << 26;        // empty intervals crossed in one search
// inverse-CDF guides: one entry per 2^-12 of the draw's range (its top 12
// bits) holding the number of thresholds <= the bucket's first value, with
// GUIDE_SCAN set when a threshold falls inside the bucket
constexpr int GUIDE_BITS = 12;
constexpr uint32_t GUIDE_N = 1u << GUIDE_BITS;
constexpr uint32_t GUIDE_SCAN = 0x80000000u;

struct SimParams {
    int32_t kind;
    uint32_t W, H, D;          // D: individuals per cell (non-spatial: J)
    uint32_t slot_deme;        // individuals per cell in the slot numbering (map: max deme)
    int32_t dt_log2;
    uint64_t nu_thr;           // ceil(nu 2^53)
    double lambda;
    uint32_t sk0, sk1;         // stream key of the seed
    int32_t gauss_half;
    uint32_t gauss_n;
    const uint64_t* gauss;     // 2 half discretised-normal CDF thresholds
    const uint32_t* gauss_guide;  // GUIDE_N entries
    int32_t sampler;              // 0: sums of exponentials, 1: Poisson point counts
    uint32_t pois_n;
    const uint64_t* pois_cdf;     // round(2^64 P(Poi(lambda dt) <= n))
    const uint32_t* pois_guide;   // GUIDE_N entries
    const uint8_t* deme_map;   // W*H
    const uint32_t* row_of;    // W*H alias row of a cell
    const uint64_t* alias;     // rows x n_off entries: q | alias << 32 | full << 63
    const int8_t* off;         // n_off (dx, dy)
    uint32_t n_off;
    uint32_t n_lineages;
    uint64_t slot_base;        // first global slot index of this simulation
    uint32_t gid_base;         // first global lineage id of this simulation
    uint32_t coop_short;       // lambda dt <= 2: the warp-cooperative searches look 4 intervals ahead
    uint64_t meta_size;        // spatially implicit: metacommunity individuals
    uint64_t m_thr;            // spatially implicit: ceil(migration 2^53)
    uint64_t meta_nu_thr;      // spatially implicit: ceil(meta_nu 2^53)
    const uint64_t* sample_loc;  // n_lineages sampled locations
    double events_per_round;
    double min_events;
    double occupancy_step;
    double tail_events;
    double busy_lineages;
    double max_step_events;
    double n_slots;            // indexed locations of the landscape
};

struct SimState {
    double horizon;
    uint64_t raw_events;
    uint64_t unique_events;
    uint64_t culled;
    uint64_t rounds;
    uint32_t n_active;
    uint32_t n_next;
    uint32_t culled_round;
    uint32_t done;
    uint32_t error;
    uint32_t pad;
};

struct Globals {
    uint32_t n_total;       // lineages in the current input buffer
    uint32_t n_total_next;  // survivors written by the running compaction
    uint32_t work_ctr;      // claim counter of the advance kernel
    uint32_t blocks_done;   // finished blocks of the running compaction
    uint32_t round;         // rounds completed (parity selects buffers)
    uint32_t mask[2];       // probe mask of the dedup tables
    uint32_t used[2];       // occupied-slot counts of the dedup tables
    uint32_t ev_used[2];    // occupied-slot counts of the event-count tables
    uint32_t error;
    uint32_t n_live_sims;
    unsigned long long* prof_events;  // profile: cumulative raw events after each round of a chunk
    uint32_t prof_slot;               // round index within the chunk
    uint32_t prof_n;
    uint32_t round_max;               // most events one lineage ran in the running round
    unsigned long long critical_events;  // sum of round_max over completed rounds
    unsigned long long log_n;            // events appended to the event log (may pass its capacity)
};

struct __align__(16) EvSlot {
    unsigned long long a, b;
};

struct LinPtrs {
    uint64_t* loc;
    double* tn;
    uint32_t* gid;
    uint32_t* sim;
    double* tp;  // the lineage's previous event time (event logging only, else null)
};

// the event log: every executed event, duplicates of not yet culled copies
// included (structure of arrays, cap entries)
struct EventLog {
    uint64_t* time;    // event time bits
    uint64_t* prior;   // the lineage's previous event time bits (0 at its first)
    uint64_t* loc;     // where the event happens
    uint64_t* target;  // dispersal target, ~0 for a speciation
    uint32_t* gid;     // lineage
    unsigned long long cap;
};

struct BatchDev {
    LinPtrs lin[2];
    uint32_t* parent;
    uint64_t* key_loc;
    uint64_t* key_time;
    unsigned long long* ht_key[2];
    uint32_t* ht_val[2];
    uint32_t* ht_used[2];
    EvSlot* ev[2];
    uint32_t* ev_used[2];
    uint32_t ev_mask;
    uint32_t ht_cap;
    const SimParams* P;
    SimState* S;
    Globals* G;
    uint32_t n_sims;
    uint32_t lpl;
    int dedup;
    int count_unique;
    int need_ln;  // some simulation uses the exponential-sums sampler
    uint32_t events_per_visit;
    uint32_t coop_lineages;  // a round with at most this many active lineages runs one warp per lineage
    EventLog log;            // cap 0: no logging
};

// ---------------------------------------------------------------------------
// per-lineage event arithmetic
// ---------------------------------------------------------------------------
struct LaneSim {
    uint32_t sim;
    int kind;
    uint32_t W, H, D;
    uint64_t nu_thr;
    uint32_t sk0, sk1;
    int dt_log2;
    double lam;
    bool lam1;
    double horizon;
    int sampler;
    bool coop_short;
    uint32_t pois_n;
    const uint64_t* pois_cdf;
    const uint32_t* pois_guide;
    int32_t gauss_half;
    uint32_t gauss_n;
    const uint64_t* gauss;
    const uint32_t* gauss_guide;
};

__device__ __forceinline__ void load_lanesim(LaneSim& c, const SimParams* __restrict__ P,
                                             const SimState* S, uint32_t sim) {
    const SimParams* p = P + sim;
    c.sim = sim;
    c.kind = __ldg(&p->kind);
    c.W = __ldg(&p->W);
    c.H = __ldg(&p->H);
    c.D = __ldg(&p->D);
    c.nu_thr = __ldg(&p->nu_thr);
    c.sk0 = __ldg(&p->sk0);
    c.sk1 = __ldg(&p->sk1);
    c.dt_log2 = __ldg(&p->dt_log2);
    c.lam = __ldg(&p->lambda);
    c.lam1 = (c.lam == 1.0);
    c.sampler = __ldg(&p->sampler);
    c.pois_n = __ldg(&p->pois_n);
    c.pois_cdf = p->pois_cdf;
    c.pois_guide = p->pois_guide;
    c.coop_short = __ldg(&p->coop_short) != 0u;
    c.gauss_half = __ldg(&p->gauss_half);
    c.gauss_n = __ldg(&p->gauss_n);
    c.gauss = p->gauss;
    c.gauss_guide = p->gauss_guide;
    c.horizon = *(volatile const double*)&S[sim].horizon;
}

// the logarithm tables (global, read through L1, or a block's shared copy)
struct LnC {
    const uint64_t* L;
    const uint32_t* R;
    uint64_t ln2;
    int64_t c3;
};

__device__ __forceinline__ LnC ln_tables() {
    return LnC{g_ln.L, g_ln.R, g_ln.ln2_q64, g_ln.c3};
}

constexpr size_t LN_SMEM_BYTES = sizeof(uint64_t) * LN_N + sizeof(uint32_t) * LN_N;

// copy the logarithm tables into shared memory (all threads of the block)
__device__ __forceinline__ LnC ln_tables_shared(unsigned char* smem) {
    uint4* dst = (uint4*)smem;
    const uint4* src = (const uint4*)&g_ln;  // L then R, contiguous, 16-byte aligned
    for (uint32_t i = threadIdx.x; i < LN_SMEM_BYTES / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    return LnC{(const uint64_t*)smem, (const uint32_t*)(smem + sizeof(uint64_t) * LN_N), g_ln.ln2_q64, g_ln.c3};
}

// binary64 of q 2^-58: the hardware conversion rounds q to nearest even, and
// the scaling by 2^-58 is exact (normal range), applied to the exponent field
__device__ __forceinline__ double q58_to_double_hw(uint64_t q) {
    if (q == 0ull) return 0.0;
    const uint64_t b = (uint64_t)__double_as_longlong(__ull2double_rn(q));
    return __longlong_as_double((long long)(b - (58ull << 52)));
}

// Exp(lambda) draw.  LAM1 (lambda = 1) is a template argument rather than a
// select: given both operands the compiler evaluates the binary64 division
// even where it is not used, on the latency chain and on B300's narrow FP64
// pipe.  Callers branch on c.lam1 once per search.
// the division out of line, for code whose lanes mix lambdas: a call is
// not evaluated speculatively
__device__ __noinline__ double div_rn_call(double x, double y) { return __ddiv_rn(x, y); }

template <bool LAM1>
__device__ __forceinline__ double exp_draw(uint64_t v, const LnC& ln, const LaneSim& c) {
    const double x = q58_to_double(exp1_q58(v >> 11, ln.L, ln.R, ln.ln2, ln.c3));
    if (LAM1) return x;
    return __ddiv_rn(x, c.lam);
}

// first point of loc's event process strictly after tau; negative on overflow.
// Times are non-negative binary64, so they order like their bit patterns: the
// compares, floor(tau / delta_t) and k delta_t are done on the bits.  WIDE
// blocks (2 WIDE draws) are generated and converted together; the draws of a
// step are independent, so their logarithms overlap, and only the binary64
// sums run one after another, in the spec's order.
template <int WIDE, bool LAM1>
__device__ double next_event_time_exp(const LaneSim& c, uint64_t loc, double tau, const LnC& ln) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    uint64_t k = floor_div_pow2(tau_b, c.dt_log2);
    for (uint32_t iv = 0; iv < INTERVAL_LIMIT; ++iv) {
        if (k >= (1ull << 52)) return -1.0;
        double p = __longlong_as_double((long long)k_times_pow2_bits(k, c.dt_log2));
        const uint64_t end_b = k_times_pow2_bits(k + 1ull, c.dt_log2);
        bool next_interval = false;
        for (uint32_t j = 0; j < INTERVAL_BLOCK_LIMIT; j += WIDE) {
            double x[2 * WIDE];
#pragma unroll
            for (int w = 0; w < WIDE; ++w) {
                const u64x2 b = stream_block(c.sk0, c.sk1, loc, k, j + w, TAG_INTERVAL);
                x[2 * w] = exp_draw<LAM1>(b.lo, ln, c);
                x[2 * w + 1] = exp_draw<LAM1>(b.hi, ln, c);
            }
#pragma unroll
            for (int d = 0; d < 2 * WIDE; ++d) {
                p = __dadd_rn(p, x[d]);
                const uint64_t pb = (uint64_t)__double_as_longlong(p);
                if (pb >= end_b) {
                    next_interval = true;
                    break;
                }
                if (pb > tau_b) return p;
            }
            if (next_interval) break;
        }
        if (!next_interval) return -1.0;
        ++k;
    }
    return -1.0;
}

// number of table entries <= r: the guide entry of r's bucket, and a scan
// of the table only where a threshold falls inside the bucket
__device__ __forceinline__ uint32_t guided_count(const uint64_t* __restrict__ t, const uint32_t* __restrict__ guide,
                                                 uint32_t n, uint64_t r) {
    const uint32_t e = __ldg(guide + (r >> (64 - GUIDE_BITS)));
    uint32_t idx = e & ~GUIDE_SCAN;
    if (e & GUIDE_SCAN)
        while (idx < n && __ldg(t + idx) <= r) ++idx;
    return idx;
}

// Poisson method: interval k holds N ~ Poi(lambda dt) points (N = the count
// of CDF thresholds <= draw 0), point i at k dt + U dt, U = (draw (1 + i)
// >> 11) 2^-53, the sum rounded to nearest; the next event is the smallest
// point > tau of the first interval that has one.  The points of an interval
// are independent of each other, so there is no sequential chain.
__device__ double next_event_time_poisson(const LaneSim& c, uint64_t loc, double tau) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    uint64_t k = floor_div_pow2(tau_b, c.dt_log2);
    for (uint32_t iv = 0; iv < INTERVAL_LIMIT; ++iv) {
        if (k >= (1ull << 52)) return -1.0;
        const double base = __longlong_as_double((long long)k_times_pow2_bits(k, c.dt_log2));
        const u64x2 b0 = stream_block(c.sk0, c.sk1, loc, k, 0, TAG_INTERVAL);
        const uint32_t N = guided_count(c.pois_cdf, c.pois_guide, c.pois_n, b0.lo);
        uint64_t best = ~0ull;
        auto consider = [&](uint64_t r) {
            const double x = q53_scaled(r >> 11, c.dt_log2 - 53);  // U dt, exact
            const uint64_t pb = (uint64_t)__double_as_longlong(__dadd_rn(base, x));
            if (pb > tau_b && pb < best) best = pb;
        };
        if (N >= 1) consider(b0.hi);
        for (uint32_t j = 1; 2 * j <= N; ++j) {
            const u64x2 bj = stream_block(c.sk0, c.sk1, loc, k, j, TAG_INTERVAL);
            consider(bj.lo);
            if (2 * j + 1 <= N) consider(bj.hi);
        }
        if (best != ~0ull) return __longlong_as_double((long long)best);
        ++k;
    }
    return -1.0;
}

// the searches return a time >= 0, or -1 when they give up: a sign-bit test
// rather than a binary64 compare, which is slow on B300 and on the chain
__device__ __forceinline__ bool search_failed(double t) { return __double_as_longlong(t) < 0; }

template <int WIDE>
__device__ __forceinline__ double next_event_time(const LaneSim& c, uint64_t loc, double tau, const LnC& ln) {
    if (c.sampler == 1) return next_event_time_poisson(c, loc, tau);
    return c.lam1 ? next_event_time_exp<WIDE, true>(c, loc, tau, ln) : next_event_time_exp<WIDE, false>(c, loc, tau, ln);
}

// ---------------------------------------------------------------------------
// Warp-cooperative next-event searches (one lineage per warp; every lane
// returns the same time).  They compute exactly what the one-lane searches
// compute; the lanes only evaluate draws that the one-lane search may need,
// ahead of time and side by side.
// ---------------------------------------------------------------------------
// Poisson sampler: lane l searches interval k + l (k = floor(tau / dt)); the
// answer is the smallest point > tau of the lowest interval that has one.
__device__ double coop_next_poisson(const LaneSim& c, uint64_t loc, double tau, uint32_t lane) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    const uint64_t k0 = floor_div_pow2(tau_b, c.dt_log2);
    for (uint32_t round = 0; round < INTERVAL_LIMIT / 32; ++round) {
        const uint64_t k = k0 + 32ull * round + lane;
        uint64_t best = ~0ull;
        if (k < (1ull << 52)) {
            const double base = __longlong_as_double((long long)k_times_pow2_bits(k, c.dt_log2));
            const u64x2 b0 = stream_block(c.sk0, c.sk1, loc, k, 0, TAG_INTERVAL);
            const uint32_t N = guided_count(c.pois_cdf, c.pois_guide, c.pois_n, b0.lo);
            auto consider = [&](uint64_t r) {
                const double x = q53_scaled(r >> 11, c.dt_log2 - 53);  // U dt, exact
                const uint64_t pb = (uint64_t)__double_as_longlong(__dadd_rn(base, x));
                if (pb > tau_b && pb < best) best = pb;
            };
            if (N >= 1) consider(b0.hi);
            for (uint32_t j = 1; 2 * j <= N; ++j) {
                const u64x2 bj = stream_block(c.sk0, c.sk1, loc, k, j, TAG_INTERVAL);
                consider(bj.lo);
                if (2 * j + 1 <= N) consider(bj.hi);
            }
        }
        const unsigned found = __ballot_sync(0xFFFFFFFFu, best != ~0ull);
        if (found) return __longlong_as_double((long long)__shfl_sync(0xFFFFFFFFu, best, __ffs(found) - 1));
        if (k0 + 32ull * round + 32ull >= (1ull << 52)) return -1.0;
    }
    return -1.0;
}

// Sums of exponentials: in each step lanes 0-15 hold draws 16 qa .. 16 qa + 15
// of interval k and lanes 16-31 draws 0 .. 15 of interval k + 1, all
// converted side by side; the binary64 running sums then follow the spec's
// order one draw at a time (shuffled from the lane that holds it).
template <bool LAM1>
__device__ double coop_next_exp(const LaneSim& c, uint64_t loc, double tau, const LnC& ln, uint32_t lane) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    uint64_t k = floor_div_pow2(tau_b, c.dt_log2);
    uint32_t qa = 0;  // 16-draw groups of interval k already summed
    double p = 0.0;   // running sum of interval k (valid when qa > 0)
    for (uint32_t it = 0; it < INTERVAL_LIMIT; ++it) {
        if (k + 2ull >= (1ull << 52) || qa >= 2u * INTERVAL_BLOCK_LIMIT / 16u) return -1.0;
        if (qa == 0) p = __longlong_as_double((long long)k_times_pow2_bits(k, c.dt_log2));
        const uint64_t end_b = k_times_pow2_bits(k + 1ull, c.dt_log2);
        const uint64_t kk = lane < 16u ? k : k + 1ull;
        const uint32_t d = lane < 16u ? 16u * qa + lane : lane - 16u;
        const u64x2 b = stream_block(c.sk0, c.sk1, loc, kk, d >> 1, TAG_INTERVAL);
        const double x = exp_draw<LAM1>((d & 1u) ? b.hi : b.lo, ln, c);
        bool done_k = false;
        for (uint32_t i = 0; i < 16u; ++i) {
            p = __dadd_rn(p, __shfl_sync(0xFFFFFFFFu, x, i));
            const uint64_t pb = (uint64_t)__double_as_longlong(p);
            if (pb >= end_b) {
                done_k = true;
                break;
            }
            if (pb > tau_b) return p;
        }
        if (!done_k) {  // interval k goes on: its next 16 draws in the next step
            ++qa;
            continue;
        }
        // interval k + 1 from its first 16 draws (lanes 16-31)
        double p1 = __longlong_as_double((long long)k_times_pow2_bits(k + 1ull, c.dt_log2));
        const uint64_t end1_b = k_times_pow2_bits(k + 2ull, c.dt_log2);
        bool done_k1 = false;
        for (uint32_t i = 0; i < 16u; ++i) {
            p1 = __dadd_rn(p1, __shfl_sync(0xFFFFFFFFu, x, 16 + i));
            const uint64_t pb = (uint64_t)__double_as_longlong(p1);
            if (pb >= end1_b) {
                done_k1 = true;
                break;
            }
            if (pb > tau_b) return p1;
        }
        if (done_k1) {
            k += 2ull;
            qa = 0;
        } else {  // interval k + 1 needs more than 16 draws: go on from draw 16
            k += 1ull;
            qa = 1;
            p = p1;
        }
    }
    return -1.0;
}

// Short searches (lambda dt <= 2, and >= 1/2 for Poisson points): lanes
// 8 m .. 8 m + 7 take interval k + m (m = 0..3, k = floor(tau / dt)), lane
// 8 m + i the interval's point i.  Intervals of more than 8 points are rare
// here (Poi(2) > 8: 2.4e-4 of intervals); the search then starts again in
// the general form above.  Four intervals without an answer: go on at k + 4.
__device__ double coop_next_poisson_short(const LaneSim& c, uint64_t loc, double tau, uint32_t lane) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    const uint32_t m = lane >> 3, i = lane & 7u;
    uint64_t k0 = floor_div_pow2(tau_b, c.dt_log2);
    for (uint32_t round = 0; round < INTERVAL_LIMIT / 4; ++round, k0 += 4ull) {
        if (k0 + 4ull >= (1ull << 52)) return coop_next_poisson(c, loc, tau, lane);
        const uint64_t k = k0 + m;
        // draw 0 gives the count N; point i is draw 1 + i
        const u64x2 b0 = stream_block(c.sk0, c.sk1, loc, k, 0, TAG_INTERVAL);
        const u64x2 bi = stream_block(c.sk0, c.sk1, loc, k, (1u + i) >> 1, TAG_INTERVAL);
        const uint32_t N = guided_count(c.pois_cdf, c.pois_guide, c.pois_n, b0.lo);
        uint64_t pb = ~0ull;
        if (i < N) {
            const uint64_t r = (i & 1u) ? bi.lo : bi.hi;
            const double base = __longlong_as_double((long long)k_times_pow2_bits(k, c.dt_log2));
            const uint64_t q = (uint64_t)__double_as_longlong(__dadd_rn(base, q53_scaled(r >> 11, c.dt_log2 - 53)));
            if (q > tau_b) pb = q;
        }
        if (__any_sync(0xFFFFFFFFu, N > 8u)) return coop_next_poisson(c, loc, tau, lane);
        // the smallest point > tau of the four intervals is the smallest of
        // the first interval that has one: points of interval k lie in
        // [k dt, (k + 1) dt], rounding included
        const uint32_t hi = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(pb >> 32));
        if (hi != 0xFFFFFFFFu) {
            const uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(pb >> 32) == hi ? (uint32_t)pb : 0xFFFFFFFFu);
            return __longlong_as_double((long long)(((uint64_t)hi << 32) | lo));
        }
    }
    return -1.0;
}

// sums of exponentials: every lane runs interval k's binary64 running sum in
// the spec's order on the shuffled draws; intervals k + 1 .. k + 3 only need
// their first point
template <bool LAM1>
__device__ double coop_next_exp_short(const LaneSim& c, uint64_t loc, double tau, const LnC& ln, uint32_t lane) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    const uint32_t m = lane >> 3, i = lane & 7u;
    uint64_t k0 = floor_div_pow2(tau_b, c.dt_log2);
    for (uint32_t round = 0; round < INTERVAL_LIMIT / 4; ++round, k0 += 4ull) {
        if (k0 + 4ull >= (1ull << 52)) return coop_next_exp<LAM1>(c, loc, tau, ln, lane);
        const uint64_t k = k0 + m;
        const u64x2 b = stream_block(c.sk0, c.sk1, loc, k, i >> 1, TAG_INTERVAL);
        const double x = exp_draw<LAM1>((i & 1u) ? b.hi : b.lo, ln, c);
        double xs[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) xs[j] = __shfl_sync(0xFFFFFFFFu, x, j);
        // first point of interval k (lanes 8 m), kept if inside the interval
        const double first = __dadd_rn(__longlong_as_double((long long)k_times_pow2_bits(k, c.dt_log2)), x);
        const bool has = i == 0u && m > 0u &&
                         (uint64_t)__double_as_longlong(first) < k_times_pow2_bits(k + 1ull, c.dt_log2);
        double p = __longlong_as_double((long long)k_times_pow2_bits(k0, c.dt_log2));
        const uint64_t end0 = k_times_pow2_bits(k0 + 1ull, c.dt_log2);
        int state = 0;  // 1: point after tau, 2: interval k0 ended first
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            p = __dadd_rn(p, xs[j]);
            const uint64_t pb = (uint64_t)__double_as_longlong(p);
            if (pb >= end0) {
                state = 2;
                break;
            }
            if (pb > tau_b) {
                state = 1;
                break;
            }
        }
        if (state == 1) return p;
        if (state == 0) return coop_next_exp<LAM1>(c, loc, tau, ln, lane);
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, has);
        if (bal) return __shfl_sync(0xFFFFFFFFu, first, __ffs(bal) - 1);
    }
    return -1.0;
}

// dispersal target from the event stream's draws 1, 2, 3 (draw 0 decided
// speciation): non-spatial uses d1; torus d1 (x), d2 (y), d3 (deme index),
// each axis a discretised normal by inversion, -half + #{k : cdf[k] <= d};
// map d1 (alias column and threshold), d2 (deme index); spatially implicit
// d1 (migration, or the metacommunity parent), d2 (parent after migration
// or locally)
// (KIND: the landscape kind when the caller knows it at compile time, -1
// for the simulation's own)
template <int KIND = -1>
__device__ __forceinline__ uint64_t disperse(const LaneSim& c, const SimParams* __restrict__ P, uint64_t loc,
                                            uint64_t d1, uint64_t d2, uint64_t d3) {
    const int kind = KIND >= 0 ? KIND : c.kind;
    if (kind == KIND_NONSPATIAL) return pack_loc(0, 0, umulhi64(d1, c.D));
    const SimParams* p = P + c.sim;
    if (kind == KIND_IMPLICIT) {
        // in the metacommunity: a uniform parent there (d1); locally:
        // migration iff d1 says so, then the parent's index (d2) in the
        // metacommunity or the local community
        const uint64_t meta_n = __ldg(&p->meta_size);
        if (in_meta(loc)) return meta_loc(umulhi64(d1, meta_n));
        if ((d1 >> 11) < __ldg(&p->m_thr)) return meta_loc(umulhi64(d2, meta_n));
        return pack_loc(0, 0, umulhi64(d2, c.D));
    }
    const uint32_t x = loc_x(loc), y = loc_y(loc);
    if (kind == KIND_TORUS) {
        // both guide entries first, so that the two loads overlap; a table
        // scan only for draws in a bucket that holds a threshold
        const uint32_t ex = __ldg(c.gauss_guide + (d1 >> (64 - GUIDE_BITS)));
        const uint32_t ey = __ldg(c.gauss_guide + (d2 >> (64 - GUIDE_BITS)));
        uint32_t cx = ex & ~GUIDE_SCAN, cy = ey & ~GUIDE_SCAN;
        if ((ex | ey) & GUIDE_SCAN) {
            if (ex & GUIDE_SCAN)
                while (cx < c.gauss_n && __ldg(c.gauss + cx) <= d1) ++cx;
            if (ey & GUIDE_SCAN)
                while (cy < c.gauss_n && __ldg(c.gauss + cy) <= d2) ++cy;
        }
        const uint32_t tx = wrap_add(x, (int32_t)cx - c.gauss_half, c.W);
        const uint32_t ty = wrap_add(y, (int32_t)cy - c.gauss_half, c.H);
        const uint64_t ti = c.D > 1 ? umulhi64(d3, c.D) : 0ull;
        return pack_loc(tx, ty, ti);
    }
    // habitat map: alias row of the origin cell
    const uint32_t n_off = __ldg(&p->n_off);
    const uint32_t row = __ldg(p->row_of + (size_t)y * c.W + x);
    const uint32_t col = (uint32_t)(((d1 >> 32) * (uint64_t)n_off) >> 32);
    const uint64_t e = __ldg(p->alias + (size_t)row * n_off + col);
    const uint32_t u = (uint32_t)d1;
    const uint32_t o = ((e >> 63) != 0 || u < (uint32_t)e) ? col : (uint32_t)((e >> 32) & 0xFFFFu);
    const int8_t* off = p->off;
    const int32_t dx = off[2 * o], dy = off[2 * o + 1];
    const uint32_t tx = wrap_add(x, dx, c.W);
    const uint32_t ty = wrap_add(y, dy, c.H);
    const uint32_t d = __ldg(p->deme_map + (size_t)ty * c.W + tx);
    return pack_loc(tx, ty, umulhi64(d2, d));
}

// speciation threshold at loc: the metacommunity's in the spatially
// implicit model, else the simulation's
__device__ __forceinline__ uint64_t spec_thr(const LaneSim& c, const SimParams* __restrict__ P, int kind,
                                             uint64_t loc) {
    return (kind == KIND_IMPLICIT && in_meta(loc)) ? __ldg(&P[c.sim].meta_nu_thr) : c.nu_thr;
}

// one event at (loc, tau); returns true if the lineage speciated, else
// moves loc to the dispersal target
__device__ __forceinline__ bool do_event(const LaneSim& c, const SimParams* __restrict__ P, uint64_t& loc,
                                         double tau) {
    const uint64_t tk = (uint64_t)__double_as_longlong(tau);
    const u64x2 b0 = stream_block(c.sk0, c.sk1, loc, tk, 0, TAG_EVENT);
    if (c.kind == KIND_NONSPATIAL || (c.kind == KIND_IMPLICIT && in_meta(loc))) {
        if ((b0.lo >> 11) < spec_thr(c, P, c.kind, loc)) return true;
        loc = disperse(c, P, loc, b0.hi, 0ull, 0ull);
        return false;
    }
    const u64x2 b1 = stream_block(c.sk0, c.sk1, loc, tk, 1, TAG_EVENT);
    if ((b0.lo >> 11) < c.nu_thr) return true;
    loc = disperse(c, P, loc, b0.hi, b1.lo, b1.hi);
    return false;
}

// do_event for one lineage per warp: lanes of even and odd index compute
// the event stream's blocks 0 and 1 side by side, then every lane takes the
// four draws by shuffle (one block's latency instead of two interleaved)
template <int KIND>
__device__ __forceinline__ bool do_event_warp(const LaneSim& c, const SimParams* __restrict__ P, uint64_t& loc,
                                              double tau, uint32_t lane) {
    const int kind = KIND >= 0 ? KIND : c.kind;
    const uint64_t tk = (uint64_t)__double_as_longlong(tau);
    if (kind == KIND_NONSPATIAL) {
        const u64x2 b0 = stream_block(c.sk0, c.sk1, loc, tk, 0, TAG_EVENT);
        if ((b0.lo >> 11) < c.nu_thr) return true;
        loc = disperse<KIND_NONSPATIAL>(c, P, loc, b0.hi, 0ull, 0ull);
        return false;
    }
    const u64x2 b = stream_block(c.sk0, c.sk1, loc, tk, lane & 1u, TAG_EVENT);
    const uint64_t d0 = __shfl_sync(0xFFFFFFFFu, b.lo, 0), d1 = __shfl_sync(0xFFFFFFFFu, b.hi, 0);
    const uint64_t d2 = __shfl_sync(0xFFFFFFFFu, b.lo, 1), d3 = __shfl_sync(0xFFFFFFFFu, b.hi, 1);
    if ((d0 >> 11) < spec_thr(c, P, kind, loc)) return true;
    loc = disperse<KIND>(c, P, loc, d1, d2, d3);
    return false;
}

// global slot index of a location: cells row-major x slot_deme + deme
// index, after the simulation's slot_base; the spatially implicit model
// numbers its J local individuals first, then the metacommunity
__device__ __forceinline__ uint64_t slot_index(const SimParams* __restrict__ p, uint64_t loc) {
    const uint64_t base = __ldg(&p->slot_base);
    if (__ldg(&p->kind) == KIND_IMPLICIT)
        return base + (in_meta(loc) ? (uint64_t)__ldg(&p->D) + meta_index(loc) : (uint64_t)loc_i(loc));
    const uint64_t cell = (uint64_t)loc_y(loc) * __ldg(&p->W) + loc_x(loc);
    return base + cell * __ldg(&p->slot_deme) + loc_i(loc);
}

__device__ __forceinline__ uint64_t slot_key(const SimParams* __restrict__ P, const LaneSim& c, uint64_t loc) {
    return slot_index(P + c.sim, loc);
}

// exact distinct-event counting: insert (slot, time bits); true if new
__device__ __forceinline__ bool count_event(const BatchDev& B, uint32_t t, uint64_t skey, double tau) {
    EvSlot mine;
    mine.a = skey;
    mine.b = (unsigned long long)__double_as_longlong(tau);
    EvSlot empty;
    empty.a = EMPTY_KEY;
    empty.b = EMPTY_KEY;
    uint32_t h = (uint32_t)mix64(skey ^ (mine.b * 0x9E3779B97F4A7C15ull)) & B.ev_mask;
    for (uint32_t probe = 0; probe <= B.ev_mask; ++probe) {
        EvSlot old = atomicCAS(&B.ev[t][h], empty, mine);
        if (old.a == EMPTY_KEY && old.b == EMPTY_KEY) {
            uint32_t k = atomicAdd(&B.G->ev_used[t], 1u);
            B.ev_used[t][k] = h;
            return true;
        }
        if (old.a == mine.a && old.b == mine.b) return false;
        h = (h + 1u) & B.ev_mask;
    }
    atomicOr(&B.G->error, 2u);
    return false;
}

// log target of a culled lineage's pending event: the lineage does not
// execute it (its winner does), but its copy carries its own prior time, so
// that a coalescence stays visible in the stream
constexpr uint64_t LOG_CULLED = ~1ull;

// append one executed event to the log; past the capacity the run fails
// with a device error (error bit 8) and the entry is dropped
__device__ __forceinline__ void log_event(const BatchDev& B, double tn, double tp, uint64_t loc, uint64_t target,
                                          uint32_t gid) {
    const unsigned long long k = atomicAdd(&B.G->log_n, 1ull);
    if (k < B.log.cap) {
        B.log.time[k] = (uint64_t)__double_as_longlong(tn);
        B.log.prior[k] = (uint64_t)__double_as_longlong(tp);
        B.log.loc[k] = loc;
        B.log.target[k] = target;
        B.log.gid[k] = gid;
    } else {
        atomicOr(&B.G->error, 8u);
    }
}

// event records of one warp: lane k holds the k-th pending one; a flush
// takes one atomic for all of them, so that the log costs no round trip on
// a lone lineage's chain of events
struct WarpLogBuf {
    uint64_t time, prior, loc, target;
    uint32_t gid;
    uint32_t n;  // records held (the same in every lane)
};

__device__ __forceinline__ void warp_log_flush(const BatchDev& B, WarpLogBuf& w, uint32_t lane) {
    if (w.n == 0) return;
    unsigned long long k0 = 0;
    if (lane == 0) k0 = atomicAdd(&B.G->log_n, (unsigned long long)w.n);
    k0 = __shfl_sync(0xFFFFFFFFu, k0, 0);
    if (lane < w.n) {
        const unsigned long long k = k0 + lane;
        if (k < B.log.cap) {
            B.log.time[k] = w.time;
            B.log.prior[k] = w.prior;
            B.log.loc[k] = w.loc;
            B.log.target[k] = w.target;
            B.log.gid[k] = w.gid;
        } else {
            atomicOr(&B.G->error, 8u);
        }
    }
    w.n = 0;
}

__device__ __forceinline__ void warp_log_event(const BatchDev& B, WarpLogBuf& w, uint32_t lane, double tn, double tp,
                                               uint64_t loc, uint64_t target, uint32_t gid) {
    if (lane == w.n) {
        w.time = (uint64_t)__double_as_longlong(tn);
        w.prior = (uint64_t)__double_as_longlong(tp);
        w.loc = loc;
        w.target = target;
        w.gid = gid;
    }
    if (++w.n == 32u) warp_log_flush(B, w, lane);
}

__device__ __forceinline__ void dedup_insert(const BatchDev& B, uint32_t t, uint64_t skey, uint32_t gid) {
    const uint32_t mask = B.G->mask[t];
    uint32_t h = (uint32_t)mix64(skey) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long old = atomicCAS(&B.ht_key[t][h], EMPTY_KEY, (unsigned long long)skey);
        if (old == EMPTY_KEY) {
            uint32_t k = atomicAdd(&B.G->used[t], 1u);
            B.ht_used[t][k] = h;
            atomicMin(&B.ht_val[t][h], gid);
            return;
        }
        if (old == skey) {
            atomicMin(&B.ht_val[t][h], gid);
            return;
        }
        h = (h + 1u) & mask;
    }
    atomicOr(&B.G->error, 4u);
}

__device__ __forceinline__ uint32_t dedup_lookup(const BatchDev& B, uint32_t t, uint64_t skey) {
    const uint32_t mask = B.G->mask[t];
    uint32_t h = (uint32_t)mix64(skey) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long k = B.ht_key[t][h];
        if (k == skey) return B.ht_val[t][h];
        if (k == EMPTY_KEY) break;
        h = (h + 1u) & mask;
    }
    return 0xFFFFFFFFu;
}

// warp-aggregated add of v to ctr[sim] over the lanes of mask
__device__ __forceinline__ void warp_add_by_sim(unsigned mask, uint32_t sim, uint64_t v, uint64_t* base,
                                                size_t stride_bytes) {
    if (!mask) return;
    const unsigned grp = __match_any_sync(mask, sim);
    const int leader = __ffs(grp) - 1;
    uint64_t sum = 0;
    // reduce within the group: every lane contributes, the leader adds
    for (int l = 0; l < 32; ++l) {
        if (!((mask >> l) & 1u)) continue;
        uint64_t x = __shfl_sync(mask, v, l);
        if ((grp >> l) & 1u) sum += x;
    }
    if ((int)(threadIdx.x & 31) == leader && sum)
        atomicAdd((unsigned long long*)((char*)base + stride_bytes * sim), (unsigned long long)sum);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__global__ void k_init(BatchDev B, const uint32_t* __restrict__ gid_base, uint32_t n_lin) {
    const LnC ln = ln_tables();
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_lin; g += gridDim.x * blockDim.x) {
        // simulation of lineage g: last s with gid_base[s] <= g
        uint32_t lo = 0, hi = B.n_sims;
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (gid_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        LaneSim c;
        load_lanesim(c, B.P, B.S, lo);
        const uint64_t loc = B.P[lo].sample_loc[g - gid_base[lo]];
        double t = next_event_time<1>(c, loc, 0.0, ln);
        if (search_failed(t)) {
            atomicOr(&B.S[lo].error, 1u);
            atomicOr(&B.G->error, 1u);
            t = INFINITY;
        }
        B.lin[0].loc[g] = loc;
        B.lin[0].tn[g] = t;
        B.lin[0].gid[g] = g;
        B.lin[0].sim[g] = lo;
        if (B.lin[0].tp) B.lin[0].tp[g] = 0.0;
        B.parent[g] = g;
    }
}

// LOG: append every executed event to the event log
template <bool COUNT, int WIDE, bool LOG>
__global__ void __launch_bounds__(512) k_advance(BatchDev B) {
    extern __shared__ __align__(16) unsigned char adv_smem[];
    const uint32_t n = B.G->n_total;
    if (n <= B.coop_lineages) return;  // a round for k_advance_coop
    const uint32_t chunk = 32u * B.lpl;
    // a block whose first possible claim lies beyond the active lineages has
    // nothing to do (claims go out in order of arrival, at most one per warp)
    if ((uint64_t)blockIdx.x * (blockDim.x >> 5) * chunk >= n) return;
    // the logarithm tables are staged only if some simulation sums exponentials
    const LnC ln = B.need_ln ? ln_tables_shared(adv_smem) : ln_tables();

    const uint32_t t = B.G->round & 1u;
    const LinPtrs L = B.lin[t];
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    uint32_t chunk_next = 0, chunk_end = 0;  // warp-uniform
    bool exhausted = false;

    bool has = false;
    uint32_t idx = 0, gid = 0;
    uint64_t loc = 0;
    double tn = 0.0, tprev = 0.0;
    LaneSim c;
    c.sim = 0xFFFFFFFFu;
    uint64_t ev_raw = 0, ev_unique = 0;
    uint32_t cnt_sim = 0xFFFFFFFFu;
    uint32_t ev_lin = 0, lane_max = 0;  // events of the lane's lineage this round, and their maximum

    for (;;) {
        unsigned need = __ballot_sync(0xFFFFFFFFu, !has);
        if (need) {
            if (chunk_next >= chunk_end && !exhausted) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&B.G->work_ctr, chunk);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (base >= n) {
                    exhausted = true;
                } else {
                    chunk_next = base;
                    chunk_end = min(base + chunk, n);
                }
            }
            if (chunk_next < chunk_end) {
                const uint32_t avail = chunk_end - chunk_next;
                const uint32_t rank = __popc(need & lt_mask);
                if (!has && rank < avail) {
                    idx = chunk_next + rank;
                    gid = L.gid[idx];
                    loc = L.loc[idx];
                    tn = L.tn[idx];
                    if (LOG) tprev = L.tp[idx];
                    const uint32_t s = L.sim[idx];
                    if (s != c.sim) {
                        if (cnt_sim != 0xFFFFFFFFu && (ev_raw | ev_unique)) {
                            atomicAdd((unsigned long long*)&B.S[cnt_sim].raw_events, (unsigned long long)ev_raw);
                            if (COUNT)
                                atomicAdd((unsigned long long*)&B.S[cnt_sim].unique_events,
                                          (unsigned long long)ev_unique);
                            ev_raw = ev_unique = 0;
                        }
                        load_lanesim(c, B.P, B.S, s);
                        cnt_sim = s;
                    }
                    has = true;
                    ev_lin = 0;
                }
                chunk_next += min(avail, (uint32_t)__popc(need));
            }
        }
        if (!__any_sync(0xFFFFFFFFu, has)) {
            if (exhausted) break;
            continue;
        }
        // up to events_per_visit events of the lane's lineage between warp votes
        for (uint32_t visit = 0; has && visit < B.events_per_visit; ++visit) {
            // both non-negative: compare the bit patterns (an integer compare)
            if ((uint64_t)__double_as_longlong(tn) > (uint64_t)__double_as_longlong(c.horizon)) {
                // at the horizon: write back and enter the dedup
                L.loc[idx] = loc;
                L.tn[idx] = tn;
                if (LOG) L.tp[idx] = tprev;
                if (B.dedup) dedup_insert(B, t, slot_key(B.P, c, loc), gid);
                has = false;
            } else {
                ++ev_raw;
                lane_max = max(lane_max, ++ev_lin);
                if (COUNT) ev_unique += count_event(B, t, slot_key(B.P, c, loc), tn) ? 1u : 0u;
                const uint64_t at = loc;
                const bool speciated = do_event(c, B.P, loc, tn);
                if (LOG) {
                    log_event(B, tn, tprev, at, speciated ? ~0ull : loc, gid);
                    tprev = tn;
                }
                if (speciated) {
                    B.key_loc[gid] = loc;
                    B.key_time[gid] = (uint64_t)__double_as_longlong(tn);
                    L.gid[idx] = gid | DONE_BIT;
                    has = false;
                } else {
                    const double nt = next_event_time<WIDE>(c, loc, tn, ln);
                    if (search_failed(nt)) {
                        atomicOr(&B.S[c.sim].error, 1u);
                        atomicOr(&B.G->error, 1u);
                        B.key_loc[gid] = ~0ull;
                        B.key_time[gid] = ~0ull;
                        L.gid[idx] = gid | DONE_BIT;
                        has = false;
                    } else {
                        tn = nt;
                    }
                }
            }
        }
    }
    // flush the event counters, aggregated over lanes of the same simulation
    const bool valid = cnt_sim != 0xFFFFFFFFu;
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    if (valid) {
        warp_add_by_sim(vm, cnt_sim, ev_raw, &B.S[0].raw_events, sizeof(SimState));
        if (COUNT) warp_add_by_sim(vm, cnt_sim, ev_unique, &B.S[0].unique_events, sizeof(SimState));
    }
    const uint32_t wmax = __reduce_max_sync(0xFFFFFFFFu, lane_max);
    if (lane == 0 && wmax) atomicMax(&B.G->round_max, wmax);
}

// Throughput phase, convergent form: every iteration each lane computes
// exactly one Philox block whose counter depends on the lane's state (event
// block 0 or 1, or the next block of its re-prime interval search), so the
// bulk of the instructions runs with all lanes active; only the short
// state-specific processing diverges.  Lanes refill from the warp's chunk
// whenever they fall idle.  Same draws, same order, same results as the
// one-lane-per-lineage loop above.
constexpr uint32_t SM_IDLE = 0, SM_EVENT0 = 1, SM_EVENT1 = 2, SM_SEARCH = 3;

template <bool COUNT>
__global__ void __launch_bounds__(512) k_advance_sm(BatchDev B) {
    extern __shared__ __align__(16) unsigned char adv_smem[];
    const uint32_t n = B.G->n_total;
    if (n <= B.coop_lineages) return;  // a round for k_advance_coop
    const uint32_t chunk = 32u * B.lpl;
    if ((uint64_t)blockIdx.x * (blockDim.x >> 5) * chunk >= n) return;
    const LnC ln = B.need_ln ? ln_tables_shared(adv_smem) : ln_tables();
    const uint32_t t = B.G->round & 1u;
    const LinPtrs L = B.lin[t];
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    uint32_t chunk_next = 0, chunk_end = 0;  // warp-uniform
    bool exhausted = false;

    uint32_t st = SM_IDLE, idx = 0, gid = 0;
    uint64_t loc = 0;
    double tn = 0.0;
    LaneSim c;
    memset(&c, 0, sizeof(c));
    c.sim = 0xFFFFFFFFu;
    c.lam = 1.0;
    c.lam1 = true;
    uint64_t hz = 0;                          // horizon bits of the lane's simulation
    uint64_t k = 0, tau_b = 0, end_b = 0, best = ~0ull, e0hi = 0;
    uint32_t j = 0, N = 0, iv = 0;
    double p = 0.0, base = 0.0;
    uint64_t ev_raw = 0, ev_unique = 0;
    uint32_t cnt_sim = 0xFFFFFFFFu;
    uint32_t ev_lin = 0, lane_max = 0;  // events of the lane's lineage this round, and their maximum

    auto fail = [&]() {
        atomicOr(&B.S[c.sim].error, 1u);
        atomicOr(&B.G->error, 1u);
        B.key_loc[gid] = ~0ull;
        B.key_time[gid] = ~0ull;
        L.gid[idx] = gid | DONE_BIT;
        st = SM_IDLE;
    };
    auto start_interval = [&]() {
        base = __longlong_as_double((long long)k_times_pow2_bits(k, c.dt_log2));
        end_b = k_times_pow2_bits(k + 1ull, c.dt_log2);
        p = base;
        best = ~0ull;
        N = 0;
        j = 0;
        if (k >= (1ull << 52) || iv >= INTERVAL_LIMIT) fail();
    };
    auto begin_search = [&]() {
        tau_b = (uint64_t)__double_as_longlong(tn);
        k = floor_div_pow2(tau_b, c.dt_log2);
        iv = 0;
        st = SM_SEARCH;
        start_interval();
    };
    auto found = [&](double v) {
        tn = v;
        if ((uint64_t)__double_as_longlong(tn) > hz) {  // beyond the horizon: park the lineage
            L.loc[idx] = loc;
            L.tn[idx] = tn;
            if (B.dedup) dedup_insert(B, t, slot_key(B.P, c, loc), gid);
            st = SM_IDLE;
        } else {
            st = SM_EVENT0;
        }
    };

    for (;;) {
        // refill idle lanes from the warp's chunk
        const unsigned need = __ballot_sync(0xFFFFFFFFu, st == SM_IDLE);
        if (need) {
            if (chunk_next >= chunk_end && !exhausted) {
                uint32_t b0 = 0;
                if (lane == 0) b0 = atomicAdd(&B.G->work_ctr, chunk);
                b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
                if (b0 >= n) {
                    exhausted = true;
                } else {
                    chunk_next = b0;
                    chunk_end = min(b0 + chunk, n);
                }
            }
            if (chunk_next < chunk_end) {
                const uint32_t avail = chunk_end - chunk_next;
                const uint32_t rank = __popc(need & lt_mask);
                if (st == SM_IDLE && rank < avail) {
                    idx = chunk_next + rank;
                    gid = L.gid[idx];
                    loc = L.loc[idx];
                    tn = L.tn[idx];
                    const uint32_t s = L.sim[idx];
                    if (s != c.sim) {
                        if (cnt_sim != 0xFFFFFFFFu && (ev_raw | ev_unique)) {
                            atomicAdd((unsigned long long*)&B.S[cnt_sim].raw_events, (unsigned long long)ev_raw);
                            if (COUNT)
                                atomicAdd((unsigned long long*)&B.S[cnt_sim].unique_events,
                                          (unsigned long long)ev_unique);
                            ev_raw = ev_unique = 0;
                        }
                        load_lanesim(c, B.P, B.S, s);
                        cnt_sim = s;
                        hz = (uint64_t)__double_as_longlong(c.horizon);
                    }
                    ev_lin = 0;
                    if ((uint64_t)__double_as_longlong(tn) > hz) {
                        if (B.dedup) dedup_insert(B, t, slot_key(B.P, c, loc), gid);  // already at the horizon
                    } else {
                        st = SM_EVENT0;
                    }
                }
                chunk_next += min(avail, (uint32_t)__popc(need));
            }
        }
        if (!__any_sync(0xFFFFFFFFu, st != SM_IDLE)) {
            if (exhausted) break;
            continue;
        }
        // one Philox block per lane, its counter chosen by the lane's state
        const bool ev = st == SM_EVENT0 || st == SM_EVENT1;
        const uint64_t tkey = ev ? (uint64_t)__double_as_longlong(tn) : k;
        const uint32_t jj = ev ? (st == SM_EVENT1 ? 1u : 0u) : j;
        const u64x2 b = stream_block(c.sk0, c.sk1, loc, tkey, jj, ev ? TAG_EVENT : TAG_INTERVAL);
        // the two exponentials of the block, when some lane of the warp sums them
        double x0 = 0.0, x1 = 0.0;
        if (__any_sync(0xFFFFFFFFu, st == SM_SEARCH && c.sampler == 0)) {
            x0 = exp_draw<true>(b.lo, ln, c);
            x1 = exp_draw<true>(b.hi, ln, c);
            if (!c.lam1) {
                x0 = div_rn_call(x0, c.lam);
                x1 = div_rn_call(x1, c.lam);
            }
        }
        if (st == SM_EVENT0) {
            ++ev_raw;
            lane_max = max(lane_max, ++ev_lin);
            if (COUNT) ev_unique += count_event(B, t, slot_key(B.P, c, loc), tn) ? 1u : 0u;
            if ((b.lo >> 11) < spec_thr(c, B.P, c.kind, loc)) {
                B.key_loc[gid] = loc;
                B.key_time[gid] = (uint64_t)__double_as_longlong(tn);
                L.gid[idx] = gid | DONE_BIT;
                st = SM_IDLE;
            } else if (c.kind == KIND_NONSPATIAL || (c.kind == KIND_IMPLICIT && in_meta(loc))) {
                loc = disperse(c, B.P, loc, b.hi, 0ull, 0ull);
                begin_search();
            } else {
                e0hi = b.hi;
                st = SM_EVENT1;
            }
        } else if (st == SM_EVENT1) {
            loc = disperse(c, B.P, loc, e0hi, b.lo, b.hi);
            begin_search();
        } else if (st == SM_SEARCH) {
            if (c.sampler == 0) {
                // sums of exponentials: draws 2j and 2j + 1 of interval k
                int r = 0;
                p = __dadd_rn(p, x0);
                uint64_t pb = (uint64_t)__double_as_longlong(p);
                r = pb >= end_b ? 2 : (pb > tau_b ? 1 : 0);
                if (r == 0) {
                    p = __dadd_rn(p, x1);
                    pb = (uint64_t)__double_as_longlong(p);
                    r = pb >= end_b ? 2 : (pb > tau_b ? 1 : 0);
                }
                if (r == 1) {
                    found(p);
                } else if (r == 2) {
                    ++k;
                    ++iv;
                    start_interval();
                } else if (++j >= INTERVAL_BLOCK_LIMIT) {
                    fail();
                }
            } else {
                // Poisson points: block j holds draws 2j, 2j + 1; draw 0 is the count
                auto consider = [&](uint64_t r) {
                    const double x = q53_scaled(r >> 11, c.dt_log2 - 53);
                    const uint64_t pb = (uint64_t)__double_as_longlong(__dadd_rn(base, x));
                    if (pb > tau_b && pb < best) best = pb;
                };
                if (j == 0) {
                    N = guided_count(c.pois_cdf, c.pois_guide, c.pois_n, b.lo);
                    if (N >= 1) consider(b.hi);
                } else {
                    if (2u * j - 1u < N) consider(b.lo);
                    if (2u * j < N) consider(b.hi);
                }
                if (2u * j + 1u >= N) {
                    if (best != ~0ull) {
                        found(__longlong_as_double((long long)best));
                    } else {
                        ++k;
                        ++iv;
                        start_interval();
                    }
                } else {
                    ++j;
                }
            }
        }
    }
    // flush the event counters, aggregated over lanes of the same simulation
    const bool valid = cnt_sim != 0xFFFFFFFFu;
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    if (valid) {
        warp_add_by_sim(vm, cnt_sim, ev_raw, &B.S[0].raw_events, sizeof(SimState));
        if (COUNT) warp_add_by_sim(vm, cnt_sim, ev_unique, &B.S[0].unique_events, sizeof(SimState));
    }
    const uint32_t wmax = __reduce_max_sync(0xFFFFFFFFu, lane_max);
    if (lane == 0 && wmax) atomicMax(&B.G->round_max, wmax);
}


// evaluates in parallel the draws a one-lane search would reach one after
// another.  Lane 0 writes the results.
// MODE 1: every simulation sums exponentials with lambda = 1 on the short
// search; MODE 2: every simulation draws Poisson points on the short search;
// MODE 0: any mix (the search chosen per lineage).  KIND: the landscape kind
// shared by every simulation, or -1.  The specialised kernels are smaller,
// which matters where one warp runs alone and waits on instruction fetch.
template <bool COUNT, int MODE, int KIND, bool LOG = false>
__global__ void __launch_bounds__(512) k_advance_coop(BatchDev B) {
    extern __shared__ __align__(16) unsigned char adv_smem[];
    const uint32_t n = B.G->n_total;
    if (n > B.coop_lineages) return;  // a round for the one-lane form
    if ((uint64_t)blockIdx.x * (blockDim.x >> 5) >= n) return;
    const LnC ln = B.need_ln ? ln_tables_shared(adv_smem) : ln_tables();
    const uint32_t t = B.G->round & 1u;
    const LinPtrs L = B.lin[t];
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t ev_raw = 0, ev_unique = 0;
    uint32_t cnt_sim = 0xFFFFFFFFu;
    uint32_t lane_max = 0;  // most events of one lineage this round (the same in every lane)
    WarpLogBuf wlog;
    wlog.n = 0;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(&B.G->work_ctr, 1u);
        idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
        if (idx >= n) break;
        const uint32_t gid = L.gid[idx];
        uint64_t loc = L.loc[idx];
        double tn = L.tn[idx];
        double tprev = LOG ? L.tp[idx] : 0.0;
        const uint32_t s = L.sim[idx];
        LaneSim c;
        load_lanesim(c, B.P, B.S, s);
        if (s != cnt_sim) {
            if (lane == 0 && cnt_sim != 0xFFFFFFFFu) {
                atomicAdd((unsigned long long*)&B.S[cnt_sim].raw_events, (unsigned long long)ev_raw);
                if (COUNT)
                    atomicAdd((unsigned long long*)&B.S[cnt_sim].unique_events, (unsigned long long)ev_unique);
            }
            ev_raw = ev_unique = 0;
            cnt_sim = s;
        }
        const uint64_t hz = (uint64_t)__double_as_longlong(c.horizon);
        uint32_t ev_lin = 0;
        for (uint32_t guard = 0; guard < 0xFFFFFFFFu; ++guard) {
            if ((uint64_t)__double_as_longlong(tn) > hz) {
                if (lane == 0) {
                    L.loc[idx] = loc;
                    L.tn[idx] = tn;
                    if (LOG) L.tp[idx] = tprev;
                    if (B.dedup) dedup_insert(B, t, slot_key(B.P, c, loc), gid);
                }
                break;
            }
            ++ev_raw;
            lane_max = max(lane_max, ++ev_lin);
            if (COUNT && lane == 0) ev_unique += count_event(B, t, slot_key(B.P, c, loc), tn) ? 1u : 0u;
            const uint64_t at = loc;
            const bool speciated = do_event_warp<KIND>(c, B.P, loc, tn, lane);
            if (LOG) {
                warp_log_event(B, wlog, lane, tn, tprev, at, speciated ? ~0ull : loc, gid);
                tprev = tn;
            }
            if (speciated) {
                if (lane == 0) {
                    B.key_loc[gid] = loc;
                    B.key_time[gid] = (uint64_t)__double_as_longlong(tn);
                    L.gid[idx] = gid | DONE_BIT;
                }
                break;
            }
            double nt;
            if (MODE == 1) {
                nt = coop_next_exp_short<true>(c, loc, tn, ln, lane);
            } else if (MODE == 2) {
                nt = coop_next_poisson_short(c, loc, tn, lane);
            } else {
                nt = c.sampler == 1 ? (c.coop_short ? coop_next_poisson_short(c, loc, tn, lane)
                                                    : coop_next_poisson(c, loc, tn, lane))
                     : c.coop_short ? (c.lam1 ? coop_next_exp_short<true>(c, loc, tn, ln, lane)
                                              : coop_next_exp_short<false>(c, loc, tn, ln, lane))
                                    : (c.lam1 ? coop_next_exp<true>(c, loc, tn, ln, lane)
                                              : coop_next_exp<false>(c, loc, tn, ln, lane));
            }
            if (search_failed(nt)) {
                if (lane == 0) {
                    atomicOr(&B.S[c.sim].error, 1u);
                    atomicOr(&B.G->error, 1u);
                    B.key_loc[gid] = ~0ull;
                    B.key_time[gid] = ~0ull;
                    L.gid[idx] = gid | DONE_BIT;
                }
                break;
            }
            tn = nt;
        }
    }
    if (lane == 0 && cnt_sim != 0xFFFFFFFFu) {
        atomicAdd((unsigned long long*)&B.S[cnt_sim].raw_events, (unsigned long long)ev_raw);
        if (COUNT) atomicAdd((unsigned long long*)&B.S[cnt_sim].unique_events, (unsigned long long)ev_unique);
    }
    if (lane == 0 && lane_max) atomicMax(&B.G->round_max, lane_max);
    if (LOG) warp_log_flush(B, wlog, lane);
}

// horizon step (time) of a simulation with n active lineages
__device__ __forceinline__ double horizon_step(const SimParams* p, uint32_t n) {
    const double dn = (double)n;
    const double floor_ev = dn < p->busy_lineages ? p->tail_events : p->min_events;
    const double per = fmax(floor_ev, fmin(p->occupancy_step * p->n_slots / dn, p->events_per_round / dn));
    return fmin(per, p->max_step_events) / p->lambda;
}

__global__ void k_compact(BatchDev B) {
    const uint32_t t = B.G->round & 1u;
    const LinPtrs in = B.lin[t];
    const LinPtrs out = B.lin[t ^ 1u];
    const uint32_t n = B.G->n_total;
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;

    for (uint32_t base = warp_global * 32u; base < n; base += n_warps * 32u) {
        const uint32_t i = base + lane;
        bool survive = false, culled = false;
        uint32_t s = 0xFFFFFFFFu, g = 0;
        uint64_t loc = 0;
        double tn = 0.0, tprev = 0.0;
        if (i < n) {
            g = in.gid[i];
            if (!(g & DONE_BIT)) {
                s = in.sim[i];
                loc = in.loc[i];
                tn = in.tn[i];
                if (in.tp) tprev = in.tp[i];
                survive = true;
                if (B.dedup) {
                    const uint32_t w = dedup_lookup(B, t, slot_index(B.P + s, loc));
                    if (w != g && w != 0xFFFFFFFFu) {
                        B.parent[g] = w;
                        survive = false;
                        culled = true;
                        if (in.tp) log_event(B, tn, tprev, loc, LOG_CULLED, g);
                    }
                }
            }
        }
        const unsigned sm = __ballot_sync(0xFFFFFFFFu, survive);
        const unsigned cm = __ballot_sync(0xFFFFFFFFu, culled);
        uint32_t pos0 = 0;
        if (lane == 0 && sm) pos0 = atomicAdd(&B.G->n_total_next, (uint32_t)__popc(sm));
        pos0 = __shfl_sync(0xFFFFFFFFu, pos0, 0);
        if (survive) {
            const uint32_t pos = pos0 + __popc(sm & lt_mask);
            out.loc[pos] = loc;
            out.tn[pos] = tn;
            out.gid[pos] = g;
            out.sim[pos] = s;
            if (out.tp) out.tp[pos] = tprev;
        }
        if (sm) {
            const unsigned grp = __match_any_sync(0xFFFFFFFFu, survive ? s : 0xFFFFFFFFu);
            if (survive && lane == (uint32_t)(__ffs(grp) - 1))
                atomicAdd(&B.S[s].n_next, (uint32_t)__popc(grp));
        }
        if (cm) {
            const unsigned grp = __match_any_sync(0xFFFFFFFFu, culled ? s : 0xFFFFFFFFu);
            if (culled && lane == (uint32_t)(__ffs(grp) - 1))
                atomicAdd(&B.S[s].culled_round, (uint32_t)__popc(grp));
        }
    }
    // clear the dedup / event tables of the previous round (no longer read)
    const uint32_t tp = t ^ 1u;
    const uint32_t nu = B.G->used[tp];
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nu; k += gridDim.x * blockDim.x) {
        const uint32_t h = B.ht_used[tp][k];
        B.ht_key[tp][h] = EMPTY_KEY;
        B.ht_val[tp][h] = 0xFFFFFFFFu;
    }
    if (B.count_unique) {
        const uint32_t ne = B.G->ev_used[tp];
        for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
            const uint32_t h = B.ev_used[tp][k];
            B.ev[tp][h].a = EMPTY_KEY;
            B.ev[tp][h].b = EMPTY_KEY;
        }
    }

    // the last block to finish advances the round
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&B.G->blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ uint32_t live;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < B.n_sims; s += blockDim.x) {
        SimState* st = B.S + s;
        const uint32_t na = atomicAdd(&st->n_next, 0u);
        const uint32_t nc = atomicAdd(&st->culled_round, 0u);
        st->culled += nc;
        st->culled_round = 0;
        st->n_next = 0;
        if (st->done) continue;
        st->n_active = na;
        st->rounds += 1;
        if (na == 0) {
            st->done = 1;
            continue;
        }
        atomicAdd(&live, 1u);
        st->horizon = st->horizon + horizon_step(B.P + s, na);
    }
    __syncthreads();
    if (B.G->prof_events) {
        __shared__ unsigned long long ev_sum;
        if (threadIdx.x == 0) ev_sum = 0;
        __syncthreads();
        unsigned long long part = 0;
        for (uint32_t s = threadIdx.x; s < B.n_sims; s += blockDim.x) part += B.S[s].raw_events;
        atomicAdd(&ev_sum, part);
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t slot = B.G->prof_slot;
            if (slot < B.G->prof_n) B.G->prof_events[slot] = ev_sum;
            B.G->prof_slot = slot + 1;
        }
    }
    if (threadIdx.x == 0) {
        Globals* G = B.G;
        const uint32_t nt = atomicAdd(&G->n_total_next, 0u);
        G->n_total = nt;
        G->n_total_next = 0;
        G->work_ctr = 0;
        G->blocks_done = 0;
        G->used[tp] = 0;
        G->ev_used[tp] = 0;
        G->n_live_sims = live;
        G->critical_events += G->round_max;
        G->round_max = 0;
        uint32_t cap = 2u;
        while (cap < 2u * nt && cap < B.ht_cap) cap <<= 1;
        G->mask[tp] = cap - 1u;  // the next round uses table tp
        G->round += 1;
        __threadfence();
    }
}

// initial horizons and counters of a fresh batch
__global__ void k_start(BatchDev B, uint32_t n_lin) {
    for (uint32_t s = threadIdx.x; s < B.n_sims; s += blockDim.x) {
        const SimParams* p = B.P + s;
        SimState* st = B.S + s;
        const uint32_t na = p->n_lineages;
        st->n_active = na;
        st->done = na == 0 ? 1u : 0u;
        st->horizon = horizon_step(p, max(na, 1u));
    }
    if (threadIdx.x == 0) {
        Globals* G = B.G;
        G->n_total = n_lin;
        uint32_t cap = 2u;
        while (cap < 2u * n_lin && cap < B.ht_cap) cap <<= 1;
        G->mask[0] = cap - 1u;
        G->mask[1] = cap - 1u;
    }
}

// root of every lineage (pointer chase over parent) and collection of roots
struct SortItem {
    unsigned long long a, b, c, d;  // sim, key location, key time bits, lineage id
};

__global__ void k_roots(BatchDev B, uint32_t n_lin, uint32_t* root, SortItem* items, uint32_t* n_items,
                        const uint32_t* __restrict__ gid_base) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_lin; g += gridDim.x * blockDim.x) {
        uint32_t r = g;
        for (uint32_t hops = 0; hops < n_lin; ++hops) {
            const uint32_t p = B.parent[r];
            if (p == r) break;
            r = p;
        }
        root[g] = r;
        if (r == g) {
            uint32_t lo = 0, hi = B.n_sims;
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (gid_base[mid] <= g) lo = mid;
                else hi = mid;
            }
            const uint32_t k = atomicAdd(n_items, 1u);
            items[k] = SortItem{lo, B.key_loc[g], B.key_time[g], g};
        }
    }
}

__device__ __forceinline__ bool item_less(const SortItem& x, const SortItem& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.c != y.c) return x.c < y.c;
    return x.d < y.d;  // a total order: equal keys come out the same on every run
}

__global__ void k_pad_items(SortItem* items, const uint32_t* n_items, uint32_t n_pad) {
    const uint32_t n = *n_items;
    for (uint32_t i = n + blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
        items[i] = SortItem{~0ull, ~0ull, ~0ull, ~0ull};
}

__global__ void k_bitonic_global(SortItem* x, uint32_t n, uint32_t j, uint32_t k) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t l = i ^ j;
    if (l <= i) return;
    const SortItem A = x[i], Bv = x[l];
    const bool up = (i & k) == 0;
    if (item_less(Bv, A) == up) {
        x[i] = Bv;
        x[l] = A;
    }
}

// all stages with j < 2 * blockDim.x for one k, in shared memory
__global__ void k_bitonic_shared(SortItem* x, uint32_t n, uint32_t k, uint32_t j_start) {
    extern __shared__ SortItem sh[];
    const uint32_t span = 2u * blockDim.x;
    const uint32_t base = blockIdx.x * span;
    for (uint32_t i = threadIdx.x; i < span; i += blockDim.x) sh[i] = x[base + i];
    __syncthreads();
    for (uint32_t j = j_start; j > 0; j >>= 1) {
        for (uint32_t ii = threadIdx.x; ii < span; ii += blockDim.x) {
            const uint32_t l = ii ^ j;
            if (l > ii) {
                const uint32_t gi = base + ii;
                const bool up = (gi & k) == 0;
                const SortItem A = sh[ii], Bv = sh[l];
                if (item_less(Bv, A) == up) {
                    sh[ii] = Bv;
                    sh[l] = A;
                }
            }
        }
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < span; i += blockDim.x) x[base + i] = sh[i];
}

// heads of distinct keys and of simulations
__global__ void k_heads(const SortItem* x, const uint32_t* n_items, uint32_t* head) {
    const uint32_t n = *n_items;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        bool h = i == 0 || x[i].a != x[i - 1].a || x[i].b != x[i - 1].b || x[i].c != x[i - 1].c;
        head[i] = h ? 1u : 0u;
    }
}

// distinct index (inclusive scan - 1) -> rank within the simulation
__global__ void k_sim_first(const SortItem* x, const uint32_t* n_items, const uint32_t* incl,
                            uint32_t* sim_first, uint64_t* sim_count) {
    const uint32_t n = *n_items;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i == 0 || x[i].a != x[i - 1].a) sim_first[x[i].a] = incl[i] - 1u;
        if (i == n - 1 || x[i].a != x[i + 1].a) sim_count[x[i].a] = incl[i];  // fixed up below
    }
}

__global__ void k_sim_count_fix(const uint32_t* sim_first, uint64_t* sim_count, uint32_t n_sims,
                                const uint32_t* n_items) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sims; s += gridDim.x * blockDim.x)
        if (sim_count[s] != 0) sim_count[s] -= sim_first[s];
}

__global__ void k_rank(const SortItem* x, const uint32_t* n_items, const uint32_t* incl,
                       const uint32_t* sim_first, uint32_t* rank_of_root) {
    const uint32_t n = *n_items;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        rank_of_root[x[i].d] = incl[i] - 1u - sim_first[x[i].a];
}

// per-individual outputs of one simulation
__global__ void k_outputs(const uint32_t* root, const uint32_t* rank_of_root, const uint64_t* key_loc,
                          const uint64_t* key_time, uint32_t gid_base, uint32_t n, uint64_t* species,
                          uint64_t* out_loc, uint64_t* out_time) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t r = root[gid_base + i];
        species[i] = rank_of_root[r];
        out_loc[i] = key_loc[r];
        out_time[i] = key_time[r];
    }
}

// ---------------------------------------------------------------------------
// exclusive scan of u32 (block scan, recursive over block sums)
// ---------------------------------------------------------------------------
constexpr uint32_t SCAN_BLOCK = 1024;
constexpr uint32_t SCAN_ITEMS = 4;
constexpr uint32_t SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[32];
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t ws = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, ws, o);
            if (lane >= (uint32_t)o) ws += y;
        }
        warp_sums[lane] = ws;
    }
    __syncthreads();
    const uint32_t before = w > 0 ? warp_sums[w - 1] : 0u;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// exclusive (inclusive if incl) scan of a tile; tile totals into sums
__global__ void k_scan_tiles(const uint32_t* in, uint32_t* out, uint32_t* sums, uint32_t n, int inclusive) {
    const uint32_t base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t local = 0;
#pragma unroll
    for (uint32_t k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        local += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(local, &total);
#pragma unroll
    for (uint32_t k = 0; k < SCAN_ITEMS; ++k) {
        if (inclusive) run += v[k];
        if (base + k < n) out[base + k] = run;
        if (!inclusive) run += v[k];
    }
    if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t* out, const uint32_t* sums_excl, uint32_t n) {
    const uint32_t base = blockIdx.x * SCAN_TILE;
    const uint32_t add = sums_excl[blockIdx.x];
    for (uint32_t k = threadIdx.x; k < SCAN_TILE; k += blockDim.x)
        if (base + k < n) out[base + k] += add;
}

// ---------------------------------------------------------------------------
// event stream: the log sorted by (time, location, prior time, lineage);
// copies of one event are adjacent, the first (earliest prior time) is the
// lineage that was at the location longest, and every later distinct prior
// time is a lineage that dispersed there at that time: a coalescence
// ---------------------------------------------------------------------------
__global__ void k_ev_items(EventLog L, uint32_t n, uint32_t n_pad, SortItem* items) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
        items[i] = i < n ? SortItem{L.time[i], L.loc[i], L.prior[i], ((unsigned long long)L.gid[i] << 32) | i}
                         : SortItem{~0ull, ~0ull, ~0ull, ~0ull};
}

__global__ void k_ev_marks(const SortItem* __restrict__ x, uint32_t n, uint32_t* head, uint32_t* coal) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool h = i == 0 || x[i].a != x[i - 1].a || x[i].b != x[i - 1].b;
        head[i] = h ? 1u : 0u;
        coal[i] = (!h && x[i].c != x[i - 1].c) ? 1u : 0u;
    }
}

__global__ void k_ev_events(const SortItem* __restrict__ x, uint32_t n, const uint32_t* head,
                            const uint32_t* incl_head, const uint64_t* __restrict__ target, uint32_t* head_pos,
                            ind_event* out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        const uint32_t g = incl_head[i] - 1u;
        head_pos[g] = i;
        const uint32_t idx = (uint32_t)x[i].d;
        out[g] = ind_event{x[i].a, x[i].c, x[i].b, target[idx], (uint32_t)(x[i].d >> 32), 0u};
    }
}

// an event's target from a copy that executed it (the first copy may be a
// culled lineage's; every executed copy has the same target)
__global__ void k_ev_targets(const SortItem* __restrict__ x, uint32_t n, const uint32_t* incl_head,
                             const uint64_t* __restrict__ target, ind_event* out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t tg = target[(uint32_t)x[i].d];
        if (tg != LOG_CULLED) out[incl_head[i] - 1u].target = tg;
    }
}

__global__ void k_ev_coalescences(const SortItem* __restrict__ x, uint32_t n, const uint32_t* coal,
                                  const uint32_t* incl_coal, const uint32_t* incl_head, const uint32_t* head_pos,
                                  ind_coalescence* out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!coal[i]) continue;
        const uint32_t parent = (uint32_t)(x[head_pos[incl_head[i] - 1u]].d >> 32);
        out[incl_coal[i] - 1u] = ind_coalescence{x[i].b, x[i].c, parent, (uint32_t)(x[i].d >> 32)};
    }
}

static ind_status scan_u32(Pool& pool, const uint32_t* in, uint32_t* out, uint32_t n, bool inclusive,
                           cudaStream_t s) {
    if (n == 0) return IND_OK;
    const uint32_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_scan_tiles<<<1, SCAN_BLOCK, 0, s>>>(in, out, nullptr, n, inclusive ? 1 : 0);
        CKL();
        return IND_OK;
    }
    uint32_t* sums = pool.get<uint32_t>(tiles);
    uint32_t* sums_ex = pool.get<uint32_t>(tiles);
    if (!sums || !sums_ex) return IND_ERR_OOM;
    k_scan_tiles<<<tiles, SCAN_BLOCK, 0, s>>>(in, out, sums, n, inclusive ? 1 : 0);
    CKL();
    ind_status st = scan_u32(pool, sums, sums_ex, tiles, false, s);
    if (st != IND_OK) return st;
    k_scan_add<<<tiles, SCAN_BLOCK, 0, s>>>(out, sums_ex, n);
    CKL();
    return IND_OK;
}

// ---------------------------------------------------------------------------
// inputs: habitat map, alias rows, sampling
// ---------------------------------------------------------------------------
__global__ void k_habitat(uint8_t* out, uint32_t W, uint32_t H, uint32_t sk0, uint32_t sk1, uint64_t thr,
                          uint32_t max_deme) {
    const uint64_t n = (uint64_t)W * H;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n; c += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(c % W), y = (uint32_t)(c / W);
        const u64x2 b = stream_block(sk0, sk1, pack_loc(x, y, 0), 0, 0, TAG_MAP);
        out[c] = (b.lo >> 11) < thr ? (uint8_t)(1u + umulhi64(b.hi, max_deme)) : (uint8_t)0;
    }
}

// one warp per habitable cell: weights, then integer Vose on lane 0
__global__ void k_alias_build(const uint8_t* __restrict__ deme, uint32_t W, uint32_t H,
                              const uint32_t* __restrict__ cells, uint32_t n_rows, const int8_t* __restrict__ off,
                              uint32_t n_off, const uint64_t* __restrict__ kw, uint64_t* __restrict__ alias) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const size_t per_warp = ((size_t)n_off * 12 + 15) & ~(size_t)15;  // 16-byte aligned regions
    uint64_t* s = (uint64_t*)(smem + per_warp * w);
    uint16_t* small_ = (uint16_t*)(s + n_off);
    uint16_t* large_ = small_ + n_off;
    for (uint32_t row = blockIdx.x * warps + w; row < n_rows; row += gridDim.x * warps) {
        const uint32_t cell = cells[row];
        const uint32_t cx = cell % W, cy = cell / W;
        unsigned long long part = 0;
        for (uint32_t o = lane; o < n_off; o += 32) {
            const int32_t dx = off[2 * o], dy = off[2 * o + 1];
            const uint32_t tx = wrap_add(cx, dx, W), ty = wrap_add(cy, dy, H);
            const uint64_t wgt = kw[dx * dx + dy * dy] * (uint64_t)deme[(size_t)ty * W + tx];
            s[o] = (uint64_t)n_off * wgt;
            part += wgt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        __syncwarp();
        if (lane == 0) {
            const uint64_t Wt = part;
            uint64_t* e = alias + (size_t)row * n_off;
            uint32_t ns = 0, nl = 0;
            for (uint32_t o = 0; o < n_off; ++o) {
                if (s[o] < Wt) small_[ns++] = (uint16_t)o;
                else large_[nl++] = (uint16_t)o;
            }
            while (ns > 0 && nl > 0) {
                const uint32_t a = small_[--ns];
                const uint32_t b = large_[--nl];
                // q = floor(s_a 2^32 / W) by restoring division (s_a < W < 2^56)
                uint64_t rem = s[a], q = 0;
                for (int bit = 0; bit < 32; ++bit) {
                    rem <<= 1;
                    q <<= 1;
                    if (rem >= Wt) {
                        rem -= Wt;
                        q |= 1ull;
                    }
                }
                e[a] = q | ((uint64_t)b << 32);
                s[b] = s[b] + s[a] - Wt;
                if (s[b] < Wt) small_[ns++] = (uint16_t)b;
                else large_[nl++] = (uint16_t)b;
            }
            while (nl > 0) {
                const uint32_t b = large_[--nl];
                e[b] = 0xFFFFFFFFull | ((uint64_t)b << 32) | (1ull << 63);
            }
            while (ns > 0) {
                const uint32_t a = small_[--ns];
                e[a] = 0xFFFFFFFFull | ((uint64_t)a << 32) | (1ull << 63);
            }
        }
        __syncwarp();
    }
}

__global__ void k_sample_flags(uint32_t* flags, uint64_t n_slots, int kind, uint32_t W, uint32_t D,
                               uint32_t slot_deme, const uint8_t* deme, int all, uint32_t sk0, uint32_t sk1,
                               uint64_t thr) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n_slots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t cell = s / slot_deme;
        const uint32_t i = (uint32_t)(s % slot_deme);
        const uint32_t d = kind == KIND_MAP ? deme[cell] : D;
        bool keep = i < d;
        if (keep && !all) {
            const uint64_t loc = pack_loc(cell % W, cell / W, i);
            keep = (stream_block(sk0, sk1, loc, 0, 0, TAG_SAMPLE).lo >> 11) < thr;
        }
        flags[s] = keep ? 1u : 0u;
    }
}

__global__ void k_sample_write(const uint32_t* flags, const uint32_t* pos, uint64_t n_slots, uint32_t W,
                               uint32_t slot_deme, uint64_t* out) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n_slots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        if (!flags[s]) continue;
        const uint64_t cell = s / slot_deme;
        out[pos[s]] = pack_loc(cell % W, cell / W, s % slot_deme);
    }
}

// device arithmetic probes for the conformance tests
__global__ void k_selftest(const uint64_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ exp_q58,
                           uint32_t* __restrict__ philox_out) {
    const LnC ln = ln_tables();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = in[i];
        if (exp_q58) exp_q58[i] = exp1_q58(v >> 11, ln.L, ln.R, ln.ln2, ln.c3);
        if (philox_out) {
            const uint64_t w = in[(i + 1) % n], z = in[(i + 2) % n];
            const u32x4 o = philox10((uint32_t)v, (uint32_t)(v >> 32), (uint32_t)w, (uint32_t)(w >> 32),
                                     (uint32_t)z, (uint32_t)(z >> 32));
            philox_out[4 * i + 0] = o.x;
            philox_out[4 * i + 1] = o.y;
            philox_out[4 * i + 2] = o.z;
            philox_out[4 * i + 3] = o.w;
        }
    }
}

// ---------------------------------------------------------------------------
// server kernels: append one admitted simulation, finish one id range
// ---------------------------------------------------------------------------
__global__ void k_append(BatchDev B, uint32_t pos, uint32_t n, uint32_t slot, uint32_t g0,
                         const uint64_t* __restrict__ sample_loc) {
    const LnC ln = ln_tables();
    LaneSim c;
    load_lanesim(c, B.P, B.S, slot);
    const LinPtrs L = B.lin[B.G->round & 1u];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t loc = sample_loc[i];
        double t = next_event_time<1>(c, loc, 0.0, ln);
        if (search_failed(t)) {
            atomicOr(&B.S[slot].error, 1u);
            atomicOr(&B.G->error, 1u);
            t = INFINITY;
        }
        L.loc[pos + i] = loc;
        L.tn[pos + i] = t;
        L.gid[pos + i] = g0 + i;
        L.sim[pos + i] = slot;
        B.parent[g0 + i] = g0 + i;
    }
}

// roots of the lineages of one id range [g0, g0 + n); root[] holds local ids
__global__ void k_roots_range(const uint32_t* __restrict__ parent, const uint64_t* __restrict__ key_loc,
                              const uint64_t* __restrict__ key_time, uint32_t g0, uint32_t n, uint32_t* root,
                              SortItem* items, uint32_t* n_items) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t r = g0 + i;
        for (uint32_t hops = 0; hops < n; ++hops) {
            const uint32_t p = parent[r];
            if (p == r) break;
            r = p;
        }
        root[i] = r - g0;
        if (r == g0 + i) {
            const uint32_t k = atomicAdd(n_items, 1u);
            items[k] = SortItem{0ull, key_loc[r], key_time[r], i};
        }
    }
}

__global__ void k_outputs_range(const uint32_t* root, const uint32_t* rank_of_root, const uint64_t* key_loc,
                                const uint64_t* key_time, uint32_t g0, uint32_t n, uint64_t* species,
                                uint64_t* out_loc, uint64_t* out_time) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t r = root[i];
        species[i] = rank_of_root[r];
        out_loc[i] = key_loc[g0 + r];
        out_time[i] = key_time[g0 + r];
    }
}

// ---------------------------------------------------------------------------
// host objects
// ---------------------------------------------------------------------------
struct Batch;

struct ind_sim {
    ind_landscape land{};
    ind_dispersal disp{};
    double nu = 0.0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    ind_tuning tuning{};
    uint32_t sk0 = 0, sk1 = 0;
    uint64_t nu_thr = 0;
    int dt_log2 = 0;
    uint32_t slot_deme = 1;
    uint64_t n_slots = 0;  // indexed locations (individuals of a full landscape)
    Pool tables;   // dispersal tables, map
    Pool sample;   // sampled locations
    Pool results;  // outputs
    uint64_t* d_gauss = nullptr;
    uint32_t* d_gauss_guide = nullptr;
    uint64_t* d_pois = nullptr;
    uint32_t* d_pois_guide = nullptr;
    uint32_t pois_n = 0;
    uint32_t gauss_n = 0;
    int gauss_half = 0;
    uint8_t* d_deme = nullptr;
    uint32_t* d_row_of = nullptr;
    uint64_t* d_alias = nullptr;
    int8_t* d_off = nullptr;
    uint32_t n_off = 0, n_rows = 0;
    uint64_t* d_sample = nullptr;
    uint64_t n_sampled = 0;
    bool sampled = false;
    bool finished = false;
    uint64_t* d_species = nullptr;
    uint64_t* d_key_loc = nullptr;
    uint64_t* d_key_time = nullptr;
    uint64_t n_species = 0;
    Batch* batch = nullptr;
    ind_run_stats stats{};
    uint64_t log_cap = 0;  // event log capacity of the next run (0: none)
    Pool events;           // the last logged run's event stream
    ind_event* d_events = nullptr;
    ind_coalescence* d_coal = nullptr;
    uint64_t n_events = 0, n_coal = 0;
    bool events_ready = false;
};

static void seed_key(uint64_t seed, uint32_t* k0, uint32_t* k1) {
    u32x4 o = philox10((uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0);
    *k0 = o.x;
    *k1 = o.y;
}

static uint32_t sm_count() {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return (uint32_t)n;
}

static uint32_t grid_for(uint64_t n, uint32_t threads, uint32_t max_blocks) {
    uint64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (uint32_t)b;
}

struct Batch {
    std::vector<ind_sim*> sims;
    uint32_t n_sims = 0;
    uint32_t n_lin = 0;
    cudaStream_t stream = nullptr;
    ind_tuning tun{};
    Pool pool;
    Pool scratch;
    SimParams* d_params = nullptr;
    SimState* d_state = nullptr;
    Globals* d_g = nullptr;
    uint32_t* d_gid_base = nullptr;
    BatchDev dev{};
    Globals* h_g = nullptr;  // pinned
    bool h_g_valid = false;
    std::vector<SimState> h_state;
    bool started = false;
    bool finished = false;
    uint64_t rounds = 0;
    cudaGraphExec_t graph = nullptr;  // captured chunk of rounds
    uint32_t graph_rounds = 0;
    int coop_mode = 0;                               // its specialisation (k_advance_coop MODE)
    int coop_kind = -1;                              // the landscape kind all simulations share, or -1
    cudaStream_t cap_stream = nullptr;  // private stream for graph capture (the legacy stream cannot capture)
    std::vector<cudaEvent_t> ev_start, ev_end;  // profile: one pair per round of a chunk
    double advance_ms = 0.0;
    uint64_t advance_launches = 0;
    unsigned long long* d_prof = nullptr;        // profile: cumulative events per round of a chunk
    std::vector<unsigned long long> h_prof;
    unsigned long long prof_last = 0;
    double best_launch_ms = 0.0;                 // the launch with the highest event rate
    uint64_t best_launch_events = 0;
    uint32_t adv_blocks = 0, adv_threads = 0, cmp_blocks = 0;
    double ms = 0.0;

    ~Batch() {
        if (graph) cudaGraphExecDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (auto e : ev_start) cudaEventDestroy(e);
        for (auto e : ev_end) cudaEventDestroy(e);
        if (h_g) cudaFreeHost(h_g);
        scratch.release_all();
        pool.release_all();
    }
};


// guide of a nondecreasing threshold table (see GUIDE_BITS): bucket u holds
// the draws [u 2^52, (u + 1) 2^52 - 1]
static std::vector<uint32_t> fine_guide(const std::vector<uint64_t>& cdf) {
    std::vector<uint32_t> g(GUIDE_N);
    constexpr int SHIFT = 64 - GUIDE_BITS;
    for (uint32_t u = 0; u < GUIDE_N; ++u) {
        const uint64_t first = (uint64_t)u << SHIFT;
        const uint64_t last = first + ((1ull << SHIFT) - 1ull);
        const uint32_t lo = (uint32_t)(std::upper_bound(cdf.begin(), cdf.end(), first) - cdf.begin());
        const uint32_t hi = (uint32_t)(std::upper_bound(cdf.begin(), cdf.end(), last) - cdf.begin());
        g[u] = lo | (hi != lo ? GUIDE_SCAN : 0u);
    }
    return g;
}

// slots a simulation takes in a batch's numbering of indexed locations
static uint64_t slot_span(const ind_sim* m) {
    if (m->land.kind == IND_IMPLICIT) return (uint64_t)m->land.deme + m->land.meta_size;
    return (uint64_t)m->land.width * m->land.height * m->slot_deme;
}

// the per-simulation device parameters shared by batches and the server
static void fill_params(const ind_sim* m, const ind_tuning& tun, SimParams& p) {
    memset(&p, 0, sizeof(p));
    p.kind = m->land.kind;
    p.W = m->land.width;
    p.H = m->land.height;
    p.D = m->land.kind == IND_MAP ? 0 : m->land.deme;
    p.slot_deme = m->slot_deme;
    p.dt_log2 = m->dt_log2;
    p.nu_thr = m->nu_thr;
    p.lambda = m->land.lambda;
    p.sk0 = m->sk0;
    p.sk1 = m->sk1;
    p.gauss_half = m->gauss_half;
    p.gauss_n = m->gauss_n;
    p.gauss = m->d_gauss;
    p.gauss_guide = m->d_gauss_guide;
    p.sampler = m->land.event_sampler;
    p.pois_n = m->pois_n;
    p.pois_cdf = m->d_pois;
    p.pois_guide = m->d_pois_guide;
    p.deme_map = m->d_deme;
    p.row_of = m->d_row_of;
    p.alias = m->d_alias;
    p.off = m->d_off;
    p.n_off = m->n_off;
    const double mu = m->land.lambda * m->land.delta_t;  // mean points per re-prime interval
    p.coop_short = mu <= 2.0 && (m->land.event_sampler != IND_SAMPLER_POISSON || mu >= 0.5) ? 1u : 0u;
    if (m->land.kind == IND_IMPLICIT) {
        p.meta_size = m->land.meta_size;
        p.m_thr = (uint64_t)std::ceil(m->land.migration * 0x1p53);
        p.meta_nu_thr = (uint64_t)std::ceil(m->land.meta_nu * 0x1p53);
    }
    p.sample_loc = m->d_sample;
    p.events_per_round = tun.events_per_round;
    p.min_events = tun.min_events_per_lineage;
    p.occupancy_step = tun.occupancy_step;
    p.tail_events = tun.tail_events;
    p.busy_lineages = tun.busy_lineages;
    p.max_step_events = tun.max_step_events;
    p.n_slots = (double)m->n_slots;
}

template <bool COUNT, int MODE, int KIND>
static cudaError_t set_smem_one() {
    return cudaFuncSetAttribute(k_advance_coop<COUNT, MODE, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)LN_SMEM_BYTES);
}

// the instantiations launch_coop uses: with counting (measurement runs) only
// the generic kind
template <bool COUNT>
static cudaError_t set_coop_smem() {
    cudaError_t e;
    if ((e = set_smem_one<COUNT, 0, -1>()) || (e = set_smem_one<COUNT, 1, -1>()) ||
        (e = set_smem_one<COUNT, 2, -1>()))
        return e;
    if (!COUNT) {
        if ((e = set_smem_one<COUNT, 1, 0>()) || (e = set_smem_one<COUNT, 1, 1>()) ||
            (e = set_smem_one<COUNT, 1, 2>()) || (e = set_smem_one<COUNT, 2, 0>()) ||
            (e = set_smem_one<COUNT, 2, 1>()) || (e = set_smem_one<COUNT, 2, 2>()))
            return e;
    }
    return cudaSuccess;
}

template <bool COUNT, int MODE>
static void launch_coop_kind(const Batch& b, size_t smem, cudaStream_t s) {
    const dim3 g(b.adv_blocks), t(b.adv_threads);
    if (COUNT || b.coop_kind < 0 || b.coop_kind > KIND_MAP)  // counting runs and mixed or implicit batches
        k_advance_coop<COUNT, MODE, -1><<<g, t, smem, s>>>(b.dev);
    else if (b.coop_kind == KIND_NONSPATIAL) k_advance_coop<COUNT, MODE, (COUNT ? -1 : 0)><<<g, t, smem, s>>>(b.dev);
    else if (b.coop_kind == KIND_TORUS) k_advance_coop<COUNT, MODE, (COUNT ? -1 : 1)><<<g, t, smem, s>>>(b.dev);
    else k_advance_coop<COUNT, MODE, (COUNT ? -1 : 2)><<<g, t, smem, s>>>(b.dev);
}

template <bool COUNT>
static void launch_coop(const Batch& b, size_t smem, cudaStream_t s) {
    if (b.coop_mode == 1) launch_coop_kind<COUNT, 1>(b, smem, s);
    else if (b.coop_mode == 2) launch_coop_kind<COUNT, 2>(b, smem, s);
    else k_advance_coop<COUNT, 0, -1><<<b.adv_blocks, b.adv_threads, smem, s>>>(b.dev);
}

static ind_status batch_build(Batch& b) {
    b.pool.stream = b.scratch.stream = b.stream;
    b.n_sims = (uint32_t)b.sims.size();
    std::vector<SimParams> hp(b.n_sims);
    std::vector<uint32_t> gid_base(b.n_sims);
    uint64_t lin = 0, slots = 0;
    for (uint32_t s = 0; s < b.n_sims; ++s) {
        ind_sim* m = b.sims[s];
        SimParams& p = hp[s];
        fill_params(m, b.tun, p);
        p.n_lineages = (uint32_t)m->n_sampled;
        p.slot_base = slots;
        p.gid_base = (uint32_t)lin;
        gid_base[s] = (uint32_t)lin;
        lin += m->n_sampled;
        slots += slot_span(m);
    }
    if (lin >= (1ull << 31)) return IND_ERR_ARG;
    b.n_lin = (uint32_t)lin;
    const uint32_t n = std::max<uint32_t>(b.n_lin, 1u);
    Pool& P = b.pool;
    b.d_params = P.get<SimParams>(b.n_sims);
    b.d_state = P.get<SimState>(b.n_sims);
    b.d_g = P.get<Globals>(1);
    b.d_gid_base = P.get<uint32_t>(b.n_sims);
    BatchDev& d = b.dev;
    for (int t = 0; t < 2; ++t) {
        d.lin[t].loc = P.get<uint64_t>(n);
        d.lin[t].tn = P.get<double>(n);
        d.lin[t].gid = P.get<uint32_t>(n);
        d.lin[t].sim = P.get<uint32_t>(n);
    }
    d.parent = P.get<uint32_t>(n);
    d.key_loc = P.get<uint64_t>(n);
    d.key_time = P.get<uint64_t>(n);
    uint32_t cap = 2;
    while (cap < 2u * n) cap <<= 1;
    d.ht_cap = cap;
    for (int t = 0; t < 2; ++t) {
        d.ht_key[t] = P.get<unsigned long long>(cap);
        d.ht_val[t] = P.get<uint32_t>(cap);
        d.ht_used[t] = P.get<uint32_t>(n);
    }
    d.count_unique = b.tun.count_unique ? 1 : 0;
    if (d.count_unique) {
        // events of one round, from the horizon-step rule: n * step <=
        // max(floor n, min(alpha S, events_per_round)) per simulation
        double est = 0;
        const double fl = std::max(b.tun.tail_events, b.tun.min_events_per_lineage);
        for (uint32_t s = 0; s < b.n_sims; ++s)
            est += 1.3 * (fl * (double)hp[s].n_lineages +
                          std::min(b.tun.occupancy_step * hp[s].n_slots, b.tun.events_per_round)) + 64.0;
        uint64_t ec = 2;
        while ((double)ec < 2.0 * est && ec < (1ull << 30)) ec <<= 1;
        d.ev_mask = (uint32_t)(ec - 1);
        for (int t = 0; t < 2; ++t) {
            d.ev[t] = P.get<EvSlot>(ec);
            d.ev_used[t] = P.get<uint32_t>(ec);
        }
    }
    // event log: one simulation per batch (sim_run)
    uint64_t log_cap = 0;
    for (auto* m : b.sims) log_cap = std::max(log_cap, m->log_cap);
    if (log_cap) {
        if (b.n_sims != 1) return IND_ERR_ARG;
        for (int t = 0; t < 2; ++t)
            if (!(d.lin[t].tp = P.get<double>(n))) return IND_ERR_OOM;
        d.log.time = P.get<uint64_t>(log_cap);
        d.log.prior = P.get<uint64_t>(log_cap);
        d.log.loc = P.get<uint64_t>(log_cap);
        d.log.target = P.get<uint64_t>(log_cap);
        d.log.gid = P.get<uint32_t>(log_cap);
        if (!d.log.time || !d.log.prior || !d.log.loc || !d.log.target || !d.log.gid) return IND_ERR_OOM;
        d.log.cap = log_cap;
    }
    for (int t = 0; t < 2; ++t)
        if (!d.lin[t].loc || !d.lin[t].tn || !d.lin[t].gid || !d.lin[t].sim || !d.ht_key[t] || !d.ht_val[t] ||
            !d.ht_used[t] || (d.count_unique && (!d.ev[t] || !d.ev_used[t])))
            return IND_ERR_OOM;
    if (!b.d_params || !b.d_state || !b.d_g || !b.d_gid_base || !d.parent || !d.key_loc || !d.key_time)
        return IND_ERR_OOM;
    d.P = b.d_params;
    d.S = b.d_state;
    d.G = b.d_g;
    d.n_sims = b.n_sims;
    d.lpl = b.tun.lineages_per_lane;
    d.events_per_visit = b.tun.events_per_visit;
    d.coop_lineages = b.tun.coop_lineages;
    d.dedup = b.tun.dedup ? 1 : 0;
    d.need_ln = 0;
    for (uint32_t si = 0; si < b.n_sims; ++si) d.need_ln |= hp[si].sampler == IND_SAMPLER_EXP ? 1 : 0;
    bool all_exp1 = b.n_sims > 0, all_pois = b.n_sims > 0;
    for (uint32_t si = 0; si < b.n_sims; ++si) {
        all_exp1 &= hp[si].sampler == IND_SAMPLER_EXP && hp[si].coop_short && hp[si].lambda == 1.0;
        all_pois &= hp[si].sampler == IND_SAMPLER_POISSON && hp[si].coop_short;
    }
    b.coop_mode = all_exp1 ? 1 : all_pois ? 2 : 0;
    b.coop_kind = b.n_sims > 0 ? hp[0].kind : -1;
    for (uint32_t si = 1; si < b.n_sims; ++si)
        if (hp[si].kind != b.coop_kind) b.coop_kind = -1;
    cudaStream_t s = b.stream;
    CK(cudaMemcpyAsync(b.d_params, hp.data(), sizeof(SimParams) * b.n_sims, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b.d_gid_base, gid_base.data(), sizeof(uint32_t) * b.n_sims, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(b.d_state, 0, sizeof(SimState) * b.n_sims, s));
    CK(cudaMemsetAsync(b.d_g, 0, sizeof(Globals), s));
    for (int t = 0; t < 2; ++t) {
        CK(cudaMemsetAsync(d.ht_key[t], 0xFF, sizeof(unsigned long long) * cap, s));
        CK(cudaMemsetAsync(d.ht_val[t], 0xFF, sizeof(uint32_t) * cap, s));
        if (d.count_unique) CK(cudaMemsetAsync(d.ev[t], 0xFF, sizeof(EvSlot) * ((size_t)d.ev_mask + 1), s));
    }
    CK(cudaMallocHost(&b.h_g, sizeof(Globals)));
    b.h_state.resize(b.n_sims);
    if (b.tun.profile) {
        b.ev_start.resize(b.tun.rounds_per_check);
        b.ev_end.resize(b.tun.rounds_per_check);
        for (uint32_t r = 0; r < b.tun.rounds_per_check; ++r) {
            CK(cudaEventCreate(&b.ev_start[r]));
            CK(cudaEventCreate(&b.ev_end[r]));
        }
        b.d_prof = P.get<unsigned long long>(b.tun.rounds_per_check);
        if (!b.d_prof) return IND_ERR_OOM;
        Globals hg;
        memset(&hg, 0, sizeof(hg));
        hg.prof_events = b.d_prof;
        hg.prof_n = b.tun.rounds_per_check;
        CK(cudaMemcpyAsync(&b.d_g->prof_events, &hg.prof_events, sizeof(hg.prof_events), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(&b.d_g->prof_n, &hg.prof_n, sizeof(hg.prof_n), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    const uint32_t sms = sm_count();
    CK(cudaFuncSetAttribute(k_advance<true, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES));
    CK(cudaFuncSetAttribute(k_advance<false, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES));
    if (b.dev.log.cap) {
        CK(cudaFuncSetAttribute(k_advance<true, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)LN_SMEM_BYTES));
        CK(cudaFuncSetAttribute(k_advance<false, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)LN_SMEM_BYTES));
        CK(cudaFuncSetAttribute(k_advance_coop<true, 0, -1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)LN_SMEM_BYTES));
        CK(cudaFuncSetAttribute(k_advance_coop<false, 0, -1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)LN_SMEM_BYTES));
    }
    CK(set_coop_smem<true>());
    CK(set_coop_smem<false>());
    CK(cudaFuncSetAttribute(k_advance_sm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES));
    CK(cudaFuncSetAttribute(k_advance_sm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES));
    b.adv_threads = b.tun.block_threads;
    b.adv_blocks = sms * b.tun.blocks_per_sm;
    b.cmp_blocks = sms * 4;
    // starting states
    k_start<<<1, 256, 0, s>>>(d, b.n_lin);
    CKL();
    if (b.n_lin) {
        k_init<<<grid_for(b.n_lin, 256, sms * 16), 256, 0, s>>>(d, b.d_gid_base, b.n_lin);
        CKL();
    }
    b.started = true;
    return IND_OK;
}

constexpr uint64_t LAUNCHES_PER_ROUND = 3;  // one-lane advance, warp-per-lineage advance, compaction

static ind_status launch_round(Batch& b, uint32_t r, bool capturing) {
    cudaStream_t s = capturing ? b.cap_stream : b.stream;
    const bool prof = b.tun.profile && r < b.ev_start.size();
    const unsigned flag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (prof) CK(cudaEventRecordWithFlags(b.ev_start[r], s, flag));
    // shared memory only when some simulation sums exponentials (leaves L1 larger otherwise)
    const size_t smem = b.dev.need_ln ? LN_SMEM_BYTES : 0;
    const bool conv = b.tun.advance_variant == 0;  // convergent state machine or one-lane loop
    // both advance forms every round: each reads the live lineage count and
    // returns at once unless the round is its own (more than coop_lineages
    // lineages: one lane per lineage; else one warp per lineage), so that the
    // choice is made per round inside captured chunks.  An event log takes
    // the logging forms (one-lane loop, generic warp form).
    const dim3 ag(b.adv_blocks), at(b.adv_threads);
    if (b.dev.log.cap) {
        if (b.dev.count_unique) {
            k_advance<true, 1, true><<<ag, at, smem, s>>>(b.dev);
            CK(cudaGetLastError());
            k_advance_coop<true, 0, -1, true><<<ag, at, smem, s>>>(b.dev);
        } else {
            k_advance<false, 1, true><<<ag, at, smem, s>>>(b.dev);
            CK(cudaGetLastError());
            k_advance_coop<false, 0, -1, true><<<ag, at, smem, s>>>(b.dev);
        }
    } else if (b.dev.count_unique) {
        if (conv) k_advance_sm<true><<<b.adv_blocks, b.adv_threads, smem, s>>>(b.dev);
        else k_advance<true, 1, false><<<b.adv_blocks, b.adv_threads, smem, s>>>(b.dev);
        CK(cudaGetLastError());
        launch_coop<true>(b, smem, s);
    } else {
        if (conv) k_advance_sm<false><<<b.adv_blocks, b.adv_threads, smem, s>>>(b.dev);
        else k_advance<false, 1, false><<<b.adv_blocks, b.adv_threads, smem, s>>>(b.dev);
        CK(cudaGetLastError());
        launch_coop<false>(b, smem, s);
    }
    CK(cudaGetLastError());
    if (prof) CK(cudaEventRecordWithFlags(b.ev_end[r], s, flag));
    k_compact<<<b.cmp_blocks, 256, 0, s>>>(b.dev);
    CK(cudaGetLastError());
    if (!capturing) g_launches.fetch_add(LAUNCHES_PER_ROUND);  // a captured chunk counts when it runs
    return IND_OK;
}

static ind_status batch_rounds(Batch& b, uint32_t rounds) {
    if (b.tun.use_graph) {
        if (!b.graph || b.graph_rounds != rounds) {
            if (b.graph) {
                cudaGraphExecDestroy(b.graph);
                b.graph = nullptr;
            }
            cudaGraph_t g;
            if (!b.cap_stream) CK(cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking));
            CK(cudaStreamBeginCapture(b.cap_stream, cudaStreamCaptureModeThreadLocal));
            for (uint32_t r = 0; r < rounds; ++r) {
                ind_status st = launch_round(b, r, true);
                if (st != IND_OK) {
                    cudaStreamEndCapture(b.cap_stream, &g);
                    return st;
                }
            }
            CK(cudaStreamEndCapture(b.cap_stream, &g));
            CK(cudaGraphInstantiate(&b.graph, g, 0));
            cudaGraphDestroy(g);
            b.graph_rounds = rounds;
        }
        CK(cudaGraphLaunch(b.graph, b.stream));
        g_launches.fetch_add(LAUNCHES_PER_ROUND * rounds);
        return IND_OK;
    }
    for (uint32_t r = 0; r < rounds; ++r) {
        ind_status st = launch_round(b, r, false);
        if (st != IND_OK) return st;
    }
    return IND_OK;
}

// after a synchronised chunk: add up the timed advance launches
static void collect_profile(Batch& b, uint32_t rounds) {
    if (!b.tun.profile) return;
    if (b.d_prof) {
        b.h_prof.resize(rounds);
        if (cudaMemcpy(b.h_prof.data(), b.d_prof, sizeof(unsigned long long) * rounds, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            cudaGetLastError();
        unsigned int zero = 0;
        cudaMemcpy(&b.d_g->prof_slot, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    }
    for (uint32_t r = 0; r < rounds && r < b.ev_start.size(); ++r) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b.ev_start[r], b.ev_end[r]) == cudaSuccess) {
            b.advance_ms += ms;
            b.advance_launches += 1;
            if (b.d_prof && r < b.h_prof.size()) {
                const unsigned long long ev = b.h_prof[r] - b.prof_last;
                b.prof_last = b.h_prof[r];
                if (ms > 0.f && (b.best_launch_events == 0 ||
                                 (double)ev / ms > (double)b.best_launch_events / b.best_launch_ms)) {
                    b.best_launch_events = ev;
                    b.best_launch_ms = ms;
                }
            }
        } else {
            cudaGetLastError();
        }
    }
}

// resolve roots, sort/unique species keys, write per-sim outputs
// ascending bitonic sort of np items (a power of two, at least 2048):
// global stages for strides of 2048 and more, shared memory for the rest
static ind_status bitonic_sort(SortItem* items, uint32_t np, cudaStream_t s) {
    const uint32_t sh_threads = 1024;
    const uint32_t span = 2 * sh_threads;
    const size_t sh_bytes = sizeof(SortItem) * span;
    static bool attr_set = false;
    if (!attr_set) {
        CK(cudaFuncSetAttribute(k_bitonic_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_bytes));
        attr_set = true;
    }
    for (uint32_t k = 2; k <= np; k <<= 1) {
        uint32_t j = k >> 1;
        for (; j >= span; j >>= 1) {
            k_bitonic_global<<<(np + 255) / 256, 256, 0, s>>>(items, np, j, k);
            CKL();
        }
        k_bitonic_shared<<<np / span, sh_threads, sh_bytes, s>>>(items, np, k, j);
        CKL();
    }
    return IND_OK;
}

static ind_status process_event_log(Batch& b);

static ind_status batch_finish(Batch& b) {
    cudaStream_t s = b.stream;
    Pool& T = b.scratch;
    const uint32_t n = std::max<uint32_t>(b.n_lin, 1u);
    const uint32_t sms = sm_count();
    uint32_t* root = T.get<uint32_t>(n);
    uint32_t* n_items = T.get<uint32_t>(1);
    uint32_t n_pad = 1;
    while (n_pad < n) n_pad <<= 1;
    if (n_pad < 2048) n_pad = 2048;
    SortItem* items = T.get<SortItem>(n_pad);
    uint32_t* head = T.get<uint32_t>(n);
    uint32_t* incl = T.get<uint32_t>(n);
    uint32_t* sim_first = T.get<uint32_t>(b.n_sims);
    uint64_t* sim_count = T.get<uint64_t>(b.n_sims);
    uint32_t* rank = T.get<uint32_t>(n);
    if (!root || !n_items || !items || !head || !incl || !sim_first || !sim_count || !rank) return IND_ERR_OOM;
    CK(cudaMemsetAsync(n_items, 0, sizeof(uint32_t), s));
    CK(cudaMemsetAsync(sim_count, 0, sizeof(uint64_t) * b.n_sims, s));
    CK(cudaMemsetAsync(sim_first, 0, sizeof(uint32_t) * b.n_sims, s));
    const uint32_t gb = grid_for(n, 256, sms * 16);
    k_roots<<<gb, 256, 0, s>>>(b.dev, b.n_lin, root, items, n_items, b.d_gid_base);
    CKL();
    uint32_t h_items = 0;
    CK(cudaMemcpyAsync(&h_items, n_items, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    uint32_t np = 2048;
    while (np < h_items) np <<= 1;
    k_pad_items<<<grid_for(np, 256, sms * 16), 256, 0, s>>>(items, n_items, np);
    CKL();
    {
        const ind_status sst = bitonic_sort(items, np, s);
        if (sst != IND_OK) return sst;
    }
    k_heads<<<grid_for(h_items, 256, sms * 16), 256, 0, s>>>(items, n_items, head);
    CKL();
    ind_status st = scan_u32(T, head, incl, h_items, true, s);
    if (st != IND_OK) return st;
    if (h_items) {
        k_sim_first<<<grid_for(h_items, 256, sms * 16), 256, 0, s>>>(items, n_items, incl, sim_first, sim_count);
        CKL();
        k_sim_count_fix<<<grid_for(b.n_sims, 256, sms), 256, 0, s>>>(sim_first, sim_count, b.n_sims, n_items);
        CKL();
        k_rank<<<grid_for(h_items, 256, sms * 16), 256, 0, s>>>(items, n_items, incl, sim_first, rank);
        CKL();
    }
    std::vector<uint64_t> counts(b.n_sims);
    for (uint32_t si = 0; si < b.n_sims; ++si) {
        ind_sim* m = b.sims[si];
        if (m->n_sampled == 0) continue;
        if (!m->d_species) {
            m->results.stream = m->stream;
            m->d_species = m->results.get<uint64_t>(m->n_sampled);
            m->d_key_loc = m->results.get<uint64_t>(m->n_sampled);
            m->d_key_time = m->results.get<uint64_t>(m->n_sampled);
            if (!m->d_species || !m->d_key_loc || !m->d_key_time) return IND_ERR_OOM;
        }
        uint32_t base = 0;
        for (uint32_t k = 0; k < si; ++k) base += (uint32_t)b.sims[k]->n_sampled;
        k_outputs<<<grid_for(m->n_sampled, 256, sms * 16), 256, 0, s>>>(
            root, rank, b.dev.key_loc, b.dev.key_time, base, (uint32_t)m->n_sampled, m->d_species, m->d_key_loc,
            m->d_key_time);
        CKL();
    }
    CK(cudaMemcpyAsync(counts.data(), sim_count, sizeof(uint64_t) * b.n_sims, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(b.h_state.data(), b.d_state, sizeof(SimState) * b.n_sims, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (uint32_t si = 0; si < b.n_sims; ++si) {
        ind_sim* m = b.sims[si];
        m->n_species = counts[si];
        m->finished = true;
        m->stats.n_species = counts[si];
    }
    if (b.dev.log.cap) {
        const ind_status lst = process_event_log(b);
        if (lst != IND_OK) return lst;
    }
    b.scratch.release_all();
    return IND_OK;
}

// the logged run's record -> the distinct events and the coalescences
static ind_status process_event_log(Batch& b) {
    ind_sim* m = b.sims[0];
    cudaStream_t s = b.stream;
    Pool& T = b.scratch;
    const uint32_t sms = sm_count();
    m->events.release_all();
    m->events.stream = m->stream;
    m->d_events = nullptr;
    m->d_coal = nullptr;
    m->n_events = m->n_coal = 0;
    m->events_ready = false;
    unsigned long long n_log = 0;
    CK(cudaMemcpyAsync(&n_log, &b.d_g->log_n, sizeof(n_log), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (n_log > b.dev.log.cap) return IND_ERR_DEVICE;
    const uint32_t n = (uint32_t)n_log;
    if (n) {
        uint32_t np = 2048;
        while (np < n) np <<= 1;
        SortItem* items = T.get<SortItem>(np);
        uint32_t* head = T.get<uint32_t>(n);
        uint32_t* coal = T.get<uint32_t>(n);
        uint32_t* incl_head = T.get<uint32_t>(n);
        uint32_t* incl_coal = T.get<uint32_t>(n);
        if (!items || !head || !coal || !incl_head || !incl_coal) return IND_ERR_OOM;
        k_ev_items<<<grid_for(np, 256, sms * 16), 256, 0, s>>>(b.dev.log, n, np, items);
        CKL();
        ind_status st = bitonic_sort(items, np, s);
        if (st != IND_OK) return st;
        k_ev_marks<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, head, coal);
        CKL();
        if ((st = scan_u32(T, head, incl_head, n, true, s)) != IND_OK) return st;
        if ((st = scan_u32(T, coal, incl_coal, n, true, s)) != IND_OK) return st;
        uint32_t hn = 0, cn = 0;
        CK(cudaMemcpyAsync(&hn, incl_head + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&cn, incl_coal + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        m->d_events = m->events.get<ind_event>(std::max<uint32_t>(hn, 1u));
        m->d_coal = m->events.get<ind_coalescence>(std::max<uint32_t>(cn, 1u));
        uint32_t* head_pos = T.get<uint32_t>(std::max<uint32_t>(hn, 1u));
        if (!m->d_events || !m->d_coal || !head_pos) return IND_ERR_OOM;
        k_ev_events<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, head, incl_head, b.dev.log.target, head_pos,
                                                               m->d_events);
        CKL();
        k_ev_targets<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, incl_head, b.dev.log.target, m->d_events);
        CKL();
        k_ev_coalescences<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, coal, incl_coal, incl_head, head_pos,
                                                                     m->d_coal);
        CKL();
        CK(cudaStreamSynchronize(s));
        m->n_events = hn;
        m->n_coal = cn;
    }
    m->events_ready = true;
    return IND_OK;
}

static void collect_stats(Batch& b, uint64_t n_roots_unknown) {
    (void)n_roots_unknown;
    for (uint32_t si = 0; si < b.n_sims; ++si) {
        ind_sim* m = b.sims[si];
        const SimState& st = b.h_state[si];
        m->stats.rounds = st.rounds;
        m->stats.raw_events = st.raw_events;
        m->stats.unique_events = st.unique_events;
        m->stats.culled = st.culled;
        m->stats.n_sampled = m->n_sampled;
        m->stats.n_roots = m->n_sampled - st.culled;
    }
}

// run rounds until finished or budget; IND_ERR_BUDGET if not finished
static ind_status batch_run(Batch& b, uint64_t round_budget) {
    auto t0 = std::chrono::steady_clock::now();
    ind_status result = IND_OK;
    uint64_t done_rounds = 0;
    for (;;) {
        uint32_t chunk = b.tun.rounds_per_check;
        if (round_budget) {
            if (done_rounds >= round_budget) {
                result = IND_ERR_BUDGET;
                break;
            }
            chunk = (uint32_t)std::min<uint64_t>(chunk, round_budget - done_rounds);
        }
        ind_status st = batch_rounds(b, chunk);
        if (st != IND_OK) return st;
        done_rounds += chunk;
        b.rounds += chunk;
        CK(cudaMemcpyAsync(b.h_g, b.d_g, sizeof(Globals), cudaMemcpyDeviceToHost, b.stream));
        CK(cudaStreamSynchronize(b.stream));
        b.h_g_valid = true;
        collect_profile(b, chunk);
        if (b.h_g->error) {
            CK(cudaMemcpyAsync(b.h_state.data(), b.d_state, sizeof(SimState) * b.n_sims, cudaMemcpyDeviceToHost,
                               b.stream));
            CK(cudaStreamSynchronize(b.stream));
            collect_stats(b, 0);
            return IND_ERR_DEVICE;
        }
        if (b.h_g->n_total == 0) break;
    }
    if (result == IND_OK) {
        ind_status st = batch_finish(b);
        if (st != IND_OK) return st;
        b.finished = true;
    } else {
        CK(cudaMemcpyAsync(b.h_state.data(), b.d_state, sizeof(SimState) * b.n_sims, cudaMemcpyDeviceToHost,
                           b.stream));
        CK(cudaStreamSynchronize(b.stream));
    }
    collect_stats(b, 0);
    auto t1 = std::chrono::steady_clock::now();
    b.ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
    for (auto* m : b.sims) {
        m->stats.ms_total = b.ms;
        m->stats.advance_ms = b.advance_ms;
        m->stats.advance_launches = b.advance_launches;
        m->stats.busiest_launch_ms = b.best_launch_ms;
        m->stats.busiest_launch_events = b.best_launch_events;
        m->stats.critical_events = b.h_g_valid ? b.h_g->critical_events : 0;
    }
    return result;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* ind_status_string(ind_status s) {
    switch (s) {
        case IND_OK: return "IND_OK";
        case IND_ERR_ARG: return "IND_ERR_ARG";
        case IND_ERR_OOM: return "IND_ERR_OOM";
        case IND_ERR_CUDA: return "IND_ERR_CUDA";
        case IND_ERR_BUDGET: return "IND_ERR_BUDGET";
        case IND_ERR_STATE: return "IND_ERR_STATE";
        case IND_ERR_DEVICE: return "IND_ERR_DEVICE";
    }
    return "IND_UNKNOWN";
}

int ind_last_cuda_error(void) { return g_last_cuda_error.load(); }

uint64_t ind_kernel_launches(void) { return g_launches.load(); }

ind_status ind_set_allocator(const ind_allocator* a) {
    if (a && (!a->alloc || !a->release)) return IND_ERR_ARG;
    if (a) g_alloc = *a;
    else g_alloc = ind_allocator{nullptr, nullptr, nullptr};
    return IND_OK;
}

void ind_default_tuning(ind_tuning* t) {
    if (!t) return;
    memset(t, 0, sizeof(*t));
    t->block_threads = 256;
    t->blocks_per_sm = 8;
    t->lineages_per_lane = 1;
    t->events_per_visit = 8;
    t->coop_lineages = 4096;
    t->advance_variant = 1;
    t->rounds_per_check = 16;
    t->use_graph = 1;
    t->dedup = 1;
    t->count_unique = 0;
    t->profile = 0;
    t->events_per_round = 4194304.0;
    t->min_events_per_lineage = 0.25;
    t->occupancy_step = 0.25;
    t->tail_events = 128.0;
    t->busy_lineages = 32768.0;
    t->max_step_events = 16384.0;
}

static bool tuning_ok(const ind_tuning* t) {
    return t->block_threads >= 64 && t->block_threads <= 512 && t->block_threads % 32 == 0 &&
           t->blocks_per_sm >= 1 && t->blocks_per_sm <= 32 && t->lineages_per_lane >= 1 &&
           t->events_per_visit >= 1 && t->events_per_visit <= 1024 && t->advance_variant <= 1 &&
           t->lineages_per_lane <= 64 && t->rounds_per_check >= 1 && t->rounds_per_check <= 4096 &&
           t->events_per_round >= 1.0 && t->min_events_per_lineage > 0.0 && t->occupancy_step > 0.0 &&
           t->tail_events > 0.0 && t->busy_lineages >= 0.0 && std::isfinite(t->tail_events) &&
           t->max_step_events > 0.0 &&
           std::isfinite(t->busy_lineages) &&
           std::isfinite(t->events_per_round) && std::isfinite(t->min_events_per_lineage) &&
           std::isfinite(t->occupancy_step);
}

static int pow2_log2(double v, bool* ok) {
    int e = 0;
    double m = std::frexp(v, &e);
    *ok = (m == 0.5) && e - 1 >= -20 && e - 1 <= 20;
    return e - 1;
}

static ind_status validate(const ind_landscape* L, const ind_dispersal* D, double nu, int* dt_log2) {
    if (!L || !D) return IND_ERR_ARG;
    // the spatially implicit model may leave speciation to its metacommunity
    const bool nu_ok = L->kind == IND_IMPLICIT ? (nu >= 0.0 && nu <= 1.0) : (nu > 0.0 && nu <= 1.0);
    if (!nu_ok) return IND_ERR_ARG;
    if (!(L->lambda > 0.0) || !std::isfinite(L->lambda)) return IND_ERR_ARG;
    bool ok = false;
    *dt_log2 = pow2_log2(L->delta_t, &ok);
    if (!ok || !(L->delta_t > 0.0)) return IND_ERR_ARG;
    if (!(L->lambda * L->delta_t >= 0x1p-20)) return IND_ERR_ARG;  // bounded interval search
    if (L->event_sampler != IND_SAMPLER_EXP && L->event_sampler != IND_SAMPLER_POISSON) return IND_ERR_ARG;
    if (L->event_sampler == IND_SAMPLER_POISSON && !(L->lambda * L->delta_t <= 64.0)) return IND_ERR_ARG;
    if (L->width < 1 || L->height < 1 || L->width > (1u << 20) || L->height > (1u << 20)) return IND_ERR_ARG;
    if (L->kind == IND_NONSPATIAL) {
        if (L->width != 1 || L->height != 1 || L->deme < 1 || L->deme >= (1u << 23)) return IND_ERR_ARG;
        if (D->kind != IND_DISPERSAL_UNIFORM) return IND_ERR_ARG;
    } else if (L->kind == IND_TORUS) {
        if (L->deme < 1 || L->deme >= (1u << 23)) return IND_ERR_ARG;
        if (D->kind != IND_DISPERSAL_GAUSSIAN) return IND_ERR_ARG;
        if (!(D->sigma > 0.0 && D->sigma <= 64.0)) return IND_ERR_ARG;
    } else if (L->kind == IND_MAP) {
        if (!L->deme_map) return IND_ERR_ARG;
        if (D->kind != IND_DISPERSAL_ALIAS_GAUSSIAN) return IND_ERR_ARG;
        if (!(D->sigma > 0.0 && D->sigma <= 64.0) || D->radius < 1 || D->radius > 40) return IND_ERR_ARG;
    } else if (L->kind == IND_IMPLICIT) {
        if (L->width != 1 || L->height != 1 || L->deme < 1 || L->deme >= (1u << 23)) return IND_ERR_ARG;
        if (D->kind != IND_DISPERSAL_UNIFORM) return IND_ERR_ARG;
        if (!(L->migration >= 0.0 && L->migration <= 1.0)) return IND_ERR_ARG;
        if (L->meta_size < 1 || L->meta_size > (1ull << 31)) return IND_ERR_ARG;
        if (!(L->meta_nu > 0.0 && L->meta_nu <= 1.0)) return IND_ERR_ARG;
        if (nu == 0.0 && L->migration == 0.0) return IND_ERR_ARG;  // no lineage could ever end
    } else {
        return IND_ERR_ARG;
    }
    const uint64_t dmax = L->kind == IND_MAP ? 255u : L->deme;
    if ((uint64_t)L->width * L->height * dmax > (1ull << 32) - 1) return IND_ERR_ARG;
    return IND_OK;
}

ind_status sim_create(const ind_landscape* L, const ind_dispersal* D, double nu, uint64_t seed, void* cuda_stream,
                      ind_sim** out) {
    if (!out) return IND_ERR_ARG;
    *out = nullptr;
    int dt_log2 = 0;
    ind_status st = validate(L, D, nu, &dt_log2);
    if (st != IND_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    st = ensure_ln_tables(s);
    if (st != IND_OK) return st;
    ind_sim* m = new (std::nothrow) ind_sim();
    if (!m) return IND_ERR_OOM;
    m->land = *L;
    m->land.deme_map = nullptr;
    m->disp = *D;
    m->nu = nu;
    m->seed = seed;
    m->stream = s;
    m->tables.stream = m->sample.stream = m->results.stream = m->events.stream = s;
    ind_default_tuning(&m->tuning);
    m->dt_log2 = dt_log2;
    seed_key(seed, &m->sk0, &m->sk1);
    m->nu_thr = (uint64_t)std::ceil(nu * 0x1p53);
    m->slot_deme = L->kind == IND_MAP ? 0 : L->deme;
    m->n_slots = (uint64_t)L->width * L->height * L->deme;
    auto fail = [&](ind_status e) {
        m->tables.release_all();
        delete m;
        return e;
    };
    if (L->event_sampler == IND_SAMPLER_POISSON) {
        std::vector<uint64_t> cdf = host_poisson_cdf(L->lambda * L->delta_t);
        const std::vector<uint32_t> guide = fine_guide(cdf);
        m->pois_n = (uint32_t)cdf.size();
        m->d_pois = m->tables.get<uint64_t>(cdf.size());
        m->d_pois_guide = m->tables.get<uint32_t>(GUIDE_N);
        if (!m->d_pois || !m->d_pois_guide) return fail(IND_ERR_OOM);
        if (cudaMemcpyAsync(m->d_pois, cdf.data(), cdf.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(m->d_pois_guide, guide.data(), GUIDE_N * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            g_last_cuda_error.store((int)cudaGetLastError());
            return fail(IND_ERR_CUDA);
        }
    }
    if (L->kind == IND_TORUS) {
        std::vector<uint64_t> cdf = host_gauss_cdf(D->sigma);
        m->gauss_half = host_gauss_half(D->sigma);
        m->gauss_n = (uint32_t)cdf.size();
        const std::vector<uint32_t> guide = fine_guide(cdf);
        m->d_gauss = m->tables.get<uint64_t>(cdf.size());
        m->d_gauss_guide = m->tables.get<uint32_t>(GUIDE_N);
        if (!m->d_gauss || !m->d_gauss_guide) return fail(IND_ERR_OOM);
        if (cudaMemcpyAsync(m->d_gauss, cdf.data(), cdf.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(m->d_gauss_guide, guide.data(), GUIDE_N * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            g_last_cuda_error.store((int)cudaGetLastError());
            return fail(IND_ERR_CUDA);
        }
    }
    if (L->kind == IND_MAP) {
        const size_t ncell = (size_t)L->width * L->height;
        std::vector<uint8_t> dm(ncell);
        if (cudaMemcpy(dm.data(), L->deme_map, ncell, cudaMemcpyDefault) != cudaSuccess) {
            g_last_cuda_error.store((int)cudaGetLastError());
            return fail(IND_ERR_CUDA);
        }
        uint32_t maxd = 0;
        m->n_slots = 0;
        std::vector<uint32_t> cells, row_of(ncell, 0xFFFFFFFFu);
        for (size_t c = 0; c < ncell; ++c) {
            maxd = std::max<uint32_t>(maxd, dm[c]);
            m->n_slots += dm[c];
            if (dm[c]) {
                row_of[c] = (uint32_t)cells.size();
                cells.push_back((uint32_t)c);
            }
        }
        if (cells.empty()) return fail(IND_ERR_ARG);
        m->slot_deme = maxd;
        const int R = (int)D->radius;
        std::vector<int8_t> off;
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx)
                if (dx * dx + dy * dy <= R * R) {
                    off.push_back((int8_t)dx);
                    off.push_back((int8_t)dy);
                }
        m->n_off = (uint32_t)(off.size() / 2);
        m->n_rows = (uint32_t)cells.size();
        std::vector<uint64_t> kw = host_kernel_weights(D->sigma, R);
        m->d_deme = m->tables.get<uint8_t>(ncell);
        m->d_row_of = m->tables.get<uint32_t>(ncell);
        m->d_off = m->tables.get<int8_t>(off.size());
        uint64_t* d_kw = m->tables.get<uint64_t>(kw.size());
        uint32_t* d_cells = m->tables.get<uint32_t>(cells.size());
        m->d_alias = m->tables.get<uint64_t>((size_t)m->n_rows * m->n_off);
        if (!m->d_deme || !m->d_row_of || !m->d_off || !d_kw || !d_cells || !m->d_alias) return fail(IND_ERR_OOM);
        bool okc = cudaMemcpyAsync(m->d_deme, dm.data(), ncell, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                   cudaMemcpyAsync(m->d_row_of, row_of.data(), ncell * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                   cudaMemcpyAsync(m->d_off, off.data(), off.size(), cudaMemcpyHostToDevice, s) == cudaSuccess &&
                   cudaMemcpyAsync(d_kw, kw.data(), kw.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                   cudaMemcpyAsync(d_cells, cells.data(), cells.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
        if (!okc) {
            g_last_cuda_error.store((int)cudaGetLastError());
            return fail(IND_ERR_CUDA);
        }
        const size_t per_warp = ((size_t)m->n_off * 12 + 15) & ~(size_t)15;
        int warps = (int)std::min<size_t>(8, std::max<size_t>(1, (96 * 1024) / per_warp));
        const size_t shb = per_warp * warps;
        if (cudaFuncSetAttribute(k_alias_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb) != cudaSuccess) {
            g_last_cuda_error.store((int)cudaGetLastError());
            return fail(IND_ERR_CUDA);
        }
        const uint32_t blocks = std::min<uint32_t>((m->n_rows + warps - 1) / warps, sm_count() * 8);
        k_alias_build<<<blocks, 32 * warps, shb, s>>>(m->d_deme, L->width, L->height, d_cells, m->n_rows, m->d_off,
                                                      m->n_off, d_kw, m->d_alias);
        g_launches.fetch_add(1);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
            g_last_cuda_error.store((int)cudaGetLastError());
            return fail(IND_ERR_CUDA);
        }
    }
    *out = m;
    return IND_OK;
}

ind_status sim_sample(ind_sim* m, double fraction, uint64_t sample_seed, uint64_t* n_sampled) {
    if (!m || !(fraction > 0.0 && fraction <= 1.0)) return IND_ERR_ARG;
    if (m->batch) {
        delete m->batch;
        m->batch = nullptr;
    }
    m->sample.release_all();
    m->results.release_all();
    m->events.release_all();
    m->d_species = m->d_key_loc = m->d_key_time = nullptr;
    m->d_events = nullptr;
    m->d_coal = nullptr;
    m->n_events = m->n_coal = 0;
    m->events_ready = false;
    m->finished = false;
    m->sampled = false;
    m->stats = ind_run_stats{};
    cudaStream_t s = m->stream;
    const uint64_t n_slots = (uint64_t)m->land.width * m->land.height * m->slot_deme;
    Pool tmp;
    tmp.stream = s;
    uint32_t* flags = tmp.get<uint32_t>(n_slots);
    uint32_t* pos = tmp.get<uint32_t>(n_slots);
    if (!flags || !pos) {
        tmp.release_all();
        return IND_ERR_OOM;
    }
    uint32_t sk0, sk1;
    seed_key(sample_seed, &sk0, &sk1);
    const uint64_t thr = (uint64_t)std::ceil(fraction * 0x1p53);
    const uint32_t sms = sm_count();
    k_sample_flags<<<grid_for(n_slots, 256, sms * 32), 256, 0, s>>>(flags, n_slots, m->land.kind, m->land.width,
                                                                   m->land.deme, m->slot_deme, m->d_deme,
                                                                   fraction >= 1.0 ? 1 : 0, sk0, sk1, thr);
    g_launches.fetch_add(1);
    ind_status st = scan_u32(tmp, flags, pos, (uint32_t)n_slots, false, s);
    if (st != IND_OK) {
        tmp.release_all();
        return st;
    }
    uint32_t last_pos = 0, last_flag = 0;
    if (cudaMemcpyAsync(&last_pos, pos + n_slots - 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&last_flag, flags + n_slots - 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        g_last_cuda_error.store((int)cudaGetLastError());
        tmp.release_all();
        return IND_ERR_CUDA;
    }
    const uint64_t count = (uint64_t)last_pos + last_flag;
    m->d_sample = m->sample.get<uint64_t>(std::max<uint64_t>(count, 1));
    // result buffers are taken now, so that finishing a run (in a batch or a
    // server) allocates nothing
    m->d_species = m->results.get<uint64_t>(std::max<uint64_t>(count, 1));
    m->d_key_loc = m->results.get<uint64_t>(std::max<uint64_t>(count, 1));
    m->d_key_time = m->results.get<uint64_t>(std::max<uint64_t>(count, 1));
    if (!m->d_sample || !m->d_species || !m->d_key_loc || !m->d_key_time) {
        tmp.release_all();
        return IND_ERR_OOM;
    }
    k_sample_write<<<grid_for(n_slots, 256, sms * 32), 256, 0, s>>>(flags, pos, n_slots, m->land.width,
                                                                   m->slot_deme, m->d_sample);
    g_launches.fetch_add(1);
    tmp.release_all();
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        g_last_cuda_error.store((int)cudaGetLastError());
        return IND_ERR_CUDA;
    }
    m->n_sampled = count;
    m->sampled = true;
    m->stats.n_sampled = count;
    if (n_sampled) *n_sampled = count;
    return IND_OK;
}

ind_status sim_set_tuning(ind_sim* m, const ind_tuning* t) {
    if (!m) return IND_ERR_ARG;
    if (!t) {
        ind_default_tuning(&m->tuning);
        return IND_OK;
    }
    if (!tuning_ok(t)) return IND_ERR_ARG;
    m->tuning = *t;
    return IND_OK;
}

ind_status sim_stats(const ind_sim* m, ind_run_stats* out) {
    if (!m || !out) return IND_ERR_ARG;
    *out = m->stats;
    return IND_OK;
}

ind_status sim_run(ind_sim* m, uint64_t round_budget, ind_run_stats* out) {
    if (!m) return IND_ERR_ARG;
    if (!m->sampled) return IND_ERR_STATE;
    if (m->finished) {
        if (out) *out = m->stats;
        return IND_OK;
    }
    if (!m->batch) {
        Batch* b = new (std::nothrow) Batch();
        if (!b) return IND_ERR_OOM;
        b->sims.push_back(m);
        b->stream = m->stream;
        b->tun = m->tuning;
        ind_status st = batch_build(*b);
        if (st != IND_OK) {
            delete b;
            return st;
        }
        m->batch = b;
    }
    ind_status st = batch_run(*m->batch, round_budget);
    if (out) *out = m->stats;
    if (st == IND_OK) {
        delete m->batch;
        m->batch = nullptr;
    }
    return st;
}

ind_status sim_batch_run(ind_sim** sims, uint32_t n, const ind_tuning* tuning, ind_run_stats* per_sim) {
    if (!sims || n == 0) return IND_ERR_ARG;
    for (uint32_t i = 0; i < n; ++i) {
        if (!sims[i]) return IND_ERR_ARG;
        if (!sims[i]->sampled || sims[i]->finished || sims[i]->batch) return IND_ERR_STATE;
        for (uint32_t j = 0; j < i; ++j)
            if (sims[j] == sims[i]) return IND_ERR_ARG;
    }
    if (tuning && !tuning_ok(tuning)) return IND_ERR_ARG;
    Batch b;
    b.sims.assign(sims, sims + n);
    b.stream = sims[0]->stream;
    b.tun = tuning ? *tuning : sims[0]->tuning;
    // other streams' work (sampling) must be complete
    for (uint32_t i = 1; i < n; ++i)
        if (sims[i]->stream != b.stream) CK(cudaStreamSynchronize(sims[i]->stream));
    ind_status st = batch_build(b);
    if (st == IND_OK) st = batch_run(b, 0);
    if (per_sim)
        for (uint32_t i = 0; i < n; ++i) per_sim[i] = sims[i]->stats;
    return st;
}

ind_status sim_set_event_log(ind_sim* m, uint64_t capacity) {
    if (!m || capacity > (1ull << 31)) return IND_ERR_ARG;
    if (m->batch) return IND_ERR_STATE;  // a run in progress keeps the log it started with
    m->log_cap = capacity;
    return IND_OK;
}

ind_status sim_events(ind_sim* m, ind_event* out, uint64_t cap, uint64_t* n_events, ind_coalescence* co_out,
                      uint64_t co_cap, uint64_t* n_coalescences) {
    if (!m) return IND_ERR_ARG;
    if (!m->finished || !m->events_ready) return IND_ERR_STATE;
    const uint64_t ne = std::min(cap, m->n_events), nc = std::min(co_cap, m->n_coal);
    if (out && ne) CK(cudaMemcpyAsync(out, m->d_events, ne * sizeof(ind_event), cudaMemcpyDefault, m->stream));
    if (co_out && nc)
        CK(cudaMemcpyAsync(co_out, m->d_coal, nc * sizeof(ind_coalescence), cudaMemcpyDefault, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (n_events) *n_events = m->n_events;
    if (n_coalescences) *n_coalescences = m->n_coal;
    return IND_OK;
}

ind_status sim_species(ind_sim* m, uint64_t* species_out, uint64_t* n_species_out) {
    if (!m) return IND_ERR_ARG;
    if (!m->finished) return IND_ERR_STATE;
    if (species_out && m->n_sampled) {
        CK(cudaMemcpyAsync(species_out, m->d_species, m->n_sampled * 8, cudaMemcpyDefault, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    if (n_species_out) *n_species_out = m->n_species;
    return IND_OK;
}

ind_status sim_species_keys(ind_sim* m, uint64_t* key_loc, uint64_t* key_time) {
    if (!m) return IND_ERR_ARG;
    if (!m->finished) return IND_ERR_STATE;
    if (m->n_sampled) {
        if (key_loc) CK(cudaMemcpyAsync(key_loc, m->d_key_loc, m->n_sampled * 8, cudaMemcpyDefault, m->stream));
        if (key_time) CK(cudaMemcpyAsync(key_time, m->d_key_time, m->n_sampled * 8, cudaMemcpyDefault, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    return IND_OK;
}

size_t sim_mem_estimate(const ind_landscape* L, const ind_dispersal* D, double fraction) {
    int dtl = 0;
    if (validate(L, D, 0.5, &dtl) != IND_OK || !(fraction > 0.0 && fraction <= 1.0)) return 0;
    const uint64_t ncell = (uint64_t)L->width * L->height;
    double individuals;
    size_t tables = 0;
    if (L->kind == IND_MAP) {
        // without reading the map: the largest possible deme everywhere
        individuals = (double)ncell * 255.0;
        uint64_t n_off = 0;
        const int R = (int)D->radius;
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx)
                if (dx * dx + dy * dy <= R * R) ++n_off;
        tables = ncell * (1 + 4 + 4 + n_off * 8) + 2 * n_off + 8 * (size_t)(R * R + 1);
    } else {
        individuals = (double)ncell * L->deme;
        if (L->kind == IND_TORUS) tables = 16 * (size_t)host_gauss_half(D->sigma) + 4 * GUIDE_N;
    }
    if (L->event_sampler == IND_SAMPLER_POISSON)
        tables += 8 * (size_t)host_poisson_n(L->lambda * L->delta_t) + 4 * GUIDE_N;
    const double sampled = std::ceil(individuals * fraction * 1.02) + 64;
    // sampling scratch (8 B per slot) is freed before the run
    const double slots = (L->kind == IND_MAP ? (double)ncell * 255.0 : individuals);
    // per lineage: 2 x 24 (buffers) + 20 (parent, keys) + 24 (outputs) + 8 (sample)
    // + 2 x 4 x 12 (dedup tables of twice the size) + 8 (used lists) + 32 x 2 (species sort)
    const double per = 48 + 20 + 24 + 8 + 96 + 8 + 64 + 16;
    const double bytes = tables + std::max(sampled * per, slots * 8.0) + (1 << 20);
    return (size_t)bytes;
}

void sim_destroy(ind_sim* m) {
    if (!m) return;
    if (m->batch) delete m->batch;
    m->results.release_all();
    m->sample.release_all();
    m->tables.release_all();
    m->events.release_all();
    delete m;
}

ind_status ind_habitat(uint64_t map_seed, uint32_t width, uint32_t height, double p_habitable, uint32_t max_deme,
                       uint8_t* deme_out, void* cuda_stream) {
    if (!deme_out || width < 1 || height < 1 || width > (1u << 20) || height > (1u << 20)) return IND_ERR_ARG;
    if (!(p_habitable >= 0.0 && p_habitable <= 1.0) || max_deme < 1 || max_deme > 255) return IND_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t sk0, sk1;
    seed_key(map_seed, &sk0, &sk1);
    const uint64_t thr = (uint64_t)std::ceil(p_habitable * 0x1p53);
    const uint64_t n = (uint64_t)width * height;
    cudaPointerAttributes attr{};
    bool on_device = cudaPointerGetAttributes(&attr, deme_out) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    uint8_t* dst = deme_out;
    Pool tmp;
    tmp.stream = s;
    if (!on_device) {
        dst = tmp.get<uint8_t>(n);
        if (!dst) return IND_ERR_OOM;
    }
    k_habitat<<<grid_for(n, 256, sm_count() * 32), 256, 0, s>>>(dst, width, height, sk0, sk1, thr, max_deme);
    g_launches.fetch_add(1);
    if (cudaGetLastError() != cudaSuccess) {
        tmp.release_all();
        return IND_ERR_CUDA;
    }
    if (!on_device) {
        if (cudaMemcpyAsync(deme_out, dst, n, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            tmp.release_all();
            return IND_ERR_CUDA;
        }
    }
    tmp.release_all();
    CK(cudaStreamSynchronize(s));
    return IND_OK;
}

ind_status ind_selftest(const uint64_t* in, uint64_t n, uint64_t* exp_q58_out, uint32_t* philox_out,
                        void* cuda_stream) {
    if (!in || n == 0 || n > (1ull << 30)) return IND_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    ind_status st = ensure_ln_tables(s);
    if (st != IND_OK) return st;
    Pool tmp;
    tmp.stream = s;
    uint64_t* d_in = tmp.get<uint64_t>(n);
    uint64_t* d_exp = exp_q58_out ? tmp.get<uint64_t>(n) : nullptr;
    uint32_t* d_ph = philox_out ? tmp.get<uint32_t>(4 * n) : nullptr;
    if (!d_in || (exp_q58_out && !d_exp) || (philox_out && !d_ph)) {
        tmp.release_all();
        return IND_ERR_OOM;
    }
    bool ok = cudaMemcpyAsync(d_in, in, n * 8, cudaMemcpyDefault, s) == cudaSuccess;
    if (ok) {
        k_selftest<<<grid_for(n, 256, sm_count() * 16), 256, 0, s>>>(d_in, n, d_exp, d_ph);
        g_launches.fetch_add(1);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok && exp_q58_out) ok = cudaMemcpyAsync(exp_q58_out, d_exp, n * 8, cudaMemcpyDefault, s) == cudaSuccess;
    if (ok && philox_out) ok = cudaMemcpyAsync(philox_out, d_ph, n * 16, cudaMemcpyDefault, s) == cudaSuccess;
    tmp.release_all();
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
        g_last_cuda_error.store((int)cudaGetLastError());
        return IND_ERR_CUDA;
    }
    return IND_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Species ranking without device allocation
//
// For callers that must not allocate device memory while they run: for
// instance a process that plans all of its device memory at start-up and
// forbids allocation afterwards, or code that runs inside an allocator of its
// own and cannot re-enter it.  The scratch of the sort/unique/rank step lives
// in one file-scope device array of fixed size, which every GPU that loads
// this library holds until the process exits.  In host code the array's name
// is only a host-side stand-in, so its device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) and passed to the
// kernels.  Every call shares the array: calls whose work overlaps on the GPU
// race and give wrong results.
// ---------------------------------------------------------------------------
constexpr uint32_t RANK_STATIC_MAX = 65536;  // individuals per call
constexpr size_t RANK_STATIC_ITEMS_BYTES = sizeof(SortItem) * RANK_STATIC_MAX;
constexpr size_t RANK_STATIC_BYTES = RANK_STATIC_ITEMS_BYTES + 2 * sizeof(uint32_t) * RANK_STATIC_MAX + 256;
static __device__ __align__(256) unsigned char g_rank_scratch[RANK_STATIC_BYTES];

static std::mutex g_rank_mutex;
static std::vector<unsigned char*> g_rank_addr;  // device address of g_rank_scratch, per device

static ind_status rank_scratch_address(unsigned char** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_rank_mutex);
    if ((int)g_rank_addr.size() <= dev) g_rank_addr.resize(dev + 1, nullptr);
    if (!g_rank_addr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_rank_scratch));
        g_rank_addr[dev] = (unsigned char*)p;
    }
    *out = g_rank_addr[dev];
    return IND_OK;
}

__global__ void k_rs_items(const uint64_t* __restrict__ kl, const uint64_t* __restrict__ kt, uint32_t n,
                           uint32_t n_pad, SortItem* __restrict__ items) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
        items[i] = i < n ? SortItem{0ull, kl[i], kt[i], i} : SortItem{~0ull, ~0ull, ~0ull, ~0ull};
}

__global__ void k_rs_heads(const SortItem* __restrict__ x, uint32_t n, uint32_t* __restrict__ head) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        head[i] = (i == 0 || x[i].b != x[i - 1].b || x[i].c != x[i - 1].c) ? 1u : 0u;
}

// inclusive scan of n <= RANK_STATIC_MAX flags in one block
__global__ void k_rs_scan(const uint32_t* __restrict__ head, uint32_t* __restrict__ incl, uint32_t n) {
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n; base += SCAN_TILE) {
        const uint32_t first = base + threadIdx.x * SCAN_ITEMS;
        uint32_t v[SCAN_ITEMS];
        uint32_t local = 0;
        for (uint32_t k = 0; k < SCAN_ITEMS; ++k) {
            v[k] = first + k < n ? head[first + k] : 0u;
            local += v[k];
        }
        uint32_t total;
        uint32_t run = carry + block_exclusive_scan(local, &total);
        for (uint32_t k = 0; k < SCAN_ITEMS; ++k) {
            run += v[k];
            if (first + k < n) incl[first + k] = run;
        }
        carry += total;
    }
}

__global__ void k_rs_out(const SortItem* __restrict__ x, const uint32_t* __restrict__ incl, uint32_t n,
                         uint64_t* __restrict__ species, uint64_t* __restrict__ count) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        species[x[i].d] = incl[i] - 1u;
        if (i == n - 1) *count = incl[i];
    }
}

extern "C" ind_status ind_species_rank_static(const uint64_t* key_loc, const uint64_t* key_time, uint64_t n,
                                              uint64_t* species_out, uint64_t* n_species_out, void* cuda_stream) {
    if (n > RANK_STATIC_MAX) return IND_ERR_ARG;  // beyond the fixed scratch
    if (n > 0 && (!key_loc || !key_time || !species_out)) return IND_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* base = nullptr;
    ind_status st = rank_scratch_address(&base);
    if (st != IND_OK) return st;
    SortItem* items = (SortItem*)base;
    uint32_t* head = (uint32_t*)(base + RANK_STATIC_ITEMS_BYTES);
    uint32_t* incl = head + RANK_STATIC_MAX;
    uint64_t* count = (uint64_t*)(incl + RANK_STATIC_MAX);
    // the count must start at zero: an empty input leaves it untouched
    CK(cudaMemsetAsync(count, 0, sizeof(uint64_t), s));
    if (n > 0) {
        const uint32_t nn = (uint32_t)n;
        uint32_t np = 2048;
        while (np < nn) np <<= 1;
        const uint32_t sms = sm_count();
        k_rs_items<<<grid_for(np, 256, sms * 8), 256, 0, s>>>(key_loc, key_time, nn, np, items);
        CKL();
        const uint32_t sh_threads = 1024, span = 2 * sh_threads;
        const size_t sh_bytes = sizeof(SortItem) * span;
        CK(cudaFuncSetAttribute(k_bitonic_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_bytes));
        for (uint32_t k = 2; k <= np; k <<= 1) {
            uint32_t j = k >> 1;
            for (; j >= span; j >>= 1) {
                k_bitonic_global<<<(np + 255) / 256, 256, 0, s>>>(items, np, j, k);
                CKL();
            }
            k_bitonic_shared<<<np / span, sh_threads, sh_bytes, s>>>(items, np, k, j);
            CKL();
        }
        k_rs_heads<<<grid_for(nn, 256, sms * 8), 256, 0, s>>>(items, nn, head);
        CKL();
        k_rs_scan<<<1, SCAN_BLOCK, 0, s>>>(head, incl, nn);
        CKL();
        k_rs_out<<<grid_for(nn, 256, sms * 8), 256, 0, s>>>(items, incl, nn, species_out, count);
        CKL();
    }
    if (n_species_out) {
        CK(cudaMemcpyAsync(n_species_out, count, sizeof(uint64_t), cudaMemcpyDefault, s));
        CK(cudaStreamSynchronize(s));
    }
    return IND_OK;
}

// ---------------------------------------------------------------------------
// Continuous-batching server
// ---------------------------------------------------------------------------
__global__ void k_rank_single(const SortItem* __restrict__ x, const uint32_t* n_items, const uint32_t* __restrict__ incl,
                              uint32_t* __restrict__ rank_of_root, uint64_t* __restrict__ count) {
    const uint32_t n = *n_items;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        rank_of_root[x[i].d] = incl[i] - 1u;
        if (i == n - 1) *count = incl[i];
    }
}

struct SrvSlot {
    ind_sim* sim = nullptr;
    uint64_t ticket = 0;
    uint32_t g0 = 0, n = 0;
    uint64_t bytes = 0;
    bool active = false;
};

struct ind_server {
    Batch b;                       // resident batch: buffers sized by capacity, one slot per request
    cudaStream_t side = nullptr;   // resolution of finished requests
    cudaEvent_t ev_main = nullptr;
    uint64_t budget = 0, bytes_admitted = 0;
    uint32_t s_cap = 0, n_cap = 0;
    std::vector<SrvSlot> slots;
    std::vector<uint32_t> free_slots;
    std::map<uint32_t, uint32_t> free_gids;  // start -> length
    std::deque<std::pair<ind_sim*, uint64_t>> queue;
    uint32_t n_total = 0;                    // active lineages (host copy after a step)
    uint32_t parity = 0;
    bool chunk_in_flight = false;
    uint64_t next_ticket = 0;
    ind_server_stats st{};
    std::vector<uint64_t> done_tickets;      // finished, not yet reported
};

static uint64_t admission_bytes(const ind_sim* m) {
    // per lineage: buffers 2 x 24, parent 4, key 16, dedup tables 2 x 2 x 12, used lists 8,
    // species outputs 24, sample 8; plus the simulation's tables
    return m->n_sampled * 156ull + m->tables.total() + 4096;
}

static bool gid_alloc(ind_server* sv, uint32_t n, uint32_t* g0) {
    for (auto it = sv->free_gids.begin(); it != sv->free_gids.end(); ++it) {
        if (it->second >= n) {
            *g0 = it->first;
            const uint32_t start = it->first + n, len = it->second - n;
            sv->free_gids.erase(it);
            if (len) sv->free_gids[start] = len;
            return true;
        }
    }
    return false;
}

static void gid_free(ind_server* sv, uint32_t g0, uint32_t n) {
    if (n == 0) return;
    auto it = sv->free_gids.emplace(g0, n).first;
    auto nx = std::next(it);
    if (nx != sv->free_gids.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        sv->free_gids.erase(nx);
    }
    if (it != sv->free_gids.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            sv->free_gids.erase(it);
        }
    }
}

// resolve one finished request (on the side stream) and publish its results
static ind_status srv_finish(ind_server* sv, SrvSlot& sl, const SimState& h) {
    ind_sim* m = sl.sim;
    cudaStream_t s = sv->side;
    const uint32_t n = sl.n;
    if (n && !m->d_species) return IND_ERR_STATE;  // sim_sample provides the result buffers
    uint64_t n_species = 0;
    if (n) {
        Pool T;
        T.stream = s;
        uint32_t* root = T.get<uint32_t>(n);
        uint32_t* n_items = T.get<uint32_t>(1);
        uint32_t* head = T.get<uint32_t>(n);
        uint32_t* incl = T.get<uint32_t>(n);
        uint32_t* rank = T.get<uint32_t>(n);
        uint64_t* count = T.get<uint64_t>(1);
        uint32_t np = 2048;
        while (np < n) np <<= 1;
        if (!root || !n_items || !head || !incl || !rank || !count) {
            T.release_all();
            return IND_ERR_OOM;
        }
        const uint32_t sms = sm_count();
        CK(cudaMemsetAsync(n_items, 0, 4, s));
        // the item buffer is sized after the roots are counted
        SortItem* items_all = T.get<SortItem>(np);
        if (!items_all) {
            T.release_all();
            return IND_ERR_OOM;
        }
        k_roots_range<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(sv->b.dev.parent, sv->b.dev.key_loc,
                                                                 sv->b.dev.key_time, sl.g0, n, root, items_all,
                                                                 n_items);
        CKL();
        uint32_t h_items = 0;
        CK(cudaMemcpyAsync(&h_items, n_items, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        uint32_t sp = 2048;
        while (sp < h_items) sp <<= 1;
        k_pad_items<<<grid_for(sp, 256, sms * 16), 256, 0, s>>>(items_all, n_items, sp);
        CKL();
        const uint32_t sh_threads = 1024, span = 2 * sh_threads;
        const size_t sh_bytes = sizeof(SortItem) * span;
        CK(cudaFuncSetAttribute(k_bitonic_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_bytes));
        for (uint32_t k = 2; k <= sp; k <<= 1) {
            uint32_t j = k >> 1;
            for (; j >= span; j >>= 1) {
                k_bitonic_global<<<(sp + 255) / 256, 256, 0, s>>>(items_all, sp, j, k);
                CKL();
            }
            k_bitonic_shared<<<sp / span, sh_threads, sh_bytes, s>>>(items_all, sp, k, j);
            CKL();
        }
        k_heads<<<grid_for(h_items, 256, sms * 16), 256, 0, s>>>(items_all, n_items, head);
        CKL();
        ind_status st = scan_u32(T, head, incl, h_items, true, s);
        if (st != IND_OK) {
            T.release_all();
            return st;
        }
        k_rank_single<<<grid_for(h_items, 256, sms * 16), 256, 0, s>>>(items_all, n_items, incl, rank, count);
        CKL();
        k_outputs_range<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(root, rank, sv->b.dev.key_loc,
                                                                   sv->b.dev.key_time, sl.g0, n, m->d_species,
                                                                   m->d_key_loc, m->d_key_time);
        CKL();
        CK(cudaMemcpyAsync(&n_species, count, 8, cudaMemcpyDeviceToHost, s));
        T.release_all();
        CK(cudaStreamSynchronize(s));
    }
    m->n_species = n_species;
    m->stats.n_species = n_species;
    m->stats.rounds = h.rounds;
    m->stats.raw_events = h.raw_events;
    m->stats.unique_events = h.unique_events;
    m->stats.culled = h.culled;
    m->stats.n_sampled = n;
    m->stats.n_roots = n - h.culled;
    m->finished = true;
    sv->st.raw_events += h.raw_events;
    return IND_OK;
}

// admit queued requests in arrival order while they fit
static ind_status srv_admit(ind_server* sv, std::vector<uint32_t>& empty_admitted) {
    Batch& b = sv->b;
    cudaStream_t s = b.stream;
    bool any = false;
    while (!sv->queue.empty()) {
        ind_sim* m = sv->queue.front().first;
        const uint64_t ticket = sv->queue.front().second;
        const uint64_t bytes = admission_bytes(m);
        const uint32_t n = (uint32_t)m->n_sampled;
        if (sv->free_slots.empty() || sv->bytes_admitted + bytes > sv->budget ||
            (uint64_t)sv->n_total + n > sv->n_cap)
            break;
        uint32_t g0 = 0;
        if (n && !gid_alloc(sv, n, &g0)) break;
        const uint32_t slot = sv->free_slots.back();
        sv->free_slots.pop_back();
        sv->queue.pop_front();
        SrvSlot& sl = sv->slots[slot];
        sl.sim = m;
        sl.ticket = ticket;
        sl.g0 = g0;
        sl.n = n;
        sl.bytes = bytes;
        sl.active = true;
        sv->bytes_admitted += bytes;
        SimParams hp;
        fill_params(m, b.tun, hp);
        hp.n_lineages = n;
        hp.slot_base = (uint64_t)slot << 32;  // slots of different requests never collide
        hp.gid_base = g0;
        SimState hs;
        memset(&hs, 0, sizeof(hs));
        hs.n_active = n;
        hs.done = n == 0 ? 1u : 0u;
        {
            // first horizon step, as horizon_step() computes it on the device
            const double dn = (double)std::max<uint32_t>(n, 1u);
            const double floor_ev = dn < hp.busy_lineages ? hp.tail_events : hp.min_events;
            const double per = std::max(floor_ev, std::min(hp.occupancy_step * hp.n_slots / dn, hp.events_per_round / dn));
            hs.horizon = std::min(per, hp.max_step_events) / hp.lambda;
        }
        CK(cudaMemcpyAsync(b.d_params + slot, &hp, sizeof(hp), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(b.d_state + slot, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
        if (n) {
            k_append<<<grid_for(n, 256, sm_count() * 16), 256, 0, s>>>(b.dev, sv->n_total, n, slot, g0, m->d_sample);
            CKL();
        }
        sv->n_total += n;
        sv->st.admitted += 1;
        if (n == 0) empty_admitted.push_back(slot);
        any = true;
    }
    if (any) {
        // resident count and the current round's dedup-table size
        Globals hg = *b.h_g;
        hg.n_total = sv->n_total;
        uint32_t cap = 2u;
        while (cap < 2u * sv->n_total && cap < b.dev.ht_cap) cap <<= 1;
        hg.mask[sv->parity] = cap - 1u;
        CK(cudaMemcpyAsync(&b.d_g->n_total, &hg.n_total, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(&b.d_g->mask[sv->parity], &hg.mask[sv->parity], sizeof(uint32_t), cudaMemcpyHostToDevice,
                           s));
        CK(cudaStreamSynchronize(s));  // the pageable sources above are locals
    }
    return IND_OK;
}

extern "C" {

ind_status srv_create(uint64_t budget, uint32_t max_sims, const ind_tuning* tuning, void* cuda_stream,
                      ind_server** out) {
    if (!out || budget < (1u << 20) || max_sims < 1 || max_sims > 65536) return IND_ERR_ARG;
    if (tuning && !tuning_ok(tuning)) return IND_ERR_ARG;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    ind_status st = ensure_ln_tables(s);
    if (st != IND_OK) return st;
    ind_server* sv = new (std::nothrow) ind_server();
    if (!sv) return IND_ERR_OOM;
    Batch& b = sv->b;
    b.stream = s;
    if (tuning) b.tun = *tuning;
    else ind_default_tuning(&b.tun);
    b.pool.stream = b.scratch.stream = s;
    sv->budget = budget;
    sv->s_cap = max_sims;
    sv->n_cap = (uint32_t)std::min<uint64_t>(budget / 156ull, (1ull << 29));
    b.n_sims = max_sims;
    const uint32_t n = std::max<uint32_t>(sv->n_cap, 1u);
    Pool& P = b.pool;
    b.d_params = P.get<SimParams>(max_sims);
    b.d_state = P.get<SimState>(max_sims);
    b.d_g = P.get<Globals>(1);
    BatchDev& d = b.dev;
    bool ok = b.d_params && b.d_state && b.d_g;
    for (int t = 0; t < 2 && ok; ++t) {
        d.lin[t].loc = P.get<uint64_t>(n);
        d.lin[t].tn = P.get<double>(n);
        d.lin[t].gid = P.get<uint32_t>(n);
        d.lin[t].sim = P.get<uint32_t>(n);
        ok = d.lin[t].loc && d.lin[t].tn && d.lin[t].gid && d.lin[t].sim;
    }
    d.parent = P.get<uint32_t>(n);
    d.key_loc = P.get<uint64_t>(n);
    d.key_time = P.get<uint64_t>(n);
    uint32_t cap = 2;
    while (cap < 2u * n && cap < (1u << 31)) cap <<= 1;
    d.ht_cap = cap;
    for (int t = 0; t < 2 && ok; ++t) {
        d.ht_key[t] = P.get<unsigned long long>(cap);
        d.ht_val[t] = P.get<uint32_t>(cap);
        d.ht_used[t] = P.get<uint32_t>(n);
        ok = d.ht_key[t] && d.ht_val[t] && d.ht_used[t];
    }
    ok = ok && d.parent && d.key_loc && d.key_time;
    if (!ok) {
        delete sv;
        return IND_ERR_OOM;
    }
    d.P = b.d_params;
    d.S = b.d_state;
    d.G = b.d_g;
    d.n_sims = max_sims;
    d.lpl = b.tun.lineages_per_lane;
    d.events_per_visit = b.tun.events_per_visit;
    d.coop_lineages = b.tun.coop_lineages;
    d.dedup = b.tun.dedup ? 1 : 0;
    d.count_unique = 0;  // exact counting is a batch-only measurement mode
    d.need_ln = 1;       // requests of either sampler may arrive
    auto fail = [&](cudaError_t e) {
        g_last_cuda_error.store((int)e);
        delete sv;
        return IND_ERR_CUDA;
    };
    cudaError_t e = cudaSuccess;
    std::vector<SimState> init(max_sims);
    for (auto& x : init) {
        memset(&x, 0, sizeof(x));
        x.done = 1;
    }
    if ((e = cudaMemcpyAsync(b.d_state, init.data(), sizeof(SimState) * max_sims, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(b.d_params, 0, sizeof(SimParams) * max_sims, s)) ||
        (e = cudaMemsetAsync(b.d_g, 0, sizeof(Globals), s)))
        return fail(e);
    for (int t = 0; t < 2; ++t)
        if ((e = cudaMemsetAsync(d.ht_key[t], 0xFF, sizeof(unsigned long long) * cap, s)) ||
            (e = cudaMemsetAsync(d.ht_val[t], 0xFF, sizeof(uint32_t) * cap, s)))
            return fail(e);
    if ((e = cudaMallocHost(&b.h_g, sizeof(Globals))) || (e = cudaStreamSynchronize(s))) return fail(e);
    memset(b.h_g, 0, sizeof(Globals));
    b.h_state.resize(max_sims);
    const uint32_t sms = sm_count();
    if ((e = cudaFuncSetAttribute(k_advance<false, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES)) ||
        (e = set_coop_smem<false>()) ||
        (e = cudaFuncSetAttribute(k_advance_sm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES)))
        return fail(e);
    b.adv_threads = b.tun.block_threads;
    b.adv_blocks = sms * b.tun.blocks_per_sm;
    b.cmp_blocks = sms * 4;
    if (b.tun.profile) {
        b.ev_start.resize(b.tun.rounds_per_check);
        b.ev_end.resize(b.tun.rounds_per_check);
        for (uint32_t r = 0; r < b.tun.rounds_per_check; ++r)
            if ((e = cudaEventCreate(&b.ev_start[r])) || (e = cudaEventCreate(&b.ev_end[r]))) return fail(e);
    }
    if ((e = cudaStreamCreateWithFlags(&sv->side, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&sv->ev_main, cudaEventDisableTiming)))
        return fail(e);
    b.started = true;
    sv->slots.resize(max_sims);
    for (uint32_t i = max_sims; i > 0; --i) sv->free_slots.push_back(i - 1);
    sv->free_gids[0] = sv->n_cap;
    sv->st.lineage_capacity = sv->n_cap;
    *out = sv;
    return IND_OK;
}

ind_status srv_submit(ind_server* sv, ind_sim* m, uint64_t* ticket) {
    if (!sv || !m) return IND_ERR_ARG;
    if (!m->sampled || m->finished || m->batch) return IND_ERR_STATE;
    if (m->log_cap) return IND_ERR_ARG;  // served requests are not logged
    if (m->n_sampled > sv->n_cap || admission_bytes(m) > sv->budget) return IND_ERR_ARG;  // could never fit
    const uint64_t t = sv->next_ticket++;
    sv->queue.emplace_back(m, t);
    sv->st.submitted += 1;
    if (ticket) *ticket = t;
    return IND_OK;
}

ind_status srv_step(ind_server* sv, uint32_t rounds, uint64_t* finished, uint32_t cap, uint32_t* n_finished) {
    if (!sv || rounds < 1 || (cap && !finished)) return IND_ERR_ARG;
    Batch& b = sv->b;
    cudaStream_t s = b.stream;
    // 1. the chunk launched by the previous step has ended: read the state
    std::vector<uint32_t> newly_done;
    if (sv->chunk_in_flight) {
        CK(cudaMemcpyAsync(b.h_g, b.d_g, sizeof(Globals), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(b.h_state.data(), b.d_state, sizeof(SimState) * sv->s_cap, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        sv->chunk_in_flight = false;
        collect_profile(b, b.tun.rounds_per_check);
        if (b.h_g->error) return IND_ERR_DEVICE;
        sv->n_total = b.h_g->n_total;
        sv->parity = b.h_g->round & 1u;
        for (uint32_t i = 0; i < sv->s_cap; ++i)
            if (sv->slots[i].active && b.h_state[i].done) newly_done.push_back(i);
    }
    // 2. admit what fits (finished requests' ids and slots free up below)
    ind_status st = srv_admit(sv, newly_done);  // requests with no lineages finish at once
    if (st != IND_OK) return st;
    // 3. launch the next chunk of rounds on the main stream
    if (sv->n_total > 0) {
        st = batch_rounds(b, rounds);
        if (st != IND_OK) return st;
        sv->chunk_in_flight = true;
        sv->st.rounds += rounds;
    }
    // 4. resolve the finished requests on the side stream while the chunk runs
    for (uint32_t i : newly_done) {
        SrvSlot& sl = sv->slots[i];
        SimState zero;
        memset(&zero, 0, sizeof(zero));
        st = srv_finish(sv, sl, sl.n ? b.h_state[i] : zero);
        if (st != IND_OK) return st;
        sv->bytes_admitted -= sl.bytes;
        gid_free(sv, sl.g0, sl.n);
        sl.active = false;
        sl.sim = nullptr;
        sv->free_slots.push_back(i);
        sv->done_tickets.push_back(sl.ticket);
        sv->st.finished += 1;
    }
    // 5. report
    uint32_t k = 0;
    while (k < cap && !sv->done_tickets.empty()) {
        finished[k++] = sv->done_tickets.front();
        sv->done_tickets.erase(sv->done_tickets.begin());
    }
    if (n_finished) *n_finished = k;
    uint64_t resident = 0;
    for (auto& sl : sv->slots) resident += sl.active ? 1 : 0;
    sv->st.queued = sv->queue.size();
    sv->st.resident = resident;
    sv->st.resident_lineages = sv->n_total;
    sv->st.bytes_admitted = sv->bytes_admitted;
    return IND_OK;
}

ind_status srv_stats(const ind_server* sv, ind_server_stats* out) {
    if (!sv || !out) return IND_ERR_ARG;
    *out = sv->st;
    return IND_OK;
}

void srv_destroy(ind_server* sv) {
    if (!sv) return;
    cudaStreamSynchronize(sv->b.stream);
    if (sv->side) {
        cudaStreamSynchronize(sv->side);
        cudaStreamDestroy(sv->side);
    }
    if (sv->ev_main) cudaEventDestroy(sv->ev_main);
    delete sv;
}

}  // extern "C"
