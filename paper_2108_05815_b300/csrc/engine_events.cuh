// engine_events.cuh -- per-lineage event arithmetic: event-time searches, dispersal, the event step, dedup and log helpers.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

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
    // spatially implicit model
    uint64_t meta_size, m_thr, meta_nu_thr;
    // habitat map: offsets of the dispersal kernel and their count, and the
    // alias rows (register copies: the row address is on the event chain)
    uint32_t n_off;
    const int8_t* off;
    const uint64_t* alias;
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
    c.meta_size = __ldg(&p->meta_size);
    c.m_thr = __ldg(&p->m_thr);
    c.meta_nu_thr = __ldg(&p->meta_nu_thr);
    c.n_off = __ldg(&p->n_off);
    c.off = p->off;
    c.alias = p->alias;
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

// Exp(lambda) draw.  LAM1 (lambda = 1) is a template argument rather than a
// select: given both operands the compiler evaluates the binary64 division
// even where it is not used, on the latency chain and on B300's narrow FP64
// pipe.  Callers branch on c.lam1 once per search.
// div_rn_call: the division out of line, for code whose lanes mix lambdas
// (a call is not evaluated speculatively)
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

// The same search for lambda = 1 in integer arithmetic (see
// coop_next_exp_int): in interval k >= 1 the points are the multiples of
// u = 2^(e-52), e = floor(log2 k) + d, the start is P = k 2^(52 - floor(log2 k))
// and a draw adds its value in u rounded to the nearest integer (a tie to
// the even sum).  The rounding of each draw is independent of the sum, so
// only an integer add and two compares per draw remain sequential, where
// the binary64 form waits 64 cycles per add on B300.  Intervals outside
// the range (k = 0, extreme delta_t) go to the binary64 form.
template <int WIDE>
__device__ double next_event_time_exp_int(const LaneSim& c, uint64_t loc, double tau, const LnC& ln) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    const int d = c.dt_log2;
    uint64_t k = floor_div_pow2(tau_b, d);
    // tau in units of its own interval (later intervals: every point is after tau)
    uint64_t T = (tau_b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    for (uint32_t iv = 0; iv < INTERVAL_LIMIT; ++iv, T = 0ull) {
        if (k >= (1ull << 52)) return -1.0;
        const int lg = 63 - __clzll((long long)k);
        const int sft = lg + d + 6;
        if (k == 0ull || sft < 0 || sft > 63) return next_event_time_exp<WIDE, true>(c, loc, tau, ln);
        const int sh = 52 - lg;
        uint64_t P = k << sh;
        const uint64_t E = (k + 1ull) << sh;
        bool next_interval = false;
        for (uint32_t j = 0; j < INTERVAL_BLOCK_LIMIT; j += WIDE) {
            uint64_t fl[2 * WIDE];
            uint32_t rnd[2 * WIDE];  // 0: round down, 1: up, 2: a tie
#pragma unroll
            for (int w = 0; w < WIDE; ++w) {
                const u64x2 b = stream_block(c.sk0, c.sk1, loc, k, j + w, TAG_INTERVAL);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // rounded once from X58 away from a midpoint of u, else
                    // to 53 bits first as binary64 does
                    const GridDraw g = exp1_grid((h ? b.hi : b.lo) >> 11, ln.L, ln.R, ln.ln2, ln.c3, sft);
                    uint64_t f = g.a;
                    uint32_t r = 0;
                    if (g.near) {
                        const uint64_t R = rn53(g.x58);
                        f = R >> sft;
                        if (sft > 0) {
                            const uint64_t rem = R & ((1ull << sft) - 1ull), half = 1ull << (sft - 1);
                            r = rem > half ? 1u : rem == half ? 2u : 0u;
                        }
                    }
                    fl[2 * w + h] = f;
                    rnd[2 * w + h] = r;
                }
            }
#pragma unroll
            for (int q = 0; q < 2 * WIDE; ++q) {
                // a draw of 2^54 u or more ends the interval whatever the rounding
                const uint64_t a = fl[q] < (1ull << 54) ? fl[q] : (1ull << 54);
                P += a + (rnd[q] == 1u ? 1ull : rnd[q] == 2u ? ((P + a) & 1ull) : 0ull);
                if (P >= E) {
                    next_interval = true;
                    break;
                }
                if (P > T) return __longlong_as_double((long long)(((uint64_t)(lg + d + 1023) << 52) |
                                                                  (P & 0xFFFFFFFFFFFFFull)));
            }
            if (next_interval) break;
        }
        if (!next_interval) return -1.0;
        ++k;
    }
    return -1.0;
}

// number of table entries <= r: the guide entry of r's bucket, and a scan
// of the table only where a threshold falls inside the bucket (plain loads:
// the warp kernel may pass tables staged in shared memory)
__device__ __forceinline__ uint32_t guided_count(const uint64_t* __restrict__ t, const uint32_t* __restrict__ guide,
                                                 uint32_t n, uint64_t r) {
    const uint32_t e = guide[r >> (64 - GUIDE_BITS)];
    uint32_t idx = e & ~GUIDE_SCAN;
    if (e & GUIDE_SCAN)
        while (idx < n && t[idx] <= r) ++idx;
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

// The same search with the points in integer arithmetic (see
// coop_next_poisson_short): point i of interval k >= 1 is
// P0 + (U dt / u rounded to the nearest integer, ties to even) in units
// u = 2^(e-52) of the interval's binade, P0 = k 2^(52 - floor(log2 k)) even.
// k = 0 goes to the binary64 form.
__device__ double next_event_time_poisson_int(const LaneSim& c, uint64_t loc, double tau) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    const int d = c.dt_log2;
    uint64_t k = floor_div_pow2(tau_b, d);
    if (k == 0ull) return next_event_time_poisson(c, loc, tau);
    for (uint32_t iv = 0; iv < INTERVAL_LIMIT; ++iv) {
        if (k >= (1ull << 52)) return -1.0;
        const int lg = 63 - __clzll((long long)k);  // 0 .. 51
        const int s = lg + 1;
        const uint64_t P0 = k << (52 - lg);
        const uint64_t ehi = (uint64_t)(lg + d + 1023) << 52;
        const u64x2 b0 = stream_block(c.sk0, c.sk1, loc, k, 0, TAG_INTERVAL);
        const uint32_t N = guided_count(c.pois_cdf, c.pois_guide, c.pois_n, b0.lo);
        uint64_t best = ~0ull;
        auto consider = [&](uint64_t r) {
            const uint64_t v = r >> 11;
            const uint64_t fl = v >> s, rem = v & ((1ull << s) - 1ull), half = 1ull << (s - 1);
            const uint64_t P = P0 + fl + ((rem > half || (rem == half && (fl & 1ull))) ? 1ull : 0ull);
            const uint64_t pb = P < (1ull << 53) ? (ehi | (P & 0xFFFFFFFFFFFFFull)) : ehi + (1ull << 52);
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
    if (c.sampler == 1) return next_event_time_poisson_int(c, loc, tau);
    return c.lam1 ? next_event_time_exp_int<WIDE>(c, loc, tau, ln) : next_event_time_exp<WIDE, false>(c, loc, tau, ln);
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
__device__ double coop_next_poisson_short_fp(const LaneSim& c, uint64_t loc, double tau, uint32_t lane) {
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

// The same search with the points in integer arithmetic.  For k >= 1,
// point i of interval k is the binary64 sum of k dt (exact) and U dt (exact,
// U = (draw >> 11) 2^-53); in the binade of k dt, e = floor(log2 k) + d,
// whose values are the multiples of u = 2^(e-52), that sum is
// P0 + (U dt / u rounded to the nearest integer, ties to even) with
// P0 = k 2^(52 - floor(log2 k)) even and U dt / u = (draw >> 11) 2^-(floor(log2 k) + 1).
// A sum that rounds up to (k + 1) dt is that value (2^(e+1) when it starts
// the next binade).  No binary64 arithmetic is on the chain.  k = 0 and
// k near 2^52 go to the binary64 form.
// k0: floor(tau / delta_t), the interval index of tau (the caller may form
// it ahead, off the event chain)
__device__ double coop_next_poisson_short(const LaneSim& c, uint64_t loc, double tau, uint32_t lane, uint64_t k0) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    const uint32_t m = lane >> 3, i = lane & 7u;
    const int d = c.dt_log2;
    if (k0 == 0ull) return coop_next_poisson_short_fp(c, loc, tau, lane);
    for (uint32_t round = 0; round < INTERVAL_LIMIT / 4; ++round, k0 += 4ull) {
        if (k0 + 4ull >= (1ull << 52)) return coop_next_poisson(c, loc, tau, lane);
        const uint64_t k = k0 + m;
        // draw 0 gives the count N; point i is draw 1 + i.  Lane i of the
        // group computes block i (0 .. 4: draws 0 .. 9), the group shares
        // them by shuffle: one block per lane instead of two
        const u64x2 bl = stream_block(c.sk0, c.sk1, loc, k, min(i, 4u), TAG_INTERVAL);
        const uint32_t g0 = lane & ~7u, src = g0 + ((1u + i) >> 1);
        const uint64_t d0 = __shfl_sync(0xFFFFFFFFu, bl.lo, g0);
        const uint64_t plo = __shfl_sync(0xFFFFFFFFu, bl.lo, src), phi = __shfl_sync(0xFFFFFFFFu, bl.hi, src);
        const int lg = 63 - __clzll((long long)k);  // 0 .. 51
        const uint64_t P0 = k << (52 - lg);
        const int e = lg + d;
        const uint32_t N = guided_count(c.pois_cdf, c.pois_guide, c.pois_n, d0);
        uint64_t pb = ~0ull;
        if (i < N) {
            const uint64_t v = ((i & 1u) ? plo : phi) >> 11;
            const int s = lg + 1;  // 1 .. 52
            const uint64_t fl = v >> s, rem = v & ((1ull << s) - 1ull), half = 1ull << (s - 1);
            const uint64_t P = P0 + fl + ((rem > half || (rem == half && (fl & 1ull))) ? 1ull : 0ull);
            const uint64_t q = P < (1ull << 53) ? ((uint64_t)(e + 1023) << 52) | (P & 0xFFFFFFFFFFFFFull)
                                                : (uint64_t)(e + 1024) << 52;
            if (q > tau_b) pb = q;
        }
        if (__any_sync(0xFFFFFFFFu, N > 8u)) return coop_next_poisson(c, loc, tau, lane);
        // the smallest point > tau of the four intervals is the smallest of
        // the first interval that has one: points of interval k lie in
        // [k dt, (k + 1) dt]
        const uint32_t hi = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(pb >> 32));
        if (hi != 0xFFFFFFFFu) {
            const uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(pb >> 32) == hi ? (uint32_t)pb : 0xFFFFFFFFu);
            return __longlong_as_double((long long)(((uint64_t)hi << 32) | lo));
        }
    }
    return -1.0;
}
__device__ __forceinline__ double coop_next_poisson_short(const LaneSim& c, uint64_t loc, double tau, uint32_t lane) {
    return coop_next_poisson_short(c, loc, tau, lane, floor_div_pow2((uint64_t)__double_as_longlong(tau), c.dt_log2));
}

// sums of exponentials: every lane runs interval k's binary64 running sum in
// the spec's order on the shuffled draws; intervals k + 1 .. k + 3 only need
// their first point
template <bool LAM1>
__device__ double coop_next_exp_short_fp(const LaneSim& c, uint64_t loc, double tau, const LnC& ln, uint32_t lane) {
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

// The short search for lambda = 1 in integer arithmetic, with the same
// result as the binary64 form.  For k >= 1 every point below the end of
// interval k lies in one binade [2^e, 2^(e+1)), e = floor(log2 k) + d
// (delta_t = 2^d), whose binary64 values are the multiples of u = 2^(e-52).
// Counted in u, interval k starts at P0 = k 2^(52 - floor(log2 k)) and ends
// at E = (k + 1) 2^(52 - floor(log2 k)) (at most 2^53), and the binary64 sum
// of a point P u and a draw x = RN53(q) 2^-58 is P + (x / u rounded to the
// nearest integer, a tie going to the even sum).  That is exact while the
// sum stays below 2^(e+1), and at or above E exactly when binary64's is,
// which ends the interval either way.  Each lane rounds its own draw; the
// direction of a tie depends on the parity of the sum before it, which
// follows from the ties and the parities of the lanes below (two ballots).
// Prefix sums over lanes 8 m .. 8 m + 7 (shuffles) then give every point of
// interval k at once, where the binary64 form adds them one after another
// at 64 cycles per add on B300.  Usually the first point after tau is among
// the first three of interval k0, or that interval ends first: every lane
// then decides from interval k0's first three draws (broadcast) and, where
// that interval ends first, the first point of the lowest later interval
// that has one (chosen by a vote), without the prefix sums or the tie
// votes.  Outside its range (k = 0, extreme delta_t,
// k near 2^52) it hands over to the binary64 form.
// DT: delta_t = 2^DT known at compile time (DT_ANY: the simulation's own)
constexpr int DT_ANY = 99;

// kio: in, floor(tau / delta_t), the interval index of tau, which the
// caller carries from the search that returned tau (so that it is not
// recomputed from tau's bits on the chain); out, that of the result.
template <int DT>
__device__ double coop_next_exp_int_dt(const LaneSim& c, uint64_t loc, double tau, const LnC& ln, uint32_t lane,
                                       uint64_t& kio) {
    const uint64_t tau_b = (uint64_t)__double_as_longlong(tau);
    const uint32_t m = lane >> 3, i = lane & 7u;
    const int d = DT == DT_ANY ? c.dt_log2 : DT;
    uint64_t k0 = kio;
    const uint64_t T = (tau_b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // tau in units of interval k0
    for (uint32_t round = 0; round < INTERVAL_LIMIT / 4; ++round, k0 += 4ull) {
        // the draws first: the range check and the interval bounds below do
        // not depend on them and overlap their latency
        const uint64_t k = k0 + m;
        const u64x2 b = stream_block(c.sk0, c.sk1, loc, k, i >> 1, TAG_INTERVAL);
        const int lg0 = 63 - __clzll((long long)k0);
        const int lg3 = 63 - __clzll((long long)(k0 + 3ull));
        const int lg = 63 - __clzll((long long)k);
        const int sft = min(max(lg + d + 6, 0), 63);  // x / u = RN53(q) 2^-sft
        const int sh = max(52 - lg, 0);  // in range below: 1 .. 52
        const uint64_t P0 = k << sh;
        const uint64_t E = (k + 1ull) << sh;
        if (k0 == 0ull || lg0 + d + 6 < 0 || lg3 + d + 6 > 63 || k0 + 4ull >= (1ull << 52)) {
            const double r = coop_next_exp_short_fp<true>(c, loc, tau, ln, lane);
            kio = floor_div_pow2((uint64_t)__double_as_longlong(r), d);
            return r;
        }
        // the lane's draw in u, rounded once from X58 (exact away from a
        // midpoint of u; the draws near one are rounded twice below)
        const GridDraw g = exp1_grid(((i & 1u) ? b.hi : b.lo) >> 11, ln.L, ln.R, ln.ln2, ln.c3, sft);
        const unsigned nearm = __ballot_sync(0xFFFFFFFFu, g.near);
        const uint64_t tu = round == 0 ? T : 0ull;  // later rounds: every point is after tau
        {
            // The decision from four draws (the usual case): interval k0's
            // first three points p0 <= p1 <= p2 by broadcast and local adds,
            // and the later intervals' first points, whose lowest one below
            // its interval's end is fetched while those adds run.  A draw of
            // more than 2^54 u ends the interval whatever follows.
            // (with delta_t = 1 a draw is below 2^58 u: three of them cannot
            // overflow, and the cap is left out)
            const uint64_t S = DT == 0 || g.a < (1ull << 54) ? g.a : (1ull << 54);
            const uint64_t P = P0 + S;
            const uint64_t bits = ((uint64_t)(lg + d + 1023) << 52) | (P & 0xFFFFFFFFFFFFFull);
            const unsigned later = __ballot_sync(0xFFFFFFFFu, m > 0u && i == 0u && P < E);
            const int wl = (later & 0x100u) ? 8 : ((later & 0x10000u) ? 16 : 24);  // lanes 8, 16, 24 vote
            const uint64_t bl = __shfl_sync(0xFFFFFFFFu, bits, wl);
            const uint64_t s0 = __shfl_sync(0xFFFFFFFFu, S, 0);
            const uint64_t s1 = __shfl_sync(0xFFFFFFFFu, S, 1);
            const uint64_t s2 = __shfl_sync(0xFFFFFFFFu, S, 2);
            const int sh0 = max(52 - lg0, 0);
            const uint64_t p0 = (k0 << sh0) + s0, p1 = p0 + s1, p2 = p1 + s2;
            // points at or below tau are passed; the first one after it
            // either lies in interval k0 or ends it
            if (!(nearm & 0x01010107u) && p2 > tu) {
                const uint64_t pj = p0 > tu ? p0 : (p1 > tu ? p1 : p2);
                if (pj < ((k0 + 1ull) << sh0)) {
                    kio = k0;
                    return __longlong_as_double(
                        (long long)(((uint64_t)(lg0 + d + 1023) << 52) | (pj & 0xFFFFFFFFFFFFFull)));
                }
                if (later) {
                    kio = k0 + (uint64_t)(wl >> 3);
                    return __longlong_as_double((long long)bl);
                }
                continue;  // intervals k0 .. k0 + 3 hold no point after tau
            }
        }
        // All eight draws of interval k0 by prefix sums, each draw near a
        // midpoint of u rounded as binary64 does: to 53 bits, then to u, the
        // tie rounded down here and settled below by the parity of the sum
        // (R + half - 1 carries exactly when the remainder is above half).
        uint64_t a = g.a;
        bool tie = false;
        if (nearm) {
            const uint64_t R = rn53(g.x58);
            const uint64_t gmask = (1ull << sft) - 1ull;
            a = (R + (gmask >> 1)) >> sft;
            tie = sft > 0 && (R & gmask) == (gmask >> 1) + 1ull;
        }
        // prefix sums as if no draw were a tie (rare); a tie redoes them
        const unsigned ties = __ballot_sync(0xFFFFFFFFu, tie);
        uint64_t S = a < (1ull << 54) ? a : (1ull << 54);
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) {
            const uint64_t o = __shfl_up_sync(0xFFFFFFFFu, S, off, 8);
            if (i >= (uint32_t)off) S += o;
        }
        if (ties) {
            // parity of the sum below lane i: the parities of the draws after
            // the last tie below i (a tie leaves an even sum; P0 is even)
            const unsigned odd = __ballot_sync(0xFFFFFFFFu, (a & 1ull) != 0ull);
            const unsigned tm = (ties >> (8u * m)) & 0xFFu, om = (odd >> (8u * m)) & 0xFFu;
            const unsigned below = (1u << i) - 1u, tb = tm & below;
            const unsigned upto = tb ? (2u << (31 - __clz(tb))) - 1u : 0u;
            const unsigned parity = (unsigned)__popc(om & below & ~upto) & 1u;
            if (tie) a += (parity ^ (unsigned)a) & 1u;
            S = a < (1ull << 54) ? a : (1ull << 54);
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                const uint64_t o = __shfl_up_sync(0xFFFFFFFFu, S, off, 8);
                if (i >= (uint32_t)off) S += o;
            }
        }
        const uint64_t P = P0 + S;
        // this lane's point as binary64 bits (meaningful where P < E), and
        // the three votes side by side: interval k0's first point after tau,
        // its end, and the later intervals' first points
        const uint64_t bits = ((uint64_t)(lg + d + 1023) << 52) | (P & 0xFFFFFFFFFFFFFull);
        const unsigned found = __ballot_sync(0xFFFFFFFFu, m == 0u && P > tu && P < E);
        const unsigned ended = __ballot_sync(0xFFFFFFFFu, m == 0u && P >= E);
        const unsigned later = __ballot_sync(0xFFFFFFFFu, m > 0u && i == 0u && P < E);
        const unsigned hit = found | ended;
        if (!hit) {  // eight points up to tau
            const double r = coop_next_exp<true>(c, loc, tau, ln, lane);
            kio = floor_div_pow2((uint64_t)__double_as_longlong(r), d);
            return r;
        }
        const int j = __ffs(hit) - 1;
        // the first point of interval k0 after tau, else (interval k0 ended
        // first) the first point of the lowest later interval that has one
        const int w = (found >> j) & 1u ? j : (later ? __ffs(later) - 1 : -1);
        if (w >= 0) {
            kio = k0 + (uint64_t)(w >> 3);
            return __longlong_as_double((long long)__shfl_sync(0xFFFFFFFFu, bits, w));
        }
    }
    return -1.0;
}

// delta_t = 1, the usual case, with its shifts and bounds folded (about 3 %
// shorter per event than the general form on B300)
__device__ __forceinline__ double coop_next_exp_int(const LaneSim& c, uint64_t loc, double tau, const LnC& ln,
                                                    uint32_t lane, uint64_t& kio) {
    return c.dt_log2 == 0 ? coop_next_exp_int_dt<0>(c, loc, tau, ln, lane, kio)
                          : coop_next_exp_int_dt<DT_ANY>(c, loc, tau, ln, lane, kio);
}
__device__ __forceinline__ double coop_next_exp_int(const LaneSim& c, uint64_t loc, double tau, const LnC& ln,
                                                    uint32_t lane) {
    uint64_t k = floor_div_pow2((uint64_t)__double_as_longlong(tau), c.dt_log2);
    return coop_next_exp_int(c, loc, tau, ln, lane, k);
}

template <bool LAM1>
__device__ __forceinline__ double coop_next_exp_short(const LaneSim& c, uint64_t loc, double tau, const LnC& ln,
                                                      uint32_t lane) {
    if (LAM1) return coop_next_exp_int(c, loc, tau, ln, lane);
    return coop_next_exp_short_fp<false>(c, loc, tau, ln, lane);
}

// dispersal target from the event stream's draws 1, 2, 3 (draw 0 decided
// speciation): non-spatial uses d1; torus d1 (x), d2 (y), d3 (deme index),
// each axis a discretised normal by inversion, -half + #{k : cdf[k] <= d};
// map d1 (alias column and threshold), d2 (deme index); spatially implicit
// d1 (migration, or the metacommunity parent), d2 (parent after migration
// or locally)
// (KIND: the landscape kind when the caller knows it at compile time, -1
// for the simulation's own; srow: the origin cell's alias row staged in
// shared memory, or null to read it from global memory)
template <int KIND = -1>
__device__ __forceinline__ uint64_t disperse(const LaneSim& c, const SimParams* __restrict__ P, uint64_t loc,
                                            uint64_t d1, uint64_t d2, uint64_t d3,
                                            const uint64_t* srow = nullptr) {
    const int kind = KIND >= 0 ? KIND : c.kind;
    if (kind == KIND_NONSPATIAL) return pack_loc(0, 0, mulhi_u64_u32(d1, c.D));
    if (kind == KIND_IMPLICIT) {
        // in the metacommunity: a uniform parent there (d1); locally:
        // migration iff d1 says so, then the parent's index (d2) in the
        // metacommunity or the local community
        const uint64_t meta_n = c.meta_size;
        if (in_meta(loc)) return meta_loc(umulhi64(d1, meta_n));
        if ((d1 >> 11) < c.m_thr) return meta_loc(umulhi64(d2, meta_n));
        return pack_loc(0, 0, mulhi_u64_u32(d2, c.D));
    }
    const uint32_t x = loc_x(loc), y = loc_y(loc);
    if (kind == KIND_TORUS) {
        // both guide entries first, so that the two loads overlap; a table
        // scan only for draws in a bucket that holds a threshold
        // (plain loads: the warp kernel may pass tables staged in shared memory)
        const uint32_t ex = c.gauss_guide[d1 >> (64 - GUIDE_BITS)];
        const uint32_t ey = c.gauss_guide[d2 >> (64 - GUIDE_BITS)];
        uint32_t cx = ex & ~GUIDE_SCAN, cy = ey & ~GUIDE_SCAN;
        if ((ex | ey) & GUIDE_SCAN) {
            if (ex & GUIDE_SCAN)
                while (cx < c.gauss_n && c.gauss[cx] <= d1) ++cx;
            if (ey & GUIDE_SCAN)
                while (cy < c.gauss_n && c.gauss[cy] <= d2) ++cy;
        }
        const uint32_t tx = wrap_add(x, (int32_t)cx - c.gauss_half, c.W);
        const uint32_t ty = wrap_add(y, (int32_t)cy - c.gauss_half, c.H);
        const uint64_t ti = c.D > 1 ? mulhi_u64_u32(d3, c.D) : 0ull;
        return pack_loc(tx, ty, ti);
    }
    // habitat map: the origin cell's alias entry (which carries the alias
    // column's offset and both target demes, k_alias_build) and the
    // column's own offset load side by side, then one choice
    const uint32_t n_off = c.n_off;
    const uint32_t col = (uint32_t)(((d1 >> 32) * (uint64_t)n_off) >> 32);
    const uint64_t e = srow ? srow[col] : __ldg(c.alias + ((size_t)y * c.W + x) * n_off + col);
    const int8_t* off = c.off;  // plain loads: the warp kernel may stage the table in shared memory
    const int32_t cdx = off[2 * col], cdy = off[2 * col + 1];
    const uint32_t u = (uint32_t)d1;
    const bool take_col = (e >> 63) != 0 || u < (uint32_t)e;
    const int32_t adx = (int32_t)((uint32_t)(e >> 32) << 25) >> 25;  // 7-bit two's complement
    const int32_t ady = (int32_t)((uint32_t)(e >> 39) << 25) >> 25;
    const int32_t dx = take_col ? cdx : adx, dy = take_col ? cdy : ady;
    const uint32_t d = (uint32_t)(e >> (take_col ? 46 : 54)) & 0xFFu;
    const uint32_t tx = wrap_add(x, dx, c.W);
    const uint32_t ty = wrap_add(y, dy, c.H);
    return pack_loc(tx, ty, mulhi_u64_u32(d2, d));
}

// A map lineage's next dispersal reads one entry of its cell's alias row.
// Where the warp kernel has no shared-memory buffer for the row (the server,
// or a kernel too large for one), the warp prefetches the row (n_off x 8
// bytes, two lines per lane for the 797 offsets of radius 16) into its SM's
// L1 once the lineage has moved, while it searches for the next event.
// Every address lies in the row.
__device__ __forceinline__ void prefetch_alias_row(const SimParams* __restrict__ P, const LaneSim& c, uint64_t loc,
                                                   uint32_t lane) {
    const SimParams* p = P + c.sim;
    const uint32_t bytes = __ldg(&p->n_off) * 8u;
    const char* row = (const char*)(p->alias + ((size_t)loc_y(loc) * c.W + loc_x(loc)) * __ldg(&p->n_off));
    for (uint32_t o = lane * 128u; o < bytes; o += 32u * 128u) asm volatile("prefetch.global.L1 [%0];" ::"l"(row + o));
}

// The warp kernel's alternative: one bulk copy (TMA, cp.async.bulk) brings
// the row into the warp's shared-memory buffer while the search runs.  Lane
// 0 issues it from the 16-byte boundary at or below the row's start (the
// allocation has two entries of padding after the last row), with an
// mbarrier that counts the bytes in; the dispersal waits on that barrier.
// The warp's buffer starts with its 16-byte barrier slot, then the row.
constexpr uint32_t ROW_BAR_BYTES = 16;
constexpr uint32_t ROW_WAIT_LIMIT = 1u << 24;  // try_wait rounds before a wait gives up (error bit 16)

struct RowStage {
    uint32_t bar;      // shared address of the warp's mbarrier
    uint32_t data;     // shared address of the row buffer (16-byte aligned)
    uint32_t issued;   // copies issued so far (the last one completes phase issued - 1)
    bool pending;      // a copy is issued and not yet waited for
};

__device__ __forceinline__ RowStage row_stage_init(unsigned char* warp_buf, uint32_t lane) {
    RowStage r;
    r.bar = (uint32_t)__cvta_generic_to_shared(warp_buf);
    r.data = r.bar + ROW_BAR_BYTES;
    r.issued = 0;
    r.pending = false;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(r.bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    return r;
}

// every lane waits until the last issued copy has landed (bounded; on the
// limit the device error bit 16 is set and the row is not used for results:
// the run fails)
__device__ __forceinline__ void row_stage_wait(RowStage& r, const BatchDev& B) {
    if (!r.pending) return;
    const uint32_t parity = (r.issued - 1u) & 1u;
    uint32_t done = 0;
    // the copy was issued a whole search earlier: it has almost always landed
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done)
                 : "r"(r.bar), "r"(parity)
                 : "memory");
    for (uint32_t it = 0; it < ROW_WAIT_LIMIT && !done; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(r.bar), "r"(parity)
                     : "memory");
    if (!done) atomicOr(&B.G->error, 16u);
    r.pending = false;
    __syncwarp();
}

// the wait split in two, so that its first probe overlaps the event's
// Philox block: poll issues one try_wait and returns its answer; finish
// acts on it only when the row is needed (bounded further probes if the
// copy is still in flight)
__device__ __forceinline__ uint32_t row_stage_poll(const RowStage& r) {
    if (!r.pending) return 1u;
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done)
                 : "r"(r.bar), "r"((r.issued - 1u) & 1u)
                 : "memory");
    return done;
}

__device__ __forceinline__ void row_stage_finish(RowStage& r, const BatchDev& B, uint32_t done) {
    if (!r.pending) return;
    const uint32_t parity = (r.issued - 1u) & 1u;
    for (uint32_t it = 0; it < ROW_WAIT_LIMIT && !done; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(r.bar), "r"(parity)
                     : "memory");
    if (!done) atomicOr(&B.G->error, 16u);
    r.pending = false;
    __syncwarp();
}

// stage the alias row of loc's cell; returns the buffer address of entry 0
__device__ __forceinline__ const uint64_t* row_stage_issue(RowStage& r, unsigned char* warp_buf,
                                                           const SimParams* __restrict__ P, const LaneSim& c,
                                                           uint64_t loc, uint32_t lane, const BatchDev& B) {
    row_stage_wait(r, B);  // a copy still in flight lands before the buffer is written again
    const uint32_t n_off = c.n_off;
    const uint64_t* row = c.alias + ((size_t)loc_y(loc) * c.W + loc_x(loc)) * n_off;
    const uintptr_t a = (uintptr_t)row;
    const uint32_t lead = (uint32_t)(a & 15u);  // 0 or 8
    const uint32_t bytes = (lead + n_off * 8u + 15u) & ~15u;
    __syncwarp();  // every lane has read the previous row
    // lane 0 issues, predicated rather than branched, so that the warp does
    // not diverge and the issue can overlap the search that follows
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.eq.u32 p, %0, 0;\n\t"
        "@p fence.proxy.async.shared::cta;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%1], %2;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%3], [%4], %2, [%1];\n\t"
        "}" ::"r"(lane),
        "r"(r.bar), "r"(bytes), "r"(r.data), "l"(a & ~(uintptr_t)15)
        : "memory");
    r.issued += 1u;
    r.pending = true;
    return (const uint64_t*)(warp_buf + ROW_BAR_BYTES + lead);
}

// speciation threshold at loc: the metacommunity's in the spatially
// implicit model, else the simulation's
__device__ __forceinline__ uint64_t spec_thr(const LaneSim& c, const SimParams* __restrict__ P, int kind,
                                             uint64_t loc) {
    return (kind == KIND_IMPLICIT && in_meta(loc)) ? c.meta_nu_thr : c.nu_thr;
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

// The event's draws for one lineage per warp: lanes of even and odd index
// compute the event stream's blocks 0 and 1 side by side, then every lane
// takes the four draws by shuffle (one block's latency instead of two
// interleaved).  spec: the lineage speciates.  The caller computes the move
// from the draws whether or not it speciates and keeps it only if not, so
// that no branch on the speciation test sits on the event chain.
struct EventDraws {
    uint64_t d1, d2, d3;
    bool spec;
};

template <int KIND>
__device__ __forceinline__ EventDraws event_draws_warp(const LaneSim& c, const SimParams* __restrict__ P,
                                                       uint64_t loc, double tau, uint32_t lane) {
    const int kind = KIND >= 0 ? KIND : c.kind;
    const uint64_t tk = (uint64_t)__double_as_longlong(tau);
    EventDraws e;
    if (kind == KIND_NONSPATIAL) {
        const u64x2 b0 = stream_block(c.sk0, c.sk1, loc, tk, 0, TAG_EVENT);
        e.spec = (b0.lo >> 11) < c.nu_thr;
        e.d1 = b0.hi;
        e.d2 = e.d3 = 0ull;
        return e;
    }
    const u64x2 b = stream_block(c.sk0, c.sk1, loc, tk, lane & 1u, TAG_EVENT);
    const uint64_t d0 = __shfl_sync(0xFFFFFFFFu, b.lo, 0);
    e.d1 = __shfl_sync(0xFFFFFFFFu, b.hi, 0);
    e.d2 = __shfl_sync(0xFFFFFFFFu, b.lo, 1);
    e.d3 = __shfl_sync(0xFFFFFFFFu, b.hi, 1);
    e.spec = (d0 >> 11) < spec_thr(c, P, kind, loc);
    return e;
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
    if (B.count_unique) {
        const unsigned act = __activemask();
        const unsigned same = __match_any_sync(act, skey);
        const bool shadowed = (same & ((1u << (threadIdx.x & 31u)) - 1u)) != 0u;
        atomicAdd(&B.G->ins_total, 1ull);
        if (shadowed) atomicAdd(&B.G->ins_warp_repeat, 1ull);
    }
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
            if (B.count_unique) atomicAdd(&B.G->ins_repeat, 1ull);
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
