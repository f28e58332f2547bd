// engine_advance.cuh -- the round kernels: lineage start, the advance forms, compaction and horizons.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

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

// a lineage with at least this many events (expected) before its horizon
// runs in the warp kernel in a round of the one-lane form
constexpr double HEAVY_EVENTS = 256.0;

// The round's work list: the lineages whose next event lies before their
// simulation's horizon (warp-aggregated appends).  The others have nothing
// to do in the round: no event, no state to write, no dedup entry.
// In a round of the one-lane form, a lineage of a simulation in its tail
// (HEAVY_EVENTS or more before the horizon) goes on the warp kernel's list
// instead, while it has room: one lane would run those events one after
// another at about twice the warp's time per event, and the round would
// last as long as that chain.
__global__ void k_filter(BatchDev B) {
    const uint32_t n = B.G->n_total;
    const LinPtrs L = B.lin[B.G->round & 1u];
    const uint32_t lane = threadIdx.x & 31u;
    const bool split = B.heavy_cap && n > B.coop_lineages;
    const uint32_t stride = gridDim.x * blockDim.x;  // a multiple of 32: warps stay whole
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += stride) {
        const uint32_t i = base + lane;
        bool due = false, heavy = false;
        if (i < n) {
            const uint32_t si = L.sim[i];
            const double h = B.S[si].horizon;
            const double tn = L.tn[i];
            due = (uint64_t)__double_as_longlong(tn) <= (uint64_t)__double_as_longlong(h);
            heavy = split && due && (h - tn) * B.P[si].lambda >= HEAVY_EVENTS;
        }
        const unsigned mh = __ballot_sync(0xFFFFFFFFu, heavy);
        if (mh) {
            uint32_t h0 = 0;
            if (lane == 0) h0 = atomicAdd(&B.G->n_heavy, (uint32_t)__popc(mh));
            h0 = __shfl_sync(0xFFFFFFFFu, h0, 0);
            if (heavy) {
                const uint32_t pos = h0 + __popc(mh & ((1u << lane) - 1u));
                if (pos < B.heavy_cap) {
                    B.heavy[pos] = i;
                    due = false;  // listed for the warp kernel
                }
            }
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, due);
        uint32_t p0 = 0;
        if (lane == 0 && m) p0 = atomicAdd(&B.G->n_work, (uint32_t)__popc(m));
        p0 = __shfl_sync(0xFFFFFFFFu, p0, 0);
        if (due) B.work[p0 + __popc(m & ((1u << lane) - 1u))] = i;
    }
}

// LOG: append every executed event to the event log
template <bool COUNT, int WIDE, bool LOG>
__global__ void __launch_bounds__(512) k_advance(BatchDev B) {
    extern __shared__ __align__(16) unsigned char adv_smem[];
    if (B.G->n_total <= B.coop_lineages) return;  // a round for k_advance_coop
    // lineages with an event before the horizon (k_filter); those listed for
    // the warp kernel too when more were listed than its list holds (the
    // warp kernel then leaves them all here)
    const uint32_t n_list = B.G->n_work;
    const uint32_t n = n_list + (B.heavy_cap && B.G->n_heavy > B.heavy_cap ? B.heavy_cap : 0u);
    const uint32_t chunk = 32u * B.lpl;
    // Warps take part in the order warp 0 of every block, then warp 1, ...
    // (the grid is one wave of resident blocks): a round with few lineages
    // spreads its warps over the SMs.  Claims go out in order of arrival, at
    // most one chunk per warp at a time, so a warp whose first possible claim
    // lies beyond the work list has nothing to do.
    const uint32_t wg = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    if ((uint64_t)blockIdx.x * chunk >= n) return;
    // the logarithm tables are staged only if some simulation sums exponentials
    const LnC ln = B.need_ln ? ln_tables_shared(adv_smem) : ln_tables();
    if ((uint64_t)wg * chunk >= n) return;  // after the block's table copy

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
                    const uint32_t j = chunk_next + rank;
                    idx = j < n_list ? B.work[j] : B.heavy[j - n_list];
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
                // at the horizon: a lineage that moved this round writes its
                // state back and enters the dedup (see k_compact)
                if (ev_lin) {
                    L.loc[idx] = loc;
                    L.tn[idx] = tn;
                    if (LOG) L.tp[idx] = tprev;
                    if (B.dedup) dedup_insert(B, t, slot_key(B.P, c, loc), gid);
                }
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
    if (B.G->n_total <= B.coop_lineages) return;  // a round for k_advance_coop
    const uint32_t n = B.G->n_work;              // lineages with an event before the horizon (k_filter)
    const uint32_t chunk = 32u * B.lpl;
    const uint32_t wg = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;  // order of taking part, as k_advance
    if ((uint64_t)blockIdx.x * chunk >= n) return;
    const LnC ln = B.need_ln ? ln_tables_shared(adv_smem) : ln_tables();
    if ((uint64_t)wg * chunk >= n) return;
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
                    idx = B.work[chunk_next + rank];
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
                        // already at the horizon: nothing to write, no dedup entry (see k_compact)
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
__global__ void __launch_bounds__(512, 1) k_advance_coop(BatchDev B) {
    extern __shared__ __align__(16) unsigned char adv_smem[];
    // a round of the warp form: every lineage with an event before the
    // horizon (k_filter); a round of the one-lane form: the heavy lineages
    // k_filter listed, when they all fit the list
    const bool lane_round = B.G->n_total > B.coop_lineages;
    if (lane_round && (!B.heavy_cap || B.G->n_heavy > B.heavy_cap)) return;
    const uint32_t n = lane_round ? B.G->n_heavy : B.G->n_work;
    const uint32_t* const list = lane_round ? B.heavy : B.work;
    uint32_t* const claims = lane_round ? &B.G->heavy_ctr : &B.G->work_ctr;
    // Warps take part in the order warp 0 of every block, then warp 1 of
    // every block, and so on (the grid is one wave of resident blocks), so
    // that a round with few lineages spreads them over the SMs instead of
    // packing one block's warps onto one SM's four schedulers.  A block
    // whose warp 0 has no part leaves at once.
    const uint32_t wg = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    if (blockIdx.x >= n) return;
    const LnC ln = B.need_ln ? ln_tables_shared(adv_smem) : ln_tables();
    // the shared Poisson tables, if every simulation has the same
    // and the torus's dispersal tables, likewise
    const uint32_t* pguide = nullptr;
    const uint64_t* pcdf = nullptr;
    const uint32_t* gguide = nullptr;
    const uint64_t* gcdf = nullptr;
    const int8_t* otab = nullptr;
    if (B.pois_guide || B.gauss_guide || B.off_tab) {
        if (B.off_tab) {
            int8_t* o = (int8_t*)(adv_smem + B.off_off);
            for (uint32_t k = threadIdx.x; k < 2u * B.off_n; k += blockDim.x) o[k] = B.off_tab[k];
            otab = o;
        }
        if (B.pois_guide) {
            uint32_t* g = (uint32_t*)(adv_smem + B.pois_off);
            uint64_t* cdf = (uint64_t*)(g + GUIDE_N);
            for (uint32_t k = threadIdx.x; k < GUIDE_N; k += blockDim.x) g[k] = __ldg(B.pois_guide + k);
            for (uint32_t k = threadIdx.x; k < B.pois_n; k += blockDim.x) cdf[k] = __ldg(B.pois_cdf + k);
            pguide = g;
            pcdf = cdf;
        }
        if (B.gauss_guide) {
            uint32_t* g = (uint32_t*)(adv_smem + B.gauss_off);
            uint64_t* cdf = (uint64_t*)(g + GUIDE_N);
            for (uint32_t k = threadIdx.x; k < GUIDE_N; k += blockDim.x) g[k] = __ldg(B.gauss_guide + k);
            for (uint32_t k = threadIdx.x; k < B.gauss_n; k += blockDim.x) cdf[k] = __ldg(B.gauss_cdf + k);
            gguide = g;
            gcdf = cdf;
        }
        __syncthreads();
    }
    if (wg >= n) return;  // after the block's table copies
    const uint32_t t = B.G->round & 1u;
    const LinPtrs L = B.lin[t];
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t ev_raw = 0, ev_unique = 0;
    uint32_t cnt_sim = 0xFFFFFFFFu;
    uint32_t lane_max = 0;  // most events of one lineage this round (the same in every lane)
    WarpLogBuf wlog;
    wlog.n = 0;
    // this warp's alias-row buffer (map lineages; after the tables): its
    // mbarrier, then the row
    unsigned char* const sbuf = adv_smem + B.stage_off + (size_t)(threadIdx.x >> 5) * B.stage_bytes;
    RowStage rs;
    rs.pending = false;
    if (B.stage_bytes) rs = row_stage_init(sbuf, lane);
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(claims, 1u);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= n) break;
        const uint32_t idx = list[k];
        const uint32_t gid = L.gid[idx];
        uint64_t loc = L.loc[idx];
        double tn = L.tn[idx];
        double tprev = LOG ? L.tp[idx] : 0.0;
        const uint32_t s = L.sim[idx];
        LaneSim c;
        load_lanesim(c, B.P, B.S, s);
        if (pguide) {
            c.pois_guide = pguide;
            c.pois_cdf = pcdf;
        }
        if (gguide && c.kind == KIND_TORUS) {
            c.gauss_guide = gguide;
            c.gauss = gcdf;
        }
        if (otab && c.kind == KIND_MAP) c.off = otab;
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
        // MODES 1 and 2: the interval index of tn, carried from search to
        // search (MODE 2 forms it as soon as the search returns, ahead of the
        // next event's draws)
        uint64_t kc = MODE == 1 || MODE == 2 ? floor_div_pow2((uint64_t)__double_as_longlong(tn), c.dt_log2) : 0ull;
        // the lineage's events, in the code specialised for its landscape kind:
        // a kernel for one kind runs that form, the general kernel chooses the
        // form once per lineage (measured on B300, the general form of the
        // event's draws and move cost about 100 cycles per event)
        auto events = [&](auto kind_tag) {
            constexpr int K = decltype(kind_tag)::value;
            // a map lineage's alias row, staged in the warp's buffer
            const bool stage = B.stage_bytes && (K == KIND_MAP || (K < 0 && c.kind == KIND_MAP));
            const uint64_t* srow = stage ? row_stage_issue(rs, sbuf, B.P, c, loc, lane, B) : nullptr;
            for (uint32_t guard = 0; guard < 0xFFFFFFFFu; ++guard) {
                // the event's draws ahead of the horizon test, so that their
                // Philox block overlaps it (a lineage at its horizon drops them)
                const uint32_t row_ready = stage ? row_stage_poll(rs) : 1u;
                const EventDraws ed = event_draws_warp<K>(c, B.P, loc, tn, lane);
                if ((uint64_t)__double_as_longlong(tn) > hz) {
                    if (lane == 0 && ev_lin) {  // moved this round (see k_compact)
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
                if (stage) row_stage_finish(rs, B, row_ready);
                const uint64_t moved = disperse<K>(c, B.P, loc, ed.d1, ed.d2, ed.d3, srow);
                const bool speciated = ed.spec;
                loc = speciated ? loc : moved;
                if (LOG) {
                    warp_log_event(B, wlog, lane, tn, tprev, at, speciated ? ~0ull : loc, gid);
                    tprev = tn;
                }
                if (!speciated && stage) srow = row_stage_issue(rs, sbuf, B.P, c, loc, lane, B);
                else if (!speciated && (K == KIND_MAP || (K < 0 && c.kind == KIND_MAP)))
                    prefetch_alias_row(B.P, c, loc, lane);
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
                    nt = coop_next_exp_int(c, loc, tn, ln, lane, kc);
                } else if (MODE == 2) {
                    nt = coop_next_poisson_short(c, loc, tn, lane, kc);
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
                if (MODE == 2) kc = floor_div_pow2((uint64_t)__double_as_longlong(tn), c.dt_log2);
            }
        };
        if constexpr (KIND >= 0) {
            events(std::integral_constant<int, KIND>());
        } else {
            if (c.kind == KIND_NONSPATIAL) events(std::integral_constant<int, KIND_NONSPATIAL>());
            else if (c.kind == KIND_TORUS) events(std::integral_constant<int, KIND_TORUS>());
            else if (c.kind == KIND_MAP) events(std::integral_constant<int, KIND_MAP>());
            else events(std::integral_constant<int, KIND_IMPLICIT>());
        }
    }
    // a row copy still in flight lands before the block's shared memory goes
    row_stage_wait(rs, B);
    if (lane == 0 && cnt_sim != 0xFFFFFFFFu) {
        atomicAdd((unsigned long long*)&B.S[cnt_sim].raw_events, (unsigned long long)ev_raw);
        if (COUNT) atomicAdd((unsigned long long*)&B.S[cnt_sim].unique_events, (unsigned long long)ev_unique);
    }
    if (lane == 0 && lane_max) atomicMax(&B.G->round_max, lane_max);
    if (LOG) warp_log_flush(B, wlog, lane);
}

// horizon step (time) of a simulation with n active lineages
// horizon step (time) of a simulation with n active lineages while `live`
// simulations share the rounds: max_step_events bounds it so that no round
// waits long on one simulation; a simulation alone is bounded 16 times
// higher (fewer rounds, nothing else waits)
constexpr double ALONE_STEP_FACTOR = 16.0;

// Relative time of one event per landscape kind in the warp kernel, for
// pacing rounds that mix kinds: measured on B300 in batches of one kind
// (128 non-spatial demes, or 128 tori, of 10^3 to 10^6 individuals), about
// 0.65 us per critical event non-spatial and 0.84 us on tori; 1.04 us on a
// 1024 x 1024 habitat map; the spatially implicit model draws like the
// non-spatial one.
__device__ __forceinline__ double kind_event_cost(int kind) {
    return kind == KIND_TORUS ? 0.84 : (kind == KIND_MAP ? 1.04 : 0.65);
}

// the least event cost among the kinds of a mask (bit k: kind k live)
__device__ __forceinline__ double least_event_cost(uint32_t kinds) {
    double c = 1.0;
    bool any = false;
    for (int k = 0; k < 4; ++k)
        if ((kinds >> k) & 1u) {
            c = any ? fmin(c, kind_event_cost(k)) : kind_event_cost(k);
            any = true;
        }
    return c;
}

// pace: the least event cost among the live simulations' kinds over this
// simulation's own, 1 when every live simulation has one kind.  A shared
// round lasts as long as its slowest lineage's events, so a simulation of a
// costlier kind takes proportionally fewer of them: a round that mixes tori
// with non-spatial demes then lasts about as long as max_step_events
// non-spatial events instead of as many torus events.
__device__ __forceinline__ double horizon_step(const SimParams* p, uint32_t n, uint32_t live, double pace = 1.0) {
    const double dn = (double)n;
    const double floor_ev = dn < p->busy_lineages ? p->tail_events : p->min_events;
    const double per = fmax(floor_ev, fmin(p->occupancy_step * p->n_slots / dn, p->events_per_round / dn));
    const double cap = live > 1u ? p->max_step_events * pace : p->max_step_events * ALONE_STEP_FACTOR;
    return fmin(per, cap) / p->lambda;
}

// Dedup at the horizon.  Lineages that moved this round entered the round's
// table (the least lineage id of a slot wins); every active lineage looks
// its slot up.  Two lineages in one slot at a horizon are exact duplicates
// (both next events are the slot's first point after the horizon), so one
// that finds another winner is culled.  A lineage that did not move made no
// entry: it is culled if a mover entered its slot, and otherwise keeps its
// place; it has no other duplicate, because duplicates are culled in the
// round they meet.
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
    __shared__ uint32_t live, kinds;
    if (threadIdx.x == 0) {
        live = 0;
        kinds = 0;
    }
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
        atomicOr(&kinds, 1u << (B.P[s].kind & 3));
    }
    __syncthreads();
    const double cmin = least_event_cost(kinds);
    // The water level per simulation, then shared: a round lasts as long as
    // the simulation with the most events per lineage needs, so every other
    // simulation may run as many in it, up to its own occupancy bound
    // (duplicate work), at little cost.  Continuous batching gains most:
    // served requests finish sooner (526 Poisson-arrival torus requests:
    // median latency 8.9 -> 8.0 s, 99th percentile 41.5 -> 38.8 s).  A
    // simulation alone is unchanged.  Where kinds mix, the level is shared
    // in time (events x the kind's pace), each simulation taking its own
    // kind's share of it.
    __shared__ unsigned long long pmax_b;
    if (threadIdx.x == 0) pmax_b = 0ull;
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < B.n_sims; s += blockDim.x) {
        const SimState* st = B.S + s;
        if (!st->done) {
            const double pace = cmin / kind_event_cost(B.P[s].kind);
            const double per = horizon_step(B.P + s, st->n_active, live, pace) * B.P[s].lambda / pace;
            atomicMax(&pmax_b, (unsigned long long)__double_as_longlong(per));  // per >= 0: bits order as values
        }
    }
    __syncthreads();
    const double pmax = __longlong_as_double((long long)pmax_b);
    for (uint32_t s = threadIdx.x; s < B.n_sims; s += blockDim.x) {
        SimState* st = B.S + s;
        if (!st->done) {
            const SimParams* p = B.P + s;
            const double pace = cmin / kind_event_cost(p->kind);
            const double per = horizon_step(p, st->n_active, live, pace) * p->lambda;
            const double occ = p->occupancy_step * p->n_slots / fmax((double)st->n_active, 1.0);
            st->horizon = st->horizon + fmax(per, fmin(occ, pmax * pace)) / p->lambda;
        }
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
        G->n_work = 0;
        G->n_heavy = 0;
        G->heavy_ctr = 0;
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
    __shared__ uint32_t live, kinds;
    if (threadIdx.x == 0) {
        live = 0;
        kinds = 0;
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < B.n_sims; s += blockDim.x)
        if (B.P[s].n_lineages) {
            atomicAdd(&live, 1u);
            atomicOr(&kinds, 1u << (B.P[s].kind & 3));
        }
    __syncthreads();
    const double cmin = least_event_cost(kinds);
    for (uint32_t s = threadIdx.x; s < B.n_sims; s += blockDim.x) {
        const SimParams* p = B.P + s;
        SimState* st = B.S + s;
        const uint32_t na = p->n_lineages;
        st->n_active = na;
        st->done = na == 0 ? 1u : 0u;
        st->horizon = horizon_step(p, max(na, 1u), live, cmin / kind_event_cost(p->kind));
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
