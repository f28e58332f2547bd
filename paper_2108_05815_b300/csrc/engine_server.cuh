// engine_server.cuh -- the continuous-batching server: its kernels and its C ABI.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

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
    // what the warp kernel's specialisation depends on: the landscape kind,
    // and whether the request sums exponentials at lambda = 1 or draws
    // Poisson points, on the short searches
    int32_t kind = -1;
    bool exp1 = false, pois = false;
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
        sl.kind = hp.kind;
        sl.exp1 = hp.sampler == IND_SAMPLER_EXP && hp.coop_short && hp.lambda == 1.0;
        sl.pois = hp.sampler == IND_SAMPLER_POISSON && hp.coop_short;
        hp.n_lineages = n;
        hp.slot_base = (uint64_t)slot << 32;  // slots of different requests never collide
        hp.gid_base = g0;
        SimState hs;
        memset(&hs, 0, sizeof(hs));
        hs.n_active = n;
        hs.done = n == 0 ? 1u : 0u;
        {
            // first horizon step, as horizon_step() computes it on the device
            // for a simulation that shares the rounds with others of its kind
            // (later rounds pace mixed kinds on the device)
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

// The warp kernel's specialisation for the resident requests, as a batch
// chooses it for its simulations (search form and landscape kind, where all
// of them share one); a change re-captures the chunk's graph.  The form is
// chosen between chunks, so the requests of every launched chunk match the
// kernel that runs them.
static void srv_specialise(ind_server* sv) {
    Batch& b = sv->b;
    bool any = false, all_exp1 = true, all_pois = true;
    int kind = -1;
    for (const SrvSlot& sl : sv->slots) {
        if (!sl.active || sl.n == 0) continue;
        kind = !any ? sl.kind : (kind == sl.kind ? kind : -1);
        any = true;
        all_exp1 &= sl.exp1;
        all_pois &= sl.pois;
    }
    if (!any) return;  // nothing resident: the next admission decides
    const int mode = all_exp1 ? 1 : all_pois ? 2 : 0;
    if (mode == b.coop_mode && kind == b.coop_kind) return;
    b.coop_mode = mode;
    b.coop_kind = kind;
    if (b.graph) {
        cudaGraphExecDestroy(b.graph);
        b.graph = nullptr;
    }
}

extern "C" {

// The server's defaults: a higher water level for requests with many
// lineages.  A shared round lasts as long as its heaviest lineage runs (a
// request in its tail, up to max_step_events), so the requests in their busy
// phase may advance about one event per lineage per round instead of a
// quarter: on Poisson arrivals of torus requests (sides 128 to 4096, demes
// 1 to 4, sample fractions 0.01 to 1, nu 1e-7 to 1e-3) at 10 requests/s
// the median latency went from 0.92-1.07 s to 0.67 s and the 99th
// percentile from about 30 s to 27 s.
void srv_default_tuning(ind_tuning* t) {
    if (!t) return;
    ind_default_tuning(t);
    t->occupancy_step = 1.0;
    t->min_events_per_lineage = 1.0;
    t->events_per_round = 16777216.0;
}

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
    else srv_default_tuning(&b.tun);
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
    d.work = P.get<uint32_t>(n);
    d.heavy = P.get<uint32_t>(HEAVY_LIST_MAX);
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
    ok = ok && d.parent && d.work && d.key_loc && d.key_time;
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
    d.stage_off = d.stage_bytes = 0;  // alias rows of map requests are read from global memory
    d.pois_guide = nullptr;           // requests of any lambda dt: each reads its own tables
    d.pois_cdf = nullptr;
    d.pois_n = d.pois_off = 0;
    d.gauss_guide = nullptr;
    d.gauss_cdf = nullptr;
    d.gauss_n = d.gauss_off = 0;
    d.off_tab = nullptr;
    d.off_n = d.off_off = 0;
    b.coop_smem = LN_SMEM_BYTES;
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
    b.h_g = pinned_globals_get();
    if (!b.h_g) return fail(cudaErrorMemoryAllocation);
    if ((e = cudaStreamSynchronize(s))) return fail(e);
    memset(b.h_g, 0, sizeof(Globals));
    b.h_state.resize(max_sims);
    const uint32_t sms = sm_count();
    if ((e = cudaFuncSetAttribute(k_advance<false, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES)) ||
        (e = (set_coop_smem<false, false>())) ||
        (e = cudaFuncSetAttribute(k_advance_sm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES)))
        return fail(e);
    b.adv_threads = b.tun.block_threads;
    b.adv_blocks = sms * b.tun.blocks_per_sm;
    b.coop_blocks = std::min(b.adv_blocks, sms * coop_blocks_per_sm(b.adv_threads, b.coop_smem));
    b.lane_blocks = std::min(b.adv_blocks, sms * lane_blocks_per_sm(b.adv_threads, LN_SMEM_BYTES));
    b.cmp_blocks = sms * 4;
    d.heavy_cap = heavy_list_cap(b);
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
    srv_specialise(sv);
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
