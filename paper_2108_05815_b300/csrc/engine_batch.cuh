// engine_batch.cuh -- host side of a batch: parameters, buffers, rounds, CUDA graphs, species and event stream.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

// ---------------------------------------------------------------------------
// host objects
// ---------------------------------------------------------------------------
struct Batch;

// Pinned host copies of the device globals, reused across batches: a
// cudaMallocHost costs about half a millisecond, as much as a short
// simulation's whole setup.  Kept until the process ends.
static std::mutex g_pinned_mu;
static std::vector<Globals*> g_pinned_free;

static Globals* pinned_globals_get() {
    {
        std::lock_guard<std::mutex> lk(g_pinned_mu);
        if (!g_pinned_free.empty()) {
            Globals* p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    Globals* p = nullptr;
    return cudaMallocHost(&p, sizeof(Globals)) == cudaSuccess ? p : nullptr;
}

static void pinned_globals_put(Globals* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned_free.push_back(p);
}

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
    size_t coop_smem = 0;                            // its dynamic shared memory (tables, alias-row buffers)
    uint32_t coop_blocks = 0;                        // its grid: one wave of resident blocks
    uint32_t lane_blocks = 0;                        // the one-lane kernels' grid: one wave of resident blocks
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
        pinned_globals_put(h_g);
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
    // indexed locations of the water level's occupancy term: the
    // metacommunity's too in the spatially implicit model, where lineages
    // that migrated rarely meet (with the local community alone the tail
    // ran 339 short rounds instead of 19)
    p.n_slots = (double)slot_span(m);
}

// dynamic shared memory a block may use, less what the kernel declares statically
static size_t coop_smem_limit() {
    static size_t lim = 0;
    if (!lim) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, k_advance_coop<false, 0, -1, false>) == cudaSuccess && optin > 0)
            lim = (size_t)optin - fa.sharedSizeBytes;
        else
            lim = LN_SMEM_BYTES;
    }
    return lim;
}

template <bool COUNT, int MODE, int KIND, bool LOG>
static cudaError_t set_smem_one() {
    return cudaFuncSetAttribute(k_advance_coop<COUNT, MODE, KIND, LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max(coop_smem_limit(), LN_SMEM_BYTES));
}

// the instantiations launch_coop uses: with counting (measurement runs) only
// the generic kind
template <bool COUNT, bool LOG>
static cudaError_t set_coop_smem() {
    cudaError_t e;
    if ((e = set_smem_one<COUNT, 0, -1, LOG>()) || (e = set_smem_one<COUNT, 1, -1, LOG>()) ||
        (e = set_smem_one<COUNT, 2, -1, LOG>()))
        return e;
    if (!COUNT) {
        if ((e = set_smem_one<COUNT, 1, 0, LOG>()) || (e = set_smem_one<COUNT, 1, 1, LOG>()) ||
            (e = set_smem_one<COUNT, 1, 2, LOG>()) || (e = set_smem_one<COUNT, 2, 0, LOG>()) ||
            (e = set_smem_one<COUNT, 2, 1, LOG>()) || (e = set_smem_one<COUNT, 2, 2, LOG>()))
            return e;
    }
    return cudaSuccess;
}

// the warp kernel's list of heavy lineages in rounds of the one-lane form:
// at most one lineage per warp of its grid (more would run one after another
// on a warp, after the one-lane kernel), none for the convergent one-lane
// form, which reads only the main list
constexpr uint32_t HEAVY_LIST_MAX = 16384;

static uint32_t heavy_list_cap(const Batch& b) {
    if (!b.dev.heavy || b.tun.advance_variant != 1) return 0;
    return std::min<uint32_t>(b.coop_blocks * (b.adv_threads / 32u), HEAVY_LIST_MAX);
}

// blocks of the warp kernel an SM holds at once (the fewest over its
// instantiations), for a block of `threads` with `smem` dynamic bytes
static uint32_t coop_blocks_per_sm(uint32_t threads, size_t smem) {
    const void* fns[] = {
        (const void*)k_advance_coop<false, 0, -1, false>, (const void*)k_advance_coop<false, 1, -1, false>,
        (const void*)k_advance_coop<false, 2, -1, false>, (const void*)k_advance_coop<false, 1, 0, false>,
        (const void*)k_advance_coop<false, 1, 1, false>, (const void*)k_advance_coop<false, 1, 2, false>,
        (const void*)k_advance_coop<false, 2, 0, false>, (const void*)k_advance_coop<false, 2, 1, false>,
        (const void*)k_advance_coop<false, 2, 2, false>, (const void*)k_advance_coop<true, 0, -1, false>,
        (const void*)k_advance_coop<true, 1, -1, false>, (const void*)k_advance_coop<true, 2, -1, false>,
        (const void*)k_advance_coop<false, 0, -1, true>, (const void*)k_advance_coop<false, 1, -1, true>,
        (const void*)k_advance_coop<false, 2, -1, true>, (const void*)k_advance_coop<false, 1, 0, true>,
        (const void*)k_advance_coop<false, 1, 1, true>, (const void*)k_advance_coop<false, 1, 2, true>,
        (const void*)k_advance_coop<false, 2, 0, true>, (const void*)k_advance_coop<false, 2, 1, true>,
        (const void*)k_advance_coop<false, 2, 2, true>, (const void*)k_advance_coop<true, 0, -1, true>,
        (const void*)k_advance_coop<true, 1, -1, true>, (const void*)k_advance_coop<true, 2, -1, true>};
    int best = 0;
    for (const void* f : fns) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, (int)threads, smem) != cudaSuccess) nb = 1;
        best = best == 0 ? nb : std::min(best, nb);
    }
    return (uint32_t)std::max(best, 1);
}

// blocks of the one-lane kernels an SM holds at once (the fewest over them)
static uint32_t lane_blocks_per_sm(uint32_t threads, size_t smem) {
    const void* fns[] = {(const void*)k_advance<false, 1, false>, (const void*)k_advance<true, 1, false>,
                         (const void*)k_advance<false, 1, true>, (const void*)k_advance<true, 1, true>,
                         (const void*)k_advance_sm<false>, (const void*)k_advance_sm<true>};
    int best = 0;
    for (const void* f : fns) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, (int)threads, smem) != cudaSuccess) nb = 1;
        best = best == 0 ? nb : std::min(best, nb);
    }
    return (uint32_t)std::max(best, 1);
}

template <bool COUNT, int MODE, bool LOG>
static void launch_coop_kind(const Batch& b, size_t smem, cudaStream_t s) {
    const dim3 g(b.coop_blocks), t(b.adv_threads);
    if (COUNT || b.coop_kind < 0 || b.coop_kind > KIND_MAP)  // counting runs and mixed or implicit batches
        k_advance_coop<COUNT, MODE, -1, LOG><<<g, t, smem, s>>>(b.dev);
    else if (b.coop_kind == KIND_NONSPATIAL)
        k_advance_coop<COUNT, MODE, (COUNT ? -1 : 0), LOG><<<g, t, smem, s>>>(b.dev);
    else if (b.coop_kind == KIND_TORUS)
        k_advance_coop<COUNT, MODE, (COUNT ? -1 : 1), LOG><<<g, t, smem, s>>>(b.dev);
    else
        k_advance_coop<COUNT, MODE, (COUNT ? -1 : 2), LOG><<<g, t, smem, s>>>(b.dev);
}

template <bool COUNT, bool LOG>
static void launch_coop(const Batch& b, size_t smem, cudaStream_t s) {
    if (b.coop_mode == 1) launch_coop_kind<COUNT, 1, LOG>(b, smem, s);
    else if (b.coop_mode == 2) launch_coop_kind<COUNT, 2, LOG>(b, smem, s);
    else k_advance_coop<COUNT, 0, -1, LOG><<<b.coop_blocks, b.adv_threads, smem, s>>>(b.dev);
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
    d.work = P.get<uint32_t>(n);
    d.heavy = P.get<uint32_t>(HEAVY_LIST_MAX);
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
    // event log: every simulation of the batch has one, or none does; one
    // shared record of their summed capacities
    uint64_t log_cap = 0;
    uint32_t logged = 0;
    for (auto* m : b.sims) {
        log_cap += m->log_cap;
        logged += m->log_cap ? 1u : 0u;
    }
    if (logged && (logged != b.n_sims || log_cap > (1ull << 31))) return IND_ERR_ARG;
    if (log_cap) {
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
    if (!b.d_params || !b.d_state || !b.d_g || !b.d_gid_base || !d.parent || !d.work || !d.key_loc || !d.key_time)
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
    // map simulations: the warp kernel stages each lineage's alias row in
    // shared memory (one buffer per warp) while it searches for the next
    // event, when buffers for the largest dispersal kernel fit beside the
    // logarithm tables
    uint32_t n_off_max = 0;
    for (auto* m : b.sims)
        if (m->land.kind == IND_MAP) n_off_max = std::max(n_off_max, m->n_off);
    const size_t ln_bytes = d.need_ln ? LN_SMEM_BYTES : 0;
    // Poisson points: when every simulation draws them from the same
    // tables (the same lambda dt), the warp kernel reads the guide and the
    // thresholds from shared memory; the guide lookup is on the chain of
    // every event
    size_t pois_bytes = 0;
    d.pois_guide = nullptr;
    d.pois_cdf = nullptr;
    d.pois_n = 0;
    d.pois_off = (uint32_t)ln_bytes;
    {
        const ind_sim* first = nullptr;
        bool same = true;
        for (auto* m : b.sims) {
            if (m->land.event_sampler != IND_SAMPLER_POISSON) continue;
            if (!first) first = m;
            else if (m->land.lambda * m->land.delta_t != first->land.lambda * first->land.delta_t ||
                     m->pois_n != first->pois_n)
                same = false;
        }
        if (first && same) {
            d.pois_guide = first->d_pois_guide;
            d.pois_cdf = first->d_pois;
            d.pois_n = first->pois_n;
            pois_bytes = sizeof(uint32_t) * GUIDE_N + (((size_t)first->pois_n * 8 + 15) & ~(size_t)15);
        }
    }
    // likewise the torus's discretised-normal guide and thresholds when every
    // torus simulation has the same sigma (its guide lookups are on the
    // chain of every dispersal)
    size_t gauss_bytes = 0;
    d.gauss_guide = nullptr;
    d.gauss_cdf = nullptr;
    d.gauss_n = 0;
    d.gauss_off = (uint32_t)(ln_bytes + pois_bytes);
    {
        const ind_sim* first = nullptr;
        bool same = true;
        for (auto* m : b.sims) {
            if (m->land.kind != IND_TORUS) continue;
            if (!first) first = m;
            else if (m->disp.sigma != first->disp.sigma || m->gauss_n != first->gauss_n) same = false;
        }
        if (first && same) {
            d.gauss_guide = first->d_gauss_guide;
            d.gauss_cdf = first->d_gauss;
            d.gauss_n = first->gauss_n;
            gauss_bytes = sizeof(uint32_t) * GUIDE_N + (((size_t)first->gauss_n * 8 + 15) & ~(size_t)15);
        }
    }
    // and the map's offset table when every map simulation has the same
    // kernel radius (the same number of offsets)
    size_t off_bytes = 0;
    d.off_tab = nullptr;
    d.off_n = 0;
    d.off_off = (uint32_t)(ln_bytes + pois_bytes + gauss_bytes);
    {
        const ind_sim* first = nullptr;
        bool same = true;
        for (auto* m : b.sims) {
            if (m->land.kind != IND_MAP) continue;
            if (!first) first = m;
            else if (m->n_off != first->n_off) same = false;
        }
        if (first && same) {
            d.off_tab = first->d_off;
            d.off_n = first->n_off;
            off_bytes = ((size_t)first->n_off * 2 + 15) & ~(size_t)15;
        }
    }
    b.coop_smem = ln_bytes + pois_bytes + gauss_bytes + off_bytes;
    d.stage_off = d.stage_bytes = 0;
    if (n_off_max) {
        // the warp's mbarrier slot, then a row copied from a 16-byte boundary
        const size_t per = ROW_BAR_BYTES + (((size_t)n_off_max * 8 + 8 + 15) & ~(size_t)15);
        const size_t total = b.coop_smem + (size_t)(b.tun.block_threads / 32) * per;
        if (total <= coop_smem_limit()) {
            d.stage_off = (uint32_t)b.coop_smem;
            d.stage_bytes = (uint32_t)per;
            b.coop_smem = total;
        }
    }
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
    b.h_g = pinned_globals_get();
    if (!b.h_g) return IND_ERR_OOM;
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
        CK((set_coop_smem<true, true>()));
        CK((set_coop_smem<false, true>()));
    }
    CK((set_coop_smem<true, false>()));
    CK((set_coop_smem<false, false>()));
    CK(cudaFuncSetAttribute(k_advance_sm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES));
    CK(cudaFuncSetAttribute(k_advance_sm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LN_SMEM_BYTES));
    b.adv_threads = b.tun.block_threads;
    b.adv_blocks = sms * b.tun.blocks_per_sm;
    b.coop_blocks = std::min(b.adv_blocks, sms * coop_blocks_per_sm(b.adv_threads, b.coop_smem));
    b.lane_blocks = std::min(b.adv_blocks, sms * lane_blocks_per_sm(b.adv_threads, LN_SMEM_BYTES));
    b.cmp_blocks = sms * 4;
    d.heavy_cap = heavy_list_cap(b);
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

constexpr uint64_t LAUNCHES_PER_ROUND = 4;  // work-list filter, one-lane and warp-per-lineage advance, compaction

static ind_status launch_round(Batch& b, uint32_t r, bool capturing) {
    cudaStream_t s = capturing ? b.cap_stream : b.stream;
    const bool prof = b.tun.profile && r < b.ev_start.size();
    const unsigned flag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (prof) CK(cudaEventRecordWithFlags(b.ev_start[r], s, flag));
    k_filter<<<b.cmp_blocks, 256, 0, s>>>(b.dev);
    CK(cudaGetLastError());
    // shared memory only when some simulation sums exponentials (leaves L1 larger otherwise)
    const size_t smem = b.dev.need_ln ? LN_SMEM_BYTES : 0;
    const bool conv = b.tun.advance_variant == 0;  // convergent state machine or one-lane loop
    // both advance forms every round: each reads the live lineage count and
    // returns at once unless the round is its own (more than coop_lineages
    // lineages: one lane per lineage; else one warp per lineage), so that the
    // choice is made per round inside captured chunks.  An event log takes
    // the logging forms (one-lane loop; the warp form as specialised as
    // without a log).
    const dim3 ag(b.lane_blocks), at(b.adv_threads);
    if (b.dev.log.cap) {
        if (b.dev.count_unique) {
            k_advance<true, 1, true><<<ag, at, smem, s>>>(b.dev);
            CK(cudaGetLastError());
            launch_coop<true, true>(b, b.coop_smem, s);
        } else {
            k_advance<false, 1, true><<<ag, at, smem, s>>>(b.dev);
            CK(cudaGetLastError());
            launch_coop<false, true>(b, b.coop_smem, s);
        }
    } else if (b.dev.count_unique) {
        if (conv) k_advance_sm<true><<<ag, at, smem, s>>>(b.dev);
        else k_advance<true, 1, false><<<ag, at, smem, s>>>(b.dev);
        CK(cudaGetLastError());
        launch_coop<true, false>(b, b.coop_smem, s);
    } else {
        if (conv) k_advance_sm<false><<<ag, at, smem, s>>>(b.dev);
        else k_advance<false, 1, false><<<ag, at, smem, s>>>(b.dev);
        CK(cudaGetLastError());
        launch_coop<false, false>(b, b.coop_smem, s);
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

// the logged run's record -> the distinct events and the coalescences of
// every simulation of the batch
static ind_status process_event_log(Batch& b) {
    cudaStream_t s = b.stream;
    Pool& T = b.scratch;
    const uint32_t sms = sm_count();
    for (auto* m : b.sims) {
        m->events.release_all();
        m->events.stream = m->stream;
        m->d_events = nullptr;
        m->d_coal = nullptr;
        m->n_events = m->n_coal = 0;
        m->events_ready = false;
    }
    unsigned long long n_log = 0;
    CK(cudaMemcpyAsync(&n_log, &b.d_g->log_n, sizeof(n_log), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (n_log > b.dev.log.cap) return IND_ERR_DEVICE;
    const uint32_t n = (uint32_t)n_log;
    const bool multi = b.n_sims > 1;
    if (n) {
        // the log's order by stable radix passes, least significant field
        // first (lineage, prior time, location, time, and the simulation in
        // a batch of several); bytes that are equal in every entry are skipped
        const uint32_t nb = (n + RS_TILE - 1) / RS_TILE;
        uint64_t* key0 = T.get<uint64_t>(n);
        uint64_t* key1 = T.get<uint64_t>(n);
        uint32_t* val0 = T.get<uint32_t>(n);
        uint32_t* val1 = T.get<uint32_t>(n);
        uint32_t* counts = T.get<uint32_t>((size_t)RS_RADIX * nb);
        uint32_t* offs = T.get<uint32_t>((size_t)RS_RADIX * nb);
        unsigned long long* d_bits = T.get<unsigned long long>(8);
        SortItem* items = T.get<SortItem>(n);
        uint32_t* head = T.get<uint32_t>(n);
        uint32_t* coal = T.get<uint32_t>(n);
        uint32_t* incl_head = T.get<uint32_t>(n);
        uint32_t* incl_coal = T.get<uint32_t>(n);
        uint32_t* lsim = multi ? T.get<uint32_t>(n) : nullptr;  // each log entry's simulation
        uint32_t* isim = multi ? T.get<uint32_t>(n) : nullptr;  // each sorted item's simulation
        if (!key0 || !key1 || !val0 || !val1 || !counts || !offs || !d_bits || !items || !head || !coal ||
            !incl_head || !incl_coal || (multi && (!lsim || !isim)))
            return IND_ERR_OOM;
        unsigned long long h_bits[8];
        for (int f = 0; f < 4; ++f) {
            h_bits[2 * f] = ~0ull;
            h_bits[2 * f + 1] = 0ull;
        }
        CK(cudaMemcpyAsync(d_bits, h_bits, sizeof(h_bits), cudaMemcpyHostToDevice, s));
        k_ev_bits<<<grid_for(n, 256, sms * 8), 256, 0, s>>>(b.dev.log, n, d_bits);
        CKL();
        CK(cudaMemcpyAsync(h_bits, d_bits, sizeof(h_bits), cudaMemcpyDeviceToHost, s));
        k_iota<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(val0, n);
        CKL();
        if (multi) {
            k_ev_sim<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(b.dev.log, n, b.d_gid_base, b.n_sims, lsim);
            CKL();
        }
        CK(cudaStreamSynchronize(s));
        ind_status st = IND_OK;
        auto radix_passes = [&](uint64_t varies) -> ind_status {
            for (int shift = 0; shift < 64; shift += 8) {
                if (!((varies >> shift) & 0xFFull)) continue;
                k_rs_count<<<nb, RS_WARPS * 32, 0, s>>>(key0, n, shift, counts);
                CKL();
                ind_status rs = scan_u32(T, counts, offs, RS_RADIX * nb, false, s);
                if (rs != IND_OK) return rs;
                k_rs_scatter<<<nb, RS_WARPS * 32, 0, s>>>(key0, val0, n, shift, offs, key1, val1);
                CKL();
                std::swap(key0, key1);
                std::swap(val0, val1);
            }
            return IND_OK;
        };
        for (int f = 0; f < 4; ++f) {
            const uint64_t varies = h_bits[2 * f] ^ h_bits[2 * f + 1];
            if (!varies) continue;
            k_ev_field<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(b.dev.log, f, val0, n, key0);
            CKL();
            if ((st = radix_passes(varies)) != IND_OK) return st;
        }
        if (multi) {
            k_ev_key_u32<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(lsim, val0, n, key0);
            CKL();
            uint64_t varies = 0;
            for (uint32_t v = b.n_sims - 1u; v; v >>= 1) varies = (varies << 1) | 1ull;
            if ((st = radix_passes(varies)) != IND_OK) return st;
        }
        k_ev_gather<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(b.dev.log, val0, n, items, lsim, isim);
        CKL();
        k_ev_marks<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, isim, head, coal);
        CKL();
        if ((st = scan_u32(T, head, incl_head, n, true, s)) != IND_OK) return st;
        if ((st = scan_u32(T, coal, incl_coal, n, true, s)) != IND_OK) return st;
        uint32_t hn = 0, cn = 0;
        CK(cudaMemcpyAsync(&hn, incl_head + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&cn, incl_coal + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // one simulation: straight into its buffers; several: into shared
        // buffers in (simulation, time, location) order, then each
        // simulation's range into its own
        ind_sim* m0 = b.sims[0];
        ind_event* ev_all = multi ? T.get<ind_event>(std::max<uint32_t>(hn, 1u))
                                  : (m0->d_events = m0->events.get<ind_event>(std::max<uint32_t>(hn, 1u)));
        ind_coalescence* co_all = multi ? T.get<ind_coalescence>(std::max<uint32_t>(cn, 1u))
                                        : (m0->d_coal = m0->events.get<ind_coalescence>(std::max<uint32_t>(cn, 1u)));
        uint32_t* head_pos = T.get<uint32_t>(std::max<uint32_t>(hn, 1u));
        if (!ev_all || !co_all || !head_pos) return IND_ERR_OOM;
        k_ev_events<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, head, incl_head, b.dev.log.target, head_pos,
                                                               ev_all, isim, b.d_gid_base);
        CKL();
        k_ev_targets<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, incl_head, b.dev.log.target, ev_all);
        CKL();
        k_ev_coalescences<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(items, n, coal, incl_coal, incl_head, head_pos,
                                                                     co_all, isim, b.d_gid_base);
        CKL();
        if (!multi) {
            CK(cudaStreamSynchronize(s));
            m0->n_events = hn;
            m0->n_coal = cn;
        } else {
            uint32_t* ev_cnt = T.get<uint32_t>(b.n_sims);
            uint32_t* co_cnt = T.get<uint32_t>(b.n_sims);
            if (!ev_cnt || !co_cnt) return IND_ERR_OOM;
            CK(cudaMemsetAsync(ev_cnt, 0, sizeof(uint32_t) * b.n_sims, s));
            CK(cudaMemsetAsync(co_cnt, 0, sizeof(uint32_t) * b.n_sims, s));
            k_ev_sim_counts<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(head, coal, isim, n, ev_cnt, co_cnt);
            CKL();
            std::vector<uint32_t> he(b.n_sims), hc(b.n_sims);
            CK(cudaMemcpyAsync(he.data(), ev_cnt, sizeof(uint32_t) * b.n_sims, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(hc.data(), co_cnt, sizeof(uint32_t) * b.n_sims, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            uint64_t eo = 0, co = 0;
            for (uint32_t si = 0; si < b.n_sims; ++si) {
                ind_sim* m = b.sims[si];
                m->d_events = m->events.get<ind_event>(std::max<uint32_t>(he[si], 1u));
                m->d_coal = m->events.get<ind_coalescence>(std::max<uint32_t>(hc[si], 1u));
                if (!m->d_events || !m->d_coal) return IND_ERR_OOM;
                if (he[si])
                    CK(cudaMemcpyAsync(m->d_events, ev_all + eo, sizeof(ind_event) * he[si], cudaMemcpyDeviceToDevice, s));
                if (hc[si])
                    CK(cudaMemcpyAsync(m->d_coal, co_all + co, sizeof(ind_coalescence) * hc[si],
                                       cudaMemcpyDeviceToDevice, s));
                m->n_events = he[si];
                m->n_coal = hc[si];
                eo += he[si];
                co += hc[si];
            }
            CK(cudaStreamSynchronize(s));
        }
    }
    for (auto* m : b.sims) m->events_ready = true;
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
        m->stats.dedup_inserts = b.h_g_valid ? b.h_g->ins_total : 0;
        m->stats.dedup_repeats = b.h_g_valid ? b.h_g->ins_repeat : 0;
        m->stats.dedup_warp_repeats = b.h_g_valid ? b.h_g->ins_warp_repeat : 0;
    }
    return result;
}
