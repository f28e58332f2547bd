// engine_api.cuh -- the C ABI of simulations (indep.h).
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

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
    t->coop_lineages = 16384;
    t->advance_variant = 1;
    t->rounds_per_check = 16;
    t->use_graph = 1;
    t->dedup = 1;
    t->count_unique = 0;
    t->profile = 0;
    t->events_per_round = 4194304.0;
    t->min_events_per_lineage = 0.25;
    t->occupancy_step = 0.25;
    t->tail_events = 64.0;
    t->busy_lineages = 32768.0;
    t->max_step_events = 1024.0;
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
        std::vector<uint32_t> cells;  // habitable cells: one alias row each
        for (size_t c = 0; c < ncell; ++c) {
            maxd = std::max<uint32_t>(maxd, dm[c]);
            m->n_slots += dm[c];
            if (dm[c]) cells.push_back((uint32_t)c);
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
        if (m->n_off > ALIAS_MAX_OFFSETS) return fail(IND_ERR_ARG);
        m->n_rows = (uint32_t)cells.size();
        std::vector<uint64_t> kw = host_kernel_weights(D->sigma, R);
        m->d_deme = m->tables.get<uint8_t>(ncell);
        m->d_off = m->tables.get<int8_t>(off.size());
        uint64_t* d_kw = m->tables.get<uint64_t>(kw.size());
        uint32_t* d_cells = m->tables.get<uint32_t>(cells.size());
        // rows by cell (HBM is plentiful); two entries of padding: the warp
        // kernel copies a row in 16-byte pieces from the 16-byte boundary at
        // or below its start, up to 15 bytes past its end
        m->d_alias = m->tables.get<uint64_t>(ncell * m->n_off + 2);
        if (!m->d_deme || !m->d_off || !d_kw || !d_cells || !m->d_alias) return fail(IND_ERR_OOM);
        bool okc = cudaMemcpyAsync(m->d_deme, dm.data(), ncell, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                   cudaMemcpyAsync(m->d_off, off.data(), off.size(), cudaMemcpyHostToDevice, s) == cudaSuccess &&
                   cudaMemcpyAsync(d_kw, kw.data(), kw.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                   cudaMemcpyAsync(d_cells, cells.data(), cells.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess;
        if (!okc) {
            g_last_cuda_error.store((int)cudaGetLastError());
            return fail(IND_ERR_CUDA);
        }
        const size_t per_warp = alias_build_warp_bytes(m->n_off);
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

// the sample of partition `part` of n_parts (n_parts = 1: the whole sample)
static ind_status sample_impl(ind_sim* m, double fraction, uint64_t sample_seed, uint32_t part, uint32_t n_parts,
                              int32_t scheme, uint64_t* n_sampled) {
    if (!m || !(fraction > 0.0 && fraction <= 1.0)) return IND_ERR_ARG;
    if (n_parts == 0 || part >= n_parts) return IND_ERR_ARG;
    if (n_parts > 1 && scheme != IND_PARTITION_LANDSCAPE && scheme != IND_PARTITION_INDIVIDUALS) return IND_ERR_ARG;
    const bool band = n_parts > 1 && scheme == IND_PARTITION_LANDSCAPE;
    const uint32_t stride = n_parts > 1 && scheme == IND_PARTITION_INDIVIDUALS ? n_parts : 1u;
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
    k_sample_flags<<<grid_for(n_slots, 256, sms * 32), 256, 0, s>>>(
        flags, n_slots, m->land.kind, m->land.width, m->land.deme, m->slot_deme, m->d_deme, fraction >= 1.0 ? 1 : 0,
        sk0, sk1, thr, m->land.height, band ? part : 0u, band ? n_parts : 1u);
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
    const uint64_t flagged = (uint64_t)last_pos + last_flag;
    // an individuals partition keeps every stride-th sampled individual from `part`
    const uint64_t count = stride > 1u ? (flagged > part ? (flagged - part + stride - 1) / stride : 0) : flagged;
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
                                                                   m->slot_deme, m->d_sample, stride > 1u ? part : 0u,
                                                                   stride);
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

ind_status sim_sample(ind_sim* m, double fraction, uint64_t sample_seed, uint64_t* n_sampled) {
    return sample_impl(m, fraction, sample_seed, 0, 1, IND_PARTITION_LANDSCAPE, n_sampled);
}

ind_status sim_sample_partition(ind_sim* m, double fraction, uint64_t sample_seed, uint32_t part,
                                uint32_t n_parts, int32_t scheme, uint64_t* n_sampled) {
    return sample_impl(m, fraction, sample_seed, part, n_parts, scheme, n_sampled);
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
        tables = ncell * (1 + 4 + n_off * 8) + 16 + 2 * n_off + 8 * (size_t)(R * R + 1);
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
    // + 4 (work list)
    const double per = 48 + 20 + 24 + 8 + 96 + 8 + 64 + 16 + 4;
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

ind_status sim_selftest_search(ind_sim* m, int form, const uint64_t* loc, const double* tau, uint64_t n,
                               double* out) {
    if (!m || !loc || !tau || !out || n == 0 || n > (1ull << 26) || form < 0 || form > 5) return IND_ERR_ARG;
    cudaStream_t s = m->stream;
    ind_status st = ensure_ln_tables(s);
    if (st != IND_OK) return st;
    SimParams hp;
    fill_params(m, m->tuning, hp);
    Pool tmp;
    tmp.stream = s;
    SimParams* d_p = tmp.get<SimParams>(1);
    SimState* d_s = tmp.get<SimState>(1);
    uint64_t* d_loc = tmp.get<uint64_t>(n);
    double* d_tau = tmp.get<double>(n);
    double* d_out = tmp.get<double>(n);
    if (!d_p || !d_s || !d_loc || !d_tau || !d_out) {
        tmp.release_all();
        return IND_ERR_OOM;
    }
    bool ok = cudaMemcpyAsync(d_p, &hp, sizeof(hp), cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemsetAsync(d_s, 0, sizeof(SimState), s) == cudaSuccess &&
              cudaMemcpyAsync(d_loc, loc, n * 8, cudaMemcpyDefault, s) == cudaSuccess &&
              cudaMemcpyAsync(d_tau, tau, n * 8, cudaMemcpyDefault, s) == cudaSuccess;
    if (ok) {
        const uint32_t threads = 256;
        const bool lane_form = form <= 1 || form == 5;
        const uint32_t grid = lane_form ? grid_for(n, threads, sm_count() * 8) : grid_for(n * 32, threads, sm_count() * 8);
        switch (form) {
            case 0: k_selftest_search<0><<<grid, threads, 0, s>>>(d_p, d_s, d_loc, d_tau, n, d_out); break;
            case 1: k_selftest_search<1><<<grid, threads, 0, s>>>(d_p, d_s, d_loc, d_tau, n, d_out); break;
            case 2: k_selftest_search<2><<<grid, threads, 0, s>>>(d_p, d_s, d_loc, d_tau, n, d_out); break;
            case 3: k_selftest_search<3><<<grid, threads, 0, s>>>(d_p, d_s, d_loc, d_tau, n, d_out); break;
            case 4: k_selftest_search<4><<<grid, threads, 0, s>>>(d_p, d_s, d_loc, d_tau, n, d_out); break;
            default: k_selftest_search<5><<<grid, threads, 0, s>>>(d_p, d_s, d_loc, d_tau, n, d_out); break;
        }
        g_launches.fetch_add(1);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok) ok = cudaMemcpyAsync(out, d_out, n * 8, cudaMemcpyDefault, s) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
    tmp.release_all();
    if (!ok) {
        g_last_cuda_error.store((int)cudaGetLastError());
        return IND_ERR_CUDA;
    }
    return IND_OK;
}

ind_status sim_alias_row(ind_sim* m, uint32_t x, uint32_t y, uint64_t* out, uint32_t cap, uint32_t* n_out) {
    if (!m || !n_out || m->land.kind != IND_MAP || x >= m->land.width || y >= m->land.height) return IND_ERR_ARG;
    *n_out = m->n_off;
    if (!out) return IND_OK;
    if (cap < m->n_off) return IND_ERR_ARG;
    const size_t cell = (size_t)y * m->land.width + x;
    uint8_t deme = 0;
    if (cudaMemcpyAsync(&deme, m->d_deme + cell, 1, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        g_last_cuda_error.store((int)cudaGetLastError());
        return IND_ERR_CUDA;
    }
    if (deme == 0) return IND_ERR_ARG;  // rows exist for habitable cells only
    if (cudaMemcpyAsync(out, m->d_alias + cell * m->n_off, (size_t)m->n_off * 8, cudaMemcpyDefault, m->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        g_last_cuda_error.store((int)cudaGetLastError());
        return IND_ERR_CUDA;
    }
    return IND_OK;
}

}  // extern "C"
