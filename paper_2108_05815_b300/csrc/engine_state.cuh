// engine_state.cuh -- process-wide state (allocator, launch counter, status macros) and the device data structures.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

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

// alias rows of a habitat map: at most 2^13 columns (the alias build's
// 16-bit work lists; radius 40 gives 5,025)
constexpr int ALIAS_COL_BITS = 13;
constexpr uint32_t ALIAS_MAX_OFFSETS = 1u << ALIAS_COL_BITS;

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
    const uint64_t* alias;     // W*H rows (by cell) x n_off entries (format: k_alias_build)
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
    uint32_t n_work;        // entries of the round's work list (k_filter)
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
    // dedup inserts, counted only in the exact-counting mode (count_unique):
    // all of them, those whose slot key was already in the table, and those
    // that another active lane of the same warp inserted in the same
    // instruction (what a warp pre-collapse of equal keys would save)
    unsigned long long ins_total, ins_repeat, ins_warp_repeat;
    // rounds of the one-lane form: lineages listed for the warp kernel
    // (k_filter's claims, possibly beyond the list's capacity) and its claim counter
    uint32_t n_heavy;
    uint32_t heavy_ctr;
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
    uint32_t* work;  // the round's work list: buffer indices of lineages with an event before the horizon
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
    const uint32_t* pois_guide;  // warp kernel: the Poisson guide and thresholds every simulation shares,
    const uint64_t* pois_cdf;    // staged in shared memory at pois_off (null: each simulation's own)
    uint32_t pois_n;
    uint32_t pois_off;
    const uint32_t* gauss_guide;  // likewise the torus dispersal tables (the same sigma everywhere)
    const uint64_t* gauss_cdf;
    uint32_t gauss_n;
    uint32_t gauss_off;
    const int8_t* off_tab;        // likewise the map's dispersal offsets (the same radius everywhere)
    uint32_t off_n;
    uint32_t off_off;
    uint32_t stage_off;      // warp kernel: shared-memory offset of the per-warp alias-row buffers
    uint32_t stage_bytes;    // bytes of one such buffer (0: map rows are read from global memory)
    EventLog log;            // cap 0: no logging
    // rounds of the one-lane form: the lineages with many events before the
    // horizon, run by the warp kernel after the one-lane kernel when they
    // fit its warps (heavy_cap entries; 0: every lineage on the one-lane list)
    uint32_t* heavy;
    uint32_t heavy_cap;
};
