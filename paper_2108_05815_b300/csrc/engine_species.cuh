// engine_species.cuh -- roots, the species sort/unique/rank, scans and the event-stream reduction kernels.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

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
// Stable least-significant-digit radix sort of (u64 key, u32 value) pairs:
// 8-bit digits, tiles of 4,096 items per block of 8 warps.  Per pass:
// per-block digit counts, one exclusive scan (digit-major, so that block b's
// items of digit d follow those of blocks before b), and a scatter in which
// every warp handles a contiguous sub-tile in order, ranking equal digits of
// each 32-item chunk with __match_any_sync: ties keep their input order.
constexpr int RS_RADIX = 256;
constexpr int RS_WARPS = 8;
constexpr int RS_ITEMS = 16;                           // per lane
constexpr uint32_t RS_SUB = 32u * RS_ITEMS;            // items per warp
constexpr uint32_t RS_TILE = RS_WARPS * RS_SUB;        // items per block

__global__ void __launch_bounds__(RS_WARPS * 32) k_rs_count(const uint64_t* __restrict__ keys, uint32_t n, int shift,
                                                             uint32_t* __restrict__ counts) {
    __shared__ uint32_t h[RS_RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t start = blockIdx.x * RS_TILE, end = min(start + RS_TILE, n);
    for (uint32_t i = start + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&h[(uint32_t)(keys[i] >> shift) & (RS_RADIX - 1)], 1u);
    __syncthreads();
    counts[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_WARPS * 32) k_rs_scatter(const uint64_t* __restrict__ keys_in,
                                                               const uint32_t* __restrict__ vals_in, uint32_t n,
                                                               int shift, const uint32_t* __restrict__ offsets,
                                                               uint64_t* __restrict__ keys_out,
                                                               uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t wbase[RS_WARPS][RS_RADIX];  // per-warp digit counts, then starting positions
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    for (uint32_t k = threadIdx.x; k < RS_WARPS * RS_RADIX; k += blockDim.x) (&wbase[0][0])[k] = 0;
    __syncthreads();
    const uint32_t sub = blockIdx.x * RS_TILE + w * RS_SUB;
    for (int j = 0; j < RS_ITEMS; ++j) {
        const uint32_t i = sub + (uint32_t)j * 32u + lane;
        if (i < n) atomicAdd(&wbase[w][(uint32_t)(keys_in[i] >> shift) & (RS_RADIX - 1)], 1u);
    }
    __syncthreads();
    {   // thread d: the block's offset of digit d, handed out to the warps in order
        const uint32_t d = threadIdx.x;
        uint32_t run = offsets[d * gridDim.x + blockIdx.x];
        for (int v = 0; v < RS_WARPS; ++v) {
            const uint32_t c = wbase[v][d];
            wbase[v][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int j = 0; j < RS_ITEMS; ++j) {
        const uint32_t i = sub + (uint32_t)j * 32u + lane;
        const bool valid = i < n;
        const uint64_t key = valid ? keys_in[i] : 0ull;
        const uint32_t d = valid ? ((uint32_t)(key >> shift) & (RS_RADIX - 1)) : (RS_RADIX + lane);  // unique when invalid
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        if (valid) {
            const uint32_t pos = wbase[w][d] + __popc(peers & lt);
            keys_out[pos] = key;
            vals_out[pos] = vals_in[i];
        }
        __syncwarp();
        if (valid && lane == (uint32_t)(__ffs(peers) - 1)) wbase[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

// sort key of one field of the log entries, in the current order
// (field 0: lineage, 1: prior time, 2: location, 3: time)
__device__ __forceinline__ uint64_t ev_field(const EventLog& L, int f, uint32_t k) {
    return f == 0 ? (uint64_t)L.gid[k] : f == 1 ? L.prior[k] : f == 2 ? L.loc[k] : L.time[k];
}

__global__ void k_ev_field(EventLog L, int f, const uint32_t* __restrict__ order, uint32_t n, uint64_t* keys) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        keys[i] = ev_field(L, f, order ? order[i] : i);
}

__global__ void k_iota(uint32_t* v, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

// AND and OR of every field over the log: a byte that is the same in every
// entry needs no radix pass
__global__ void k_ev_bits(EventLog L, uint32_t n, unsigned long long* and_or /* 4 fields x (and, or) */) {
    uint64_t a[4], o[4];
    for (int f = 0; f < 4; ++f) {
        a[f] = ~0ull;
        o[f] = 0ull;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int f = 0; f < 4; ++f) {
            const uint64_t v = ev_field(L, f, i);
            a[f] &= v;
            o[f] |= v;
        }
    for (int f = 0; f < 4; ++f) {
        for (int d = 16; d > 0; d >>= 1) {
            a[f] &= __shfl_xor_sync(0xFFFFFFFFu, a[f], d);
            o[f] |= __shfl_xor_sync(0xFFFFFFFFu, o[f], d);
        }
        if ((threadIdx.x & 31u) == 0) {
            atomicAnd(&and_or[2 * f], (unsigned long long)a[f]);
            atomicOr(&and_or[2 * f + 1], (unsigned long long)o[f]);
        }
    }
}

// batches of several simulations: each entry's simulation, the last one
// whose first lineage id is at or below the entry's lineage
__global__ void k_ev_sim(EventLog L, uint32_t n, const uint32_t* __restrict__ gid_base, uint32_t n_sims,
                         uint32_t* out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t g = L.gid[i];
        uint32_t lo = 0, hi = n_sims;  // gid_base[lo] <= g < gid_base[hi] (hi: past the end)
        while (hi - lo > 1u) {
            const uint32_t mid = (lo + hi) >> 1;
            if (gid_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        out[i] = lo;
    }
}

// radix key of the simulation field, through the current order
__global__ void k_ev_key_u32(const uint32_t* __restrict__ src, const uint32_t* __restrict__ order, uint32_t n,
                             uint64_t* keys) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        keys[i] = src[order[i]];
}

// the log in (simulation, time, location, prior time, lineage) order as sort
// items; isim (batches of several simulations) receives each item's
// simulation
__global__ void k_ev_gather(EventLog L, const uint32_t* __restrict__ order, uint32_t n, SortItem* items,
                            const uint32_t* __restrict__ lsim, uint32_t* isim) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = order[i];
        items[i] = SortItem{L.time[k], L.loc[k], L.prior[k], ((unsigned long long)L.gid[k] << 32) | k};
        if (isim) isim[i] = lsim[k];
    }
}

// a new distinct event where (simulation, time, location) changes; a
// coalescence where, within one event, the prior time changes
__global__ void k_ev_marks(const SortItem* __restrict__ x, uint32_t n, const uint32_t* __restrict__ isim,
                           uint32_t* head, uint32_t* coal) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool h = i == 0 || x[i].a != x[i - 1].a || x[i].b != x[i - 1].b || (isim && isim[i] != isim[i - 1]);
        head[i] = h ? 1u : 0u;
        coal[i] = (!h && x[i].c != x[i - 1].c) ? 1u : 0u;
    }
}

// a lineage id as its simulation numbers it (batches: less the simulation's
// first global id)
__device__ __forceinline__ uint32_t ev_lineage(const SortItem& x, uint32_t i, const uint32_t* __restrict__ isim,
                                               const uint32_t* __restrict__ gid_base) {
    const uint32_t g = (uint32_t)(x.d >> 32);
    return isim ? g - gid_base[isim[i]] : g;
}

__global__ void k_ev_events(const SortItem* __restrict__ x, uint32_t n, const uint32_t* head,
                            const uint32_t* incl_head, const uint64_t* __restrict__ target, uint32_t* head_pos,
                            ind_event* out, const uint32_t* __restrict__ isim, const uint32_t* __restrict__ gid_base) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        const uint32_t g = incl_head[i] - 1u;
        head_pos[g] = i;
        const uint32_t idx = (uint32_t)x[i].d;
        out[g] = ind_event{x[i].a, x[i].c, x[i].b, target[idx], ev_lineage(x[i], i, isim, gid_base), 0u};
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
                                  ind_coalescence* out, const uint32_t* __restrict__ isim,
                                  const uint32_t* __restrict__ gid_base) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!coal[i]) continue;
        const uint32_t hp = head_pos[incl_head[i] - 1u];
        out[incl_coal[i] - 1u] = ind_coalescence{x[i].b, x[i].c, ev_lineage(x[hp], hp, isim, gid_base),
                                                 ev_lineage(x[i], i, isim, gid_base)};
    }
}

// batches: distinct events and coalescences per simulation
__global__ void k_ev_sim_counts(const uint32_t* __restrict__ head, const uint32_t* __restrict__ coal,
                                const uint32_t* __restrict__ isim, uint32_t n, uint32_t* ev_count,
                                uint32_t* co_count) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (head[i]) atomicAdd(ev_count + isim[i], 1u);
        if (coal[i]) atomicAdd(co_count + isim[i], 1u);
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
