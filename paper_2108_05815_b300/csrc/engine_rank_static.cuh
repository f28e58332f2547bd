// engine_rank_static.cuh -- species ranking without device allocation (ind_species_rank_static).
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

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
