// engine_partition.cuh -- the merge of isolated partitions: distinct speciation keys and their global ranks.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

// items (0, location, time bits, index) of n keys
__global__ void k_keys_items(const uint64_t* __restrict__ kl, const uint64_t* __restrict__ kt, uint32_t n,
                             uint32_t n_pad, SortItem* items) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
        items[i] = i < n ? SortItem{0ull, kl[i], kt[i], i} : SortItem{~0ull, ~0ull, ~0ull, ~0ull};
}

// 1 where a sorted item starts a run of equal keys
__global__ void k_keys_heads(const SortItem* __restrict__ x, uint32_t n, uint32_t* head) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        head[i] = (i == 0 || x[i].b != x[i - 1].b || x[i].c != x[i - 1].c) ? 1u : 0u;
}

__global__ void k_keys_write(const SortItem* __restrict__ x, const uint32_t* __restrict__ head,
                             const uint32_t* __restrict__ pos, uint32_t n, uint64_t* out_loc, uint64_t* out_time) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (head[i]) {
            out_loc[pos[i]] = x[i].b;
            out_time[pos[i]] = x[i].c;
        }
}

// binary search of each key in the sorted distinct reference; a missing key
// gets ~0 and sets *missing
__global__ void k_keys_rank(const uint64_t* __restrict__ kl, const uint64_t* __restrict__ kt, uint64_t n,
                            const uint64_t* __restrict__ rl, const uint64_t* __restrict__ rt, uint64_t n_ref,
                            uint64_t* rank, uint32_t* missing) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = kl[i], b = kt[i];
        uint64_t lo = 0, hi = n_ref;  // first reference key not below (a, b)
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            const uint64_t ma = rl[mid], mb = rt[mid];
            if (ma < a || (ma == a && mb < b)) lo = mid + 1;
            else hi = mid;
        }
        if (lo < n_ref && rl[lo] == a && rt[lo] == b) {
            rank[i] = lo;
        } else {
            rank[i] = ~0ull;
            atomicOr(missing, 1u);
        }
    }
}

extern "C" {

ind_status ind_keys_unique(const uint64_t* key_loc, const uint64_t* key_time, uint64_t n, uint64_t* out_loc,
                           uint64_t* out_time, uint64_t* n_out, void* stream) {
    if (!n_out || n > (1ull << 31) || (n && (!key_loc || !key_time || !out_loc || !out_time))) return IND_ERR_ARG;
    *n_out = 0;
    if (n == 0) return IND_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n32 = (uint32_t)n;
    uint32_t n_pad = 2048;
    while (n_pad < n32) n_pad <<= 1;
    Pool T;
    T.stream = s;
    SortItem* items = T.get<SortItem>(n_pad);
    uint32_t* head = T.get<uint32_t>(n32);
    uint32_t* pos = T.get<uint32_t>(n32);
    if (!items || !head || !pos) {
        T.release_all();
        return IND_ERR_OOM;
    }
    const uint32_t sms = sm_count();
    k_keys_items<<<grid_for(n_pad, 256, sms * 16), 256, 0, s>>>(key_loc, key_time, n32, n_pad, items);
    g_launches.fetch_add(1);
    ind_status st = bitonic_sort(items, n_pad, s);
    if (st == IND_OK) {
        k_keys_heads<<<grid_for(n32, 256, sms * 16), 256, 0, s>>>(items, n32, head);
        g_launches.fetch_add(1);
        st = scan_u32(T, head, pos, n32, false, s);
    }
    uint32_t last_pos = 0, last_head = 0;
    if (st == IND_OK) {
        k_keys_write<<<grid_for(n32, 256, sms * 16), 256, 0, s>>>(items, head, pos, n32, out_loc, out_time);
        g_launches.fetch_add(1);
        if (cudaMemcpyAsync(&last_pos, pos + n32 - 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&last_head, head + n32 - 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            g_last_cuda_error.store((int)cudaGetLastError());
            st = IND_ERR_CUDA;
        }
    }
    T.release_all();
    if (st != IND_OK) return st;
    *n_out = (uint64_t)last_pos + last_head;
    return IND_OK;
}

ind_status ind_keys_rank(const uint64_t* key_loc, const uint64_t* key_time, uint64_t n, const uint64_t* ref_loc,
                         const uint64_t* ref_time, uint64_t n_ref, uint64_t* rank_out, void* stream) {
    if (n && (!key_loc || !key_time || !rank_out)) return IND_ERR_ARG;
    if (n_ref && (!ref_loc || !ref_time)) return IND_ERR_ARG;
    if (n == 0) return IND_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Pool T;
    T.stream = s;
    uint32_t* missing = T.get<uint32_t>(1);
    if (!missing) return IND_ERR_OOM;
    uint32_t h_missing = 0;
    ind_status st = IND_OK;
    if (cudaMemsetAsync(missing, 0, 4, s) != cudaSuccess) st = IND_ERR_CUDA;
    if (st == IND_OK) {
        k_keys_rank<<<grid_for(n, 256, sm_count() * 16), 256, 0, s>>>(key_loc, key_time, n, ref_loc, ref_time, n_ref,
                                                                      rank_out, missing);
        g_launches.fetch_add(1);
        if (cudaMemcpyAsync(&h_missing, missing, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            g_last_cuda_error.store((int)cudaGetLastError());
            st = IND_ERR_CUDA;
        }
    }
    T.release_all();
    if (st != IND_OK) return st;
    return h_missing ? IND_ERR_ARG : IND_OK;
}

}  // extern "C"
