// engine.cu -- kernels and C ABI of the Independent-algorithm engine: one
// translation unit made of the engine_*.cuh parts included at the end of this
// file, in order (state, per-lineage event arithmetic, round kernels, species
// and event-stream reduction, inputs, batch host side, C ABI, the merge of
// isolated partitions, allocation-free ranking, server).
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
#include <type_traits>
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

#include "engine_state.cuh"
#include "engine_events.cuh"
#include "engine_advance.cuh"
#include "engine_species.cuh"
#include "engine_inputs.cuh"
#include "engine_batch.cuh"
#include "engine_api.cuh"
#include "engine_partition.cuh"
#include "engine_rank_static.cuh"
#include "engine_server.cuh"
