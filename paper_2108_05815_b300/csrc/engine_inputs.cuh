// engine_inputs.cuh -- inputs: habitat map, alias rows, sampling, the arithmetic self-test.
// A part of the engine.cu translation unit, included there in order after
// the parts before it; not a standalone header.
#pragma once

// ---------------------------------------------------------------------------
// inputs: habitat map, alias rows, sampling
// ---------------------------------------------------------------------------
__global__ void k_habitat(uint8_t* out, uint32_t W, uint32_t H, uint32_t sk0, uint32_t sk1, uint64_t thr,
                          uint32_t max_deme) {
    const uint64_t n = (uint64_t)W * H;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n; c += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(c % W), y = (uint32_t)(c / W);
        const u64x2 b = stream_block(sk0, sk1, pack_loc(x, y, 0), 0, 0, TAG_MAP);
        out[c] = (b.lo >> 11) < thr ? (uint8_t)(1u + umulhi64(b.hi, max_deme)) : (uint8_t)0;
    }
}

// one warp per habitable cell: weights, then integer Vose.  Rows are
// indexed by cell (those of cells without habitat are never read), and an
// entry holds everything a dispersal that falls on the alias needs:
// threshold q (bits 0-31), the alias column's offset dx (32-38) and dy
// (39-45) as 7-bit two's complement, the deme of the column's own target
// (46-53) and of the alias column's target (54-61), and bit 63 for a column
// that is always taken.  A dispersal that keeps its column reads the
// column's offset from the offset table, a load that does not wait for the
// entry.
__device__ __forceinline__ uint64_t alias_entry(uint64_t q, int32_t adx, int32_t ady, uint8_t deme_col,
                                                uint8_t deme_alias, bool full) {
    return q | ((uint64_t)((uint32_t)adx & 0x7Fu) << 32) | ((uint64_t)((uint32_t)ady & 0x7Fu) << 39) |
           ((uint64_t)deme_col << 46) | ((uint64_t)deme_alias << 54) | (full ? (1ull << 63) : 0ull);
}

// shared-memory bytes of one warp of k_alias_build for n_off offsets
__host__ __device__ constexpr size_t alias_build_warp_bytes(uint32_t n_off) {
    return ((size_t)n_off * 15 + 15) & ~(size_t)15;
}

constexpr uint16_t ALIAS_FULL = 0xFFFFu;  // a column that is always taken

// Vose's pairing is sequential (lane 0 pops the small and large stacks in
// order); the threshold of a column depends only on its scaled weight when
// it was popped as small, which never changes afterwards.  So all lanes
// fill the stacks (a stable partition by ballot), lane 0 only pairs, with
// the stacks' tops in registers, all lanes mark the columns left over as
// always taken, and then compute the thresholds floor(s_a 2^32 / W) by
// restoring division and write the entries, 32 columns at a time.
__global__ void k_alias_build(const uint8_t* __restrict__ deme, uint32_t W, uint32_t H,
                              const uint32_t* __restrict__ cells, uint32_t n_rows, const int8_t* __restrict__ off,
                              uint32_t n_off, const uint64_t* __restrict__ kw, uint64_t* __restrict__ alias) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    uint64_t* s = (uint64_t*)(smem + alias_build_warp_bytes(n_off) * w);  // 16-byte aligned regions
    uint16_t* small_ = (uint16_t*)(s + n_off);
    uint16_t* large_ = small_ + n_off;
    uint16_t* alias_of = large_ + n_off;                // alias column, or ALIAS_FULL
    uint8_t* tdeme = (uint8_t*)(alias_of + n_off);      // deme of each offset's target
    for (uint32_t row = blockIdx.x * warps + w; row < n_rows; row += gridDim.x * warps) {
        const uint32_t cell = cells[row];
        const uint32_t cx = cell % W, cy = cell / W;
        unsigned long long part = 0;
        for (uint32_t o = lane; o < n_off; o += 32) {
            const int32_t dx = off[2 * o], dy = off[2 * o + 1];
            const uint32_t tx = wrap_add(cx, dx, W), ty = wrap_add(cy, dy, H);
            const uint8_t td = deme[(size_t)ty * W + tx];
            const uint64_t wgt = kw[dx * dx + dy * dy] * (uint64_t)td;
            s[o] = (uint64_t)n_off * wgt;
            tdeme[o] = td;
            part += wgt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        const uint64_t Wt = part;
        __syncwarp();
        // the small and large stacks filled in ascending column order, 32
        // columns at a time (a stable partition by ballot)
        uint32_t ns = 0, nl = 0;  // the same in every lane
        for (uint32_t base = 0; base < n_off; base += 32u) {
            const uint32_t o = base + lane;
            const bool valid = o < n_off;
            const bool sm = valid && s[o] < Wt;
            const unsigned ms = __ballot_sync(0xFFFFFFFFu, sm);
            const unsigned ml = __ballot_sync(0xFFFFFFFFu, valid && !sm);
            const unsigned below = (1u << lane) - 1u;
            if (sm) small_[ns + __popc(ms & below)] = (uint16_t)o;
            else if (valid) large_[nl + __popc(ml & below)] = (uint16_t)o;
            ns += (uint32_t)__popc(ms);
            nl += (uint32_t)__popc(ml);
        }
        __syncwarp();
        if (lane == 0 && ns > 0 && nl > 0) {
            // Vose's pairing, in its order: pop a (small) and b (large),
            // alias(a) = b, s_b += s_a - W, push b onto the stack its new
            // weight belongs to.  The pushed b is the next pop of that stack,
            // so it stays in registers; s[a] is never changed again (a's
            // threshold comes from it) and s[b] is written when b leaves.
            uint32_t a = small_[--ns], b = large_[--nl];
            uint64_t sa = s[a], sb = s[b];
            for (;;) {
                alias_of[a] = (uint16_t)b;
                sb = sb + sa - Wt;
                if (sb < Wt) {  // b moves to the small stack: it is the next a
                    s[b] = sb;
                    if (nl == 0) {
                        small_[ns++] = (uint16_t)b;
                        break;
                    }
                    a = b;
                    sa = sb;
                    b = large_[--nl];
                    sb = s[b];
                } else {        // b stays on top of the large stack
                    if (ns == 0) {
                        s[b] = sb;
                        large_[nl++] = (uint16_t)b;
                        break;
                    }
                    a = small_[--ns];
                    sa = s[a];
                }
            }
        }
        ns = __shfl_sync(0xFFFFFFFFu, ns, 0);
        nl = __shfl_sync(0xFFFFFFFFu, nl, 0);
        __syncwarp();
        // the columns left on either stack are always taken
        for (uint32_t k = lane; k < nl; k += 32u) alias_of[large_[k]] = ALIAS_FULL;
        for (uint32_t k = lane; k < ns; k += 32u) alias_of[small_[k]] = ALIAS_FULL;
        __syncwarp();
        uint64_t* e = alias + (size_t)cell * n_off;
        for (uint32_t o = lane; o < n_off; o += 32) {
            const uint32_t b = alias_of[o];
            if (b == ALIAS_FULL) {
                e[o] = alias_entry(0xFFFFFFFFull, off[2 * o], off[2 * o + 1], tdeme[o], tdeme[o], true);
                continue;
            }
            // q = floor(s_o 2^32 / W) by restoring division (s_o < W < 2^56)
            uint64_t rem = s[o], q = 0;
            for (int bit = 0; bit < 32; ++bit) {
                rem <<= 1;
                q <<= 1;
                if (rem >= Wt) {
                    rem -= Wt;
                    q |= 1ull;
                }
            }
            e[o] = alias_entry(q, off[2 * b], off[2 * b + 1], tdeme[o], tdeme[b], false);
        }
        __syncwarp();
    }
}

// band: a landscape partition keeps only the cells of rows y with
// floor(y n_parts / H) == part (n_parts = 1: every row)
__global__ void k_sample_flags(uint32_t* flags, uint64_t n_slots, int kind, uint32_t W, uint32_t D,
                               uint32_t slot_deme, const uint8_t* deme, int all, uint32_t sk0, uint32_t sk1,
                               uint64_t thr, uint32_t H, uint32_t part, uint32_t n_parts) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n_slots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t cell = s / slot_deme;
        const uint32_t i = (uint32_t)(s % slot_deme);
        const uint32_t d = kind == KIND_MAP ? deme[cell] : D;
        bool keep = i < d && (n_parts <= 1u || (cell / W) * n_parts / H == part);
        if (keep && !all) {
            const uint64_t loc = pack_loc(cell % W, cell / W, i);
            keep = (stream_block(sk0, sk1, loc, 0, 0, TAG_SAMPLE).lo >> 11) < thr;
        }
        flags[s] = keep ? 1u : 0u;
    }
}

// stride > 1: an individuals partition keeps the sampled individuals whose
// sample index j has j mod stride == part, as entry j / stride
__global__ void k_sample_write(const uint32_t* flags, const uint32_t* pos, uint64_t n_slots, uint32_t W,
                               uint32_t slot_deme, uint64_t* out, uint32_t part, uint32_t stride) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n_slots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        if (!flags[s]) continue;
        const uint32_t j = pos[s];
        if (stride > 1u && j % stride != part) continue;
        const uint64_t cell = s / slot_deme;
        out[j / stride] = pack_loc(cell % W, cell / W, s % slot_deme);
    }
}

// device arithmetic probes for the conformance tests
__global__ void k_selftest(const uint64_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ exp_q58,
                           uint32_t* __restrict__ philox_out) {
    const LnC ln = ln_tables();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = in[i];
        if (exp_q58) exp_q58[i] = exp1_q58(v >> 11, ln.L, ln.R, ln.ln2, ln.c3);
        if (philox_out) {
            const uint64_t w = in[(i + 1) % n], z = in[(i + 2) % n];
            const u32x4 o = philox10((uint32_t)v, (uint32_t)(v >> 32), (uint32_t)w, (uint32_t)(w >> 32),
                                     (uint32_t)z, (uint32_t)(z >> 32));
            philox_out[4 * i + 0] = o.x;
            philox_out[4 * i + 1] = o.y;
            philox_out[4 * i + 2] = o.z;
            philox_out[4 * i + 3] = o.w;
        }
    }
}

// event-time search probe (sim_selftest_search): the first event time after
// tau[q] at loc[q] by one search form; forms 0 and 1 one lane per query
// (one or two draw blocks per step, as the one-lane kernel runs them), 2 to
// 4 one warp per query (general, short in binary64, short as the tail
// kernel runs it), 5 one lane per query in binary64 throughout
template <int FORM>
__global__ void k_selftest_search(const SimParams* __restrict__ P, const SimState* S, const uint64_t* __restrict__ loc,
                                  const double* __restrict__ tau, uint64_t n, double* __restrict__ out) {
    LaneSim c;
    load_lanesim(c, P, S, 0);
    const LnC ln = ln_tables();
    if (FORM <= 1 || FORM == 5) {
        for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n;
             q += (uint64_t)gridDim.x * blockDim.x) {
            if (FORM == 5)
                out[q] = c.sampler == 1 ? next_event_time_poisson(c, loc[q], tau[q])
                         : c.lam1       ? next_event_time_exp<1, true>(c, loc[q], tau[q], ln)
                                        : next_event_time_exp<1, false>(c, loc[q], tau[q], ln);
            else
                out[q] = next_event_time<FORM + 1>(c, loc[q], tau[q], ln);
        }
        return;
    }
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; q < n; q += warps) {
        const uint64_t l = loc[q];
        const double t0 = tau[q];
        double t;
        if (c.sampler == 1) {
            t = FORM == 2   ? coop_next_poisson(c, l, t0, lane)
                : FORM == 3 ? coop_next_poisson_short_fp(c, l, t0, lane)
                            : coop_next_poisson_short(c, l, t0, lane);
        } else if (FORM == 2) {
            t = c.lam1 ? coop_next_exp<true>(c, l, t0, ln, lane) : coop_next_exp<false>(c, l, t0, ln, lane);
        } else if (FORM == 3) {
            t = c.lam1 ? coop_next_exp_short_fp<true>(c, l, t0, ln, lane)
                       : coop_next_exp_short_fp<false>(c, l, t0, ln, lane);
        } else {
            t = c.lam1 ? coop_next_exp_short<true>(c, l, t0, ln, lane) : coop_next_exp_short<false>(c, l, t0, ln, lane);
        }
        if (lane == 0) out[q] = t;
    }
}
