// Test-side host wrapper (not part of the library): the device header's
// event-search draw rounding, exp1_grid, compiled for the host so that the
// CPU test suite can compare it with the oracle.  On the host the
// normalising length comes from a leading-zero count instead of the
// device's binary32 conversion; both are floor(log2 x) exactly.
#include <cstdint>
#include "../../paper_2108_05815_b300/csrc/device.cuh"

namespace indep {
void host_ln_tables(uint64_t* L, uint32_t* R, int n, uint64_t* ln2_q64, int64_t* c3);
}
using namespace indep;

static LnTables g_tab;
static int g_ready = 0;

// for i < n: x58[i], a[i] and near[i] of exp1_grid(r[i], sft[i])
extern "C" int grid_draws(const uint64_t* r, const int32_t* sft, int64_t n, uint64_t* x58, uint64_t* a,
                          uint8_t* near) {
    if (!g_ready) {
        host_ln_tables(g_tab.L, g_tab.R, (int)LN_N, &g_tab.ln2_q64, &g_tab.c3);
        g_ready = 1;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (r[i] >= (1ull << 53) || sft[i] < 0 || sft[i] > 63) return -1;
        const GridDraw g = exp1_grid(r[i], g_tab.L, g_tab.R, g_tab.ln2_q64, g_tab.c3, sft[i]);
        x58[i] = g.x58;
        a[i] = g.a;
        near[i] = g.near ? 1 : 0;
    }
    return 0;
}
