/*
 * oracle.c -- plain, slow CPU oracle of the Independent algorithm.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes (Langenstein 2021, "Communication-free and Parallel
 * Simulation of Neutral Biodiversity Models"):
 *   - every sampled individual's lineage is traced backwards in time on its
 *     own (Independent algorithm, section "The Independent Algorithm" and its
 *     summary listing);
 *   - randomness comes from an RNG that is re-primed on the environment
 *     (seed, indexed location, time) before every use (section
 *     "Environmental RNG Priming"), realised here with the counter-based
 *     Philox4x32-10 generator of Salmon et al. (2011), which the paper's
 *     background on counter-based generators cites;
 *   - inter-event times are exponential, generated as memoryless sums of
 *     Exp(lambda) variates inside re-prime intervals of length delta_t
 *     (sections "Aligning the RNGs of Colliding Individuals" and
 *     "Memoryless sums of exponentials"), with Exp drawn by inverse transform
 *     -ln(U)/lambda (appendix "Inverse Transform: Uniform and Exponential");
 *   - at each event the RNG is primed on (location, event time), the
 *     individual speciates with probability nu, else disperses (summary
 *     listing of the Independent algorithm);
 *   - species identity = the speciation event an individual's lineage ends in
 *     (section "A Neutral Coalescence-based Simulation");
 *   - the spatially implicit scenario (background section "Spatially
 *     Implicit", appendix of the neutral scenarios): a non-spatial local
 *     community of J individuals whose parents live, with probability m per
 *     event, in a static non-spatial metacommunity of J_meta individuals with
 *     its own speciation probability nu_meta.
 *
 * Mode P (or_trace*) is the plain definition: one lineage, no interaction.
 * Mode M (or_run_merge) processes all events of all lineages in global time
 * order and merges a lineage into the occupant of the slot it disperses to
 * (the classical coalescence structure); every event is then executed exactly
 * once, so its event count is the number of unique events.
 *
 * Floating point: IEEE binary64, round-to-nearest; build with
 * -ffp-contract=off and without -ffast-math.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

#define OR_TAG_INTERVAL 1u
#define OR_TAG_EVENT 2u
#define OR_TAG_MAP 3u
#define OR_TAG_SAMPLE 4u

#define OR_NONSPATIAL 0
#define OR_TORUS 1
#define OR_MAP 2
#define OR_IMPLICIT 3

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplications with a Weyl-sequence key schedule.
 * ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t key_in[2], const uint32_t ctr_in[4], uint32_t out[4])
{
    uint32_t k0 = key_in[0], k1 = key_in[1];
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream base key of a simulation seed: the first two output words of
 * Philox keyed by the seed at counter zero. */
void or_seed_key(uint64_t seed, uint32_t sk[2])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {0, 0, 0, 0};
    uint32_t out[4];
    or_philox4x32_10(key, ctr, out);
    sk[0] = out[0];
    sk[1] = out[1];
}

/* prime(seed, location, time) followed by the draws of that stream: the
 * block j of the stream primed at (loc, tkey, tag) holds the 64-bit draws
 * 2j and 2j+1.  The location enters the key, (time, j, tag) the counter. */
void or_draw_pair(const uint32_t sk[2], uint64_t loc, uint64_t tkey, uint32_t tag, uint32_t j,
                  uint64_t v[2])
{
    uint32_t key[2] = {sk[0] ^ (uint32_t)loc, sk[1] ^ (uint32_t)(loc >> 32)};
    uint32_t ctr[4] = {(uint32_t)tkey, (uint32_t)(tkey >> 32), j, tag};
    uint32_t out[4];
    or_philox4x32_10(key, ctr, out);
    v[0] = (uint64_t)out[0] | ((uint64_t)out[1] << 32);
    v[1] = (uint64_t)out[2] | ((uint64_t)out[3] << 32);
}

/* the idx-th 64-bit draw of a primed stream */
uint64_t or_draw(const uint32_t sk[2], uint64_t loc, uint64_t tkey, uint32_t tag, uint32_t idx)
{
    uint64_t v[2];
    or_draw_pair(sk, loc, tkey, tag, idx / 2u, v);
    return v[idx % 2u];
}

static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((u128)a * (u128)b) >> 64);
}

/* ------------------------------------------------------------------------
 * Exp(1) by inverse transform, X = -ln(U), U = (r + 1) / 2^53 in (0, 1],
 * r = the top 53 bits of a draw.  ln is evaluated in fixed point:
 *   n = r + 1 = 2^e * m,  m in [1, 2)
 *   -ln U = (53 - e) ln 2 - ln m
 *   ln m = ln(2^32 / R_j) + ln(1 + s),  1 + s = m R_j / 2^32
 * where the 12 fraction bits after the leading one of m select j, R_j is a
 * 32-bit reciprocal of the bucket midpoint (so |s| < 2^-12.9), L_j =
 * ln(2^32/R_j) comes from a table, and
 *   ln(1 + s) = s - s^2 (1/2 - s/3 + s^2/4)
 * (the series to s^4; the s^5/5 term is below 2^-66) is evaluated with s in
 * signed Q0.64 and the bracket in Q2.62.  The result is rounded half up to
 * Q6.58 and converted to double.  Tables (inputs): L_j = round(2^62 ln(2^32 /
 * R_j)), ln2_q64 = round(2^64 ln 2), c3 = round(2^64 / 3).
 * ------------------------------------------------------------------------ */
#define OR_LN_BITS 12
typedef struct {
    uint64_t ln_tab[1 << OR_LN_BITS];
    uint64_t ln2_q64;
    int64_t c3;
} or_ln_tables;

uint32_t or_ln_recip(uint32_t j)
{
    /* round(2^45 / (8193 + 2j)), ties up */
    uint64_t d = 8193u + 2u * (uint64_t)j;
    return (uint32_t)(((1ull << 46) + d) / (2u * d));
}

/* floor(a b / 2^64) for signed a, b */
static int64_t mulhi_s(int64_t a, int64_t b)
{
    return (int64_t)(((i128)a * (i128)b) >> 64);
}

/* the fixed-point value of -ln((r + 1) 2^-53) in units of 2^-58 */
uint64_t or_exp1_q58(uint64_t r53, const or_ln_tables* T)
{
    uint64_t n = r53 + 1u;                 /* 1 .. 2^53 */
    int e = 63 - __builtin_clzll(n);       /* floor(log2 n) */
    uint64_t M = n << (63 - e);            /* m * 2^63 */
    uint32_t j = (uint32_t)((M >> (63 - OR_LN_BITS)) & ((1u << OR_LN_BITS) - 1u));
    u128 P = (u128)M * (u128)or_ln_recip(j);             /* (1 + s) 2^95 */
    int64_t s = (int64_t)(uint64_t)(P >> 31);            /* Q0.64, wraps to s */
    int64_t s2 = mulhi_s(s, s);                           /* s^2, Q0.64 */
    int64_t s3 = mulhi_s(s, T->c3);                       /* s/3, Q0.64 */
    int64_t t = ((int64_t)1 << 61) - (s3 >> 2) + (s2 >> 4); /* 1/2 - s/3 + s^2/4, Q2.62 */
    int64_t q = (int64_t)(((u128)(uint64_t)s2 * (u128)(uint64_t)t) >> 64); /* s^2 t, Q2.62 */
    int64_t ln1p = s - q * 4;                             /* ln(1 + s), Q0.64 */
    int64_t lnm = (int64_t)T->ln_tab[j] + (ln1p >> 2);    /* ln m, Q2.62 */
    i128 x64 = (i128)(53 - e) * (i128)T->ln2_q64 - (i128)lnm * 4;
    if (x64 < 0)
        x64 = 0;
    return (uint64_t)(((u128)x64 + 32u) >> 6);
}

double or_exp1(uint64_t draw, const or_ln_tables* T)
{
    uint64_t q = or_exp1_q58(draw >> 11, T);
    return (double)q * 0x1p-58;
}

/* ------------------------------------------------------------------------
 * Model
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;              /* OR_NONSPATIAL, OR_TORUS, OR_MAP */
    uint32_t width, height;    /* cells; 1 x 1 for the non-spatial model */
    uint32_t deme;             /* non-spatial: J; torus: individuals per cell;
                                  map: largest deme in deme_map */
    const uint8_t* deme_map;   /* map: width*height demes, 0 = not habitable */
    double lambda, delta_t, nu;
    uint64_t seed;
    /* torus: discretised-normal CDF per axis, 2*gauss_half entries,
     * gauss_cdf[k] = round(2^64 Phi((k - half + 1/2)/sigma)) clamped */
    int32_t gauss_half;
    const uint64_t* gauss_cdf;
    /* map: Gaussian kernel weights kw[d2] = round(2^32 exp(-d2/(2 sigma^2)))
     * for squared offsets d2 = 0..radius^2 */
    int32_t radius;
    const uint64_t* kw;
    const or_ln_tables* ln;
    /* event-time sampler: 0 = sums of exponentials, 1 = Poisson point counts
     * with uniform points; for 1, pois_cdf[n] = round(2^64 P(Poi(lambda
     * delta_t) <= n)) clamped, n = 0 .. pois_n - 1 */
    int32_t sampler;
    int32_t pois_n;
    const uint64_t* pois_cdf;
    /* spatially implicit: migration probability per event of a local
     * lineage, metacommunity size J_meta (<= 2^31) and its speciation
     * probability; the local community is the deme of J = deme individuals */
    double migration;
    uint64_t meta_size;
    double meta_nu;
} or_model;

static uint64_t pack_loc(uint64_t x, uint64_t y, uint64_t i)
{
    return x | (y << 20) | (i << 40);
}
static uint32_t loc_x(uint64_t l) { return (uint32_t)(l & 0xFFFFFu); }
static uint32_t loc_y(uint64_t l) { return (uint32_t)((l >> 20) & 0xFFFFFu); }
static uint32_t loc_i(uint64_t l) { return (uint32_t)(l >> 40); }

/* spatially implicit locations: local individual i at (0, 0, i);
 * metacommunity individual i at y = 1, with i's low 20 bits in x and the
 * rest in the deme index */
static int in_meta(uint64_t l) { return loc_y(l) == 1u; }
static uint64_t meta_loc(uint64_t i) { return pack_loc(i & 0xFFFFFu, 1, i >> 20); }
static uint64_t meta_index(uint64_t l) { return ((uint64_t)loc_i(l) << 20) | loc_x(l); }

static uint64_t dbl_bits(double d)
{
    uint64_t b;
    memcpy(&b, &d, 8);
    return b;
}

static uint32_t deme_at(const or_model* m, int64_t x, int64_t y)
{
    if (m->kind == OR_MAP)
        return m->deme_map[(uint64_t)y * m->width + (uint64_t)x];
    return m->deme;
}

static int64_t wrap(int64_t v, int64_t n)
{
    int64_t r = v % n;
    return r < 0 ? r + n : r;
}

/* first point of the location's event process strictly after tau
 * (memoryless sums inside re-prime intervals [k dt, (k+1) dt));
 * returns a negative value if an interval needs more than 2^20 draws */
static double next_event_time_poisson(const or_model* m, uint32_t sk[2], uint64_t loc, double tau);

static double next_event_time(const or_model* m, uint32_t sk[2], uint64_t loc, double tau)
{
    if (m->sampler == 1)
        return next_event_time_poisson(m, sk, loc, tau);
    double k = floor(tau / m->delta_t);
    for (;;) {
        double p = k * m->delta_t;
        double end = (k + 1.0) * m->delta_t;
        uint64_t tkey = (uint64_t)k;
        int found = 0;
        for (uint32_t idx = 0; idx < (1u << 20); idx++) {
            double x = or_exp1(or_draw(sk, loc, tkey, OR_TAG_INTERVAL, idx), m->ln);
            p = p + x / m->lambda;
            if (p >= end) {
                found = 1;
                break;
            }
            if (p > tau)
                return p;
        }
        if (!found)
            return -1.0;
        k = k + 1.0;
    }
}

/* Poisson method (section "Homogeneous Poisson Point Process"): interval k
 * of the location's process holds N ~ Poi(lambda delta_t) points, N = the
 * number of CDF thresholds <= draw 0 of the interval stream, placed
 * uniformly: point i (i = 0..N-1) is k dt + U dt with U = (draw (1 + i) >> 11)
 * 2^-53, the sum rounded to nearest.  The next event after tau is the
 * smallest point > tau of the first interval that has one. */
static double next_event_time_poisson(const or_model* m, uint32_t sk[2], uint64_t loc, double tau)
{
    double k = floor(tau / m->delta_t);
    for (uint64_t iv = 0; iv < (1ull << 26); iv++) {
        uint64_t tkey = (uint64_t)k;
        uint64_t r = or_draw(sk, loc, tkey, OR_TAG_INTERVAL, 0);
        uint32_t N = 0;
        for (int32_t n = 0; n < m->pois_n; n++)
            if (m->pois_cdf[n] <= r)
                N++;
        double base = k * m->delta_t;
        int found = 0;
        double best = 0.0;
        for (uint32_t i = 0; i < N; i++) {
            uint64_t d = or_draw(sk, loc, tkey, OR_TAG_INTERVAL, 1 + i);
            double p = base + (double)(d >> 11) * 0x1p-53 * m->delta_t;
            if (p > tau && (!found || p < best)) {
                best = p;
                found = 1;
            }
        }
        if (found)
            return best;
        k = k + 1.0;
    }
    return -1.0;
}

/* discretised normal per axis: the number of CDF thresholds <= r, shifted */
static int64_t gauss_offset(const or_model* m, uint64_t r)
{
    int64_t count = 0;
    for (int64_t k = 0; k < 2 * (int64_t)m->gauss_half; k++)
        if (m->gauss_cdf[k] <= r)
            count++;
    return count - m->gauss_half;
}

/* exact integer Vose alias table of one habitable origin cell of the map:
 * column o is the o-th disk offset in (dy, dx) row-major order, weight
 * kw[dx^2+dy^2] * deme(target) on the torus-wrapped map */
typedef struct {
    uint32_t n;
    int8_t dx[4096], dy[4096];
    uint32_t q[4096];
    uint16_t alias[4096];
    uint8_t full[4096];
} or_alias_row;

static void alias_build(const or_model* m, uint32_t cx, uint32_t cy, or_alias_row* row)
{
    static __thread uint64_t s[4096];
    static __thread uint32_t small_[4096], large_[4096];
    int32_t R = m->radius;
    uint32_t n = 0;
    for (int32_t dy = -R; dy <= R; dy++)
        for (int32_t dx = -R; dx <= R; dx++)
            if (dx * dx + dy * dy <= R * R) {
                row->dx[n] = (int8_t)dx;
                row->dy[n] = (int8_t)dy;
                n++;
            }
    row->n = n;
    uint64_t W = 0;
    for (uint32_t o = 0; o < n; o++) {
        int64_t tx = wrap((int64_t)cx + row->dx[o], m->width);
        int64_t ty = wrap((int64_t)cy + row->dy[o], m->height);
        uint64_t w = m->kw[row->dx[o] * row->dx[o] + row->dy[o] * row->dy[o]] *
                     (uint64_t)deme_at(m, tx, ty);
        s[o] = (uint64_t)n * w;
        W += w;
    }
    uint32_t ns = 0, nl = 0;
    for (uint32_t o = 0; o < n; o++) {
        if (s[o] < W)
            small_[ns++] = o;
        else
            large_[nl++] = o;
    }
    while (ns > 0 && nl > 0) {
        uint32_t a = small_[--ns];
        uint32_t b = large_[--nl];
        row->q[a] = (uint32_t)(((u128)s[a] << 32) / W);
        row->full[a] = 0;
        row->alias[a] = (uint16_t)b;
        s[b] = s[b] + s[a] - W;
        if (s[b] < W)
            small_[ns++] = b;
        else
            large_[nl++] = b;
    }
    while (nl > 0) {
        uint32_t b = large_[--nl];
        row->q[b] = 0xFFFFFFFFu;
        row->full[b] = 1;
        row->alias[b] = (uint16_t)b;
    }
    while (ns > 0) { /* unreachable with exact integer weights */
        uint32_t a = small_[--ns];
        row->q[a] = 0xFFFFFFFFu;
        row->full[a] = 1;
        row->alias[a] = (uint16_t)a;
    }
}

static uint32_t alias_sample(const or_alias_row* row, uint64_t r)
{
    uint32_t c = (uint32_t)(((r >> 32) * (uint64_t)row->n) >> 32);
    uint32_t u = (uint32_t)r;
    if (row->full[c] || u < row->q[c])
        return c;
    return row->alias[c];
}

/* the dispersal target of an event at loc, from the event stream's draws
 * v[1], v[2], v[3] (draw 0 decided speciation) */
static uint64_t disperse(const or_model* m, uint32_t sk[2], uint64_t loc, double tau)
{
    uint64_t tkey = dbl_bits(tau);
    uint64_t v[4];
    or_draw_pair(sk, loc, tkey, OR_TAG_EVENT, 0, v);
    or_draw_pair(sk, loc, tkey, OR_TAG_EVENT, 1, v + 2);
    if (m->kind == OR_NONSPATIAL)
        return pack_loc(0, 0, mulhi64(v[1], m->deme));
    if (m->kind == OR_IMPLICIT) {
        /* in the metacommunity: a uniform parent there (draw 1); locally:
         * migration iff draw 1 says so, then the parent's index (draw 2) in
         * the metacommunity or the local community */
        if (in_meta(loc))
            return meta_loc(mulhi64(v[1], m->meta_size));
        if ((v[1] >> 11) < (uint64_t)ceil(m->migration * 0x1p53))
            return meta_loc(mulhi64(v[2], m->meta_size));
        return pack_loc(0, 0, mulhi64(v[2], m->deme));
    }
    int64_t x = loc_x(loc), y = loc_y(loc);
    if (m->kind == OR_TORUS) {
        int64_t tx = wrap(x + gauss_offset(m, v[1]), m->width);
        int64_t ty = wrap(y + gauss_offset(m, v[2]), m->height);
        uint64_t ti = m->deme > 1 ? mulhi64(v[3], m->deme) : 0;
        return pack_loc((uint64_t)tx, (uint64_t)ty, ti);
    }
    static __thread or_alias_row row;
    alias_build(m, (uint32_t)x, (uint32_t)y, &row);
    uint32_t o = alias_sample(&row, v[1]);
    int64_t tx = wrap(x + row.dx[o], m->width);
    int64_t ty = wrap(y + row.dy[o], m->height);
    uint64_t ti = mulhi64(v[2], deme_at(m, tx, ty));
    return pack_loc((uint64_t)tx, (uint64_t)ty, ti);
}

static int speciates(const or_model* m, uint32_t sk[2], uint64_t loc, double tau)
{
    double nu = (m->kind == OR_IMPLICIT && in_meta(loc)) ? m->meta_nu : m->nu;
    double thr_d = ceil(nu * 0x1p53);
    uint64_t thr = (uint64_t)thr_d;
    uint64_t v0 = or_draw(sk, loc, dbl_bits(tau), OR_TAG_EVENT, 0);
    return (v0 >> 11) < thr;
}

/* Mode P: one lineage from loc0 at the present (tau = 0) until it speciates.
 * Returns 0 and the speciation key (location, IEEE bits of the time), or -1
 * if max_events were executed first, -2 on an interval overflow. */
int or_trace(const or_model* m, uint64_t loc0, uint64_t max_events, uint64_t* key_loc,
             uint64_t* key_time, uint64_t* n_events)
{
    uint32_t sk[2];
    or_seed_key(m->seed, sk);
    uint64_t loc = loc0;
    double tau = 0.0;
    for (uint64_t ev = 0; ev < max_events; ev++) {
        tau = next_event_time(m, sk, loc, tau);
        if (tau < 0.0)
            return -2;
        if (speciates(m, sk, loc, tau)) {
            *key_loc = loc;
            *key_time = dbl_bits(tau);
            *n_events = ev + 1;
            return 0;
        }
        loc = disperse(m, sk, loc, tau);
    }
    *n_events = max_events;
    return -1;
}

/* Mode P with an event log: the (location, time bits) of every event of the
 * lineage, in order, up to cap entries.  Returns the event count, or -1. */
int64_t or_trace_log(const or_model* m, uint64_t loc0, uint64_t cap, uint64_t* ev_loc,
                     uint64_t* ev_time)
{
    uint32_t sk[2];
    or_seed_key(m->seed, sk);
    uint64_t loc = loc0;
    double tau = 0.0;
    for (uint64_t ev = 0; ev < cap; ev++) {
        tau = next_event_time(m, sk, loc, tau);
        if (tau < 0.0)
            return -1;
        ev_loc[ev] = loc;
        ev_time[ev] = dbl_bits(tau);
        if (speciates(m, sk, loc, tau))
            return (int64_t)(ev + 1);
        loc = disperse(m, sk, loc, tau);
    }
    return -1;
}

/* threads a parallel loop of mode P may use (OpenMP's default team size) */
int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Mode P over many lineages (independent; parallel over lineages) */
int or_trace_many(const or_model* m, const uint64_t* loc0, uint64_t n, uint64_t max_events,
                  uint64_t* key_loc, uint64_t* key_time, uint64_t* n_events)
{
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : status)
    for (uint64_t s = 0; s < n; s++) {
        int st = or_trace(m, loc0[s], max_events, key_loc + s, key_time + s, n_events + s);
        if (st < status)
            status = st;
    }
    return status;
}

/* ------------------------------------------------------------------------
 * Mode M: all lineages, events in global time order, a lineage that
 * disperses onto an occupied slot merges into its occupant.
 * ------------------------------------------------------------------------ */
typedef struct {
    double t;
    uint64_t slot;
} or_heap_item;

static int heap_less(const or_heap_item* a, const or_heap_item* b)
{
    if (a->t != b->t)
        return a->t < b->t;
    return a->slot < b->slot;
}

static void heap_push(or_heap_item* h, uint64_t* n, or_heap_item it)
{
    uint64_t i = (*n)++;
    h[i] = it;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!heap_less(&h[i], &h[p]))
            break;
        or_heap_item tmp = h[i];
        h[i] = h[p];
        h[p] = tmp;
        i = p;
    }
}

static or_heap_item heap_pop(or_heap_item* h, uint64_t* n)
{
    or_heap_item top = h[0];
    h[0] = h[--(*n)];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, best = i;
        if (l < *n && heap_less(&h[l], &h[best]))
            best = l;
        if (r < *n && heap_less(&h[r], &h[best]))
            best = r;
        if (best == i)
            break;
        or_heap_item tmp = h[i];
        h[i] = h[best];
        h[best] = tmp;
        i = best;
    }
    return top;
}

static uint64_t slot_of(const or_model* m, uint64_t loc)
{
    if (m->kind == OR_IMPLICIT)
        return in_meta(loc) ? (uint64_t)m->deme + meta_index(loc) : loc_i(loc);
    return ((uint64_t)loc_y(loc) * m->width + loc_x(loc)) * (uint64_t)m->deme + loc_i(loc);
}

/* Returns 0, or -1 if more than max_events events were needed, -2 on an
 * interval overflow, -3 on an exact tie between a lineage's arrival time and
 * the occupant's pending event time (not handled), -4 on out-of-memory.
 * key_loc/key_time receive every lineage's species key; *n_unique the number
 * of events executed (each is unique). */
/* The event stream of mode M (section "Reporting Coalescence Events
 * Independently"): every executed event -- (time, the lineage's prior event
 * time, location, dispersal target or ~0 for a speciation, lineage) -- in
 * global time order, and every coalescence: a lineage (child) dispersing at
 * time t into the location of another (parent). */
typedef struct {
    uint64_t cap, n;
    uint64_t* time_bits;
    uint64_t* prior_bits;
    uint64_t* loc;
    uint64_t* target;
    int64_t* lineage;
    uint64_t co_cap, n_co;
    uint64_t* co_loc;
    uint64_t* co_time_bits;
    int64_t* co_parent;
    int64_t* co_child;
} or_event_log;

static int run_merge(const or_model* m, const uint64_t* loc0, uint64_t n, uint64_t max_events,
                     uint64_t* key_loc, uint64_t* key_time, uint64_t* n_unique, or_event_log* log,
                     uint64_t* longest);

int or_run_merge(const or_model* m, const uint64_t* loc0, uint64_t n, uint64_t max_events,
                 uint64_t* key_loc, uint64_t* key_time, uint64_t* n_unique)
{
    return run_merge(m, loc0, n, max_events, key_loc, key_time, n_unique, 0, 0);
}

/* mode M that also reports the longest line of descent: the most events any
 * one sampled individual's lineage runs before it speciates, which is the
 * longest mode-P trace.  A lineage carries the most events of any individual
 * it stands for; on a merge the occupant takes the larger of the two counts,
 * since from then on both groups share the occupant's events. */
int or_run_merge_longest(const or_model* m, const uint64_t* loc0, uint64_t n, uint64_t max_events,
                         uint64_t* key_loc, uint64_t* key_time, uint64_t* n_unique, uint64_t* longest)
{
    *longest = 0;
    return run_merge(m, loc0, n, max_events, key_loc, key_time, n_unique, 0, longest);
}

/* mode M with its event stream; -5 if the log's arrays are too small */
int or_run_merge_events(const or_model* m, const uint64_t* loc0, uint64_t n, uint64_t max_events,
                        uint64_t* key_loc, uint64_t* key_time, uint64_t* n_unique, or_event_log* log)
{
    log->n = log->n_co = 0;
    return run_merge(m, loc0, n, max_events, key_loc, key_time, n_unique, log, 0);
}

static int run_merge(const or_model* m, const uint64_t* loc0, uint64_t n, uint64_t max_events,
                     uint64_t* key_loc, uint64_t* key_time, uint64_t* n_unique, or_event_log* log,
                     uint64_t* longest)
{
    uint32_t sk[2];
    or_seed_key(m->seed, sk);
    uint64_t n_slots = m->kind == OR_IMPLICIT ? (uint64_t)m->deme + m->meta_size
                                               : (uint64_t)m->width * m->height * m->deme;
    int64_t* occupant = (int64_t*)malloc(n_slots * sizeof(int64_t));
    double* pending = (double*)malloc(n_slots * sizeof(double));
    uint64_t* loc_of = (uint64_t*)malloc(n * sizeof(uint64_t));
    int64_t* parent = (int64_t*)malloc(n * sizeof(int64_t));
    double* last = (double*)malloc(n * sizeof(double)); /* each lineage's prior event time */
    or_heap_item* heap = (or_heap_item*)malloc((n + 1) * sizeof(or_heap_item));
    uint64_t* depth = longest ? (uint64_t*)calloc(n, sizeof(uint64_t)) : 0;
    int status = 0;
    if (!occupant || !pending || !loc_of || !parent || !last || !heap || (longest && !depth)) {
        status = -4;
        goto done;
    }
    for (uint64_t s = 0; s < n_slots; s++)
        occupant[s] = -1;
    uint64_t hn = 0;
    for (uint64_t a = 0; a < n; a++) {
        uint64_t slot = slot_of(m, loc0[a]);
        parent[a] = -1;
        loc_of[a] = loc0[a];
        last[a] = 0.0;
        if (occupant[slot] >= 0) { /* duplicate sample location */
            parent[a] = occupant[slot];
            continue;
        }
        double t = next_event_time(m, sk, loc0[a], 0.0);
        if (t < 0.0) {
            status = -2;
            goto done;
        }
        occupant[slot] = (int64_t)a;
        pending[slot] = t;
        or_heap_item it = {t, slot};
        heap_push(heap, &hn, it);
    }
    uint64_t events = 0;
    while (hn > 0) {
        if (events >= max_events) {
            status = -1;
            goto done;
        }
        or_heap_item it = heap_pop(heap, &hn);
        int64_t a = occupant[it.slot];
        uint64_t loc = loc_of[a];
        double tau = it.t;
        occupant[it.slot] = -1;
        events++;
        if (depth)
            depth[a]++;
        int spec = speciates(m, sk, loc, tau);
        uint64_t target = spec ? ~0ull : disperse(m, sk, loc, tau);
        if (log) {
            if (log->n >= log->cap) {
                status = -5;
                goto done;
            }
            log->time_bits[log->n] = dbl_bits(tau);
            log->prior_bits[log->n] = dbl_bits(last[a]);
            log->loc[log->n] = loc;
            log->target[log->n] = target;
            log->lineage[log->n] = a;
            log->n++;
        }
        last[a] = tau;
        if (spec) {
            key_loc[a] = loc;
            key_time[a] = dbl_bits(tau);
            if (depth && depth[a] > *longest)
                *longest = depth[a];
            continue;
        }
        uint64_t ts = slot_of(m, target);
        if (occupant[ts] >= 0) {
            if (pending[ts] == tau) {
                status = -3;
                goto done;
            }
            parent[a] = occupant[ts];
            if (depth && depth[a] > depth[occupant[ts]])
                depth[occupant[ts]] = depth[a];
            if (log) {
                if (log->n_co >= log->co_cap) {
                    status = -5;
                    goto done;
                }
                log->co_loc[log->n_co] = target;
                log->co_time_bits[log->n_co] = dbl_bits(tau);
                log->co_parent[log->n_co] = occupant[ts];
                log->co_child[log->n_co] = a;
                log->n_co++;
            }
            continue;
        }
        double t = next_event_time(m, sk, target, tau);
        if (t < 0.0) {
            status = -2;
            goto done;
        }
        loc_of[a] = target;
        occupant[ts] = a;
        pending[ts] = t;
        or_heap_item nx = {t, ts};
        heap_push(heap, &hn, nx);
    }
    /* every merged lineage takes the key of the lineage it merged into */
    for (uint64_t a = 0; a < n; a++) {
        int64_t r = (int64_t)a;
        while (parent[r] >= 0)
            r = parent[r];
        key_loc[a] = key_loc[r];
        key_time[a] = key_time[r];
    }
    *n_unique = events;
done:
    free(occupant);
    free(pending);
    free(loc_of);
    free(parent);
    free(last);
    free(heap);
    free(depth);
    return status;
}

/* ------------------------------------------------------------------------
 * Inputs: habitat map and sample
 * ------------------------------------------------------------------------ */

/* seeded site-percolation habitat: cell (x, y) is habitable iff the top 53
 * bits of its first map draw are below ceil(p 2^53); its deme is then
 * 1 + mulhi(second draw, max_deme) */
void or_habitat(uint64_t map_seed, uint32_t width, uint32_t height, double p_habitable,
                uint32_t max_deme, uint8_t* deme_out)
{
    uint32_t sk[2];
    or_seed_key(map_seed, sk);
    uint64_t thr = (uint64_t)ceil(p_habitable * 0x1p53);
    for (uint64_t y = 0; y < height; y++)
        for (uint64_t x = 0; x < width; x++) {
            uint64_t v[2];
            or_draw_pair(sk, pack_loc(x, y, 0), 0, OR_TAG_MAP, 0, v);
            deme_out[y * width + x] =
                (v[0] >> 11) < thr ? (uint8_t)(1u + mulhi64(v[1], max_deme)) : 0;
        }
}

/* sampled individuals in (cell row-major, deme index) order: each one is
 * kept iff fraction >= 1 or the top 53 bits of its sample draw are below
 * ceil(fraction 2^53).  Returns the count; writes locations if out != 0. */
uint64_t or_sample(const or_model* m, double fraction, uint64_t sample_seed, uint64_t* out)
{
    uint32_t sk[2];
    or_seed_key(sample_seed, sk);
    uint64_t thr = (uint64_t)ceil(fraction * 0x1p53);
    uint64_t count = 0;
    for (uint64_t y = 0; y < m->height; y++)
        for (uint64_t x = 0; x < m->width; x++) {
            uint32_t d = deme_at(m, (int64_t)x, (int64_t)y);
            for (uint64_t i = 0; i < d; i++) {
                uint64_t loc = pack_loc(x, y, i);
                if (fraction < 1.0 && (or_draw(sk, loc, 0, OR_TAG_SAMPLE, 0) >> 11) >= thr)
                    continue;
                if (out)
                    out[count] = loc;
                count++;
            }
        }
    return count;
}

/* building blocks exposed for the oracle's own tests */
uint64_t or_gauss_offset(const or_model* m, uint64_t r) { return (uint64_t)gauss_offset(m, r); }
double or_next_event_time(const or_model* m, uint64_t loc, double tau)
{
    uint32_t sk[2];
    or_seed_key(m->seed, sk);
    return next_event_time(m, sk, loc, tau);
}
uint64_t or_disperse(const or_model* m, uint64_t loc, double tau)
{
    uint32_t sk[2];
    or_seed_key(m->seed, sk);
    return disperse(m, sk, loc, tau);
}
int or_speciates(const or_model* m, uint64_t loc, double tau)
{
    uint32_t sk[2];
    or_seed_key(m->seed, sk);
    return speciates(m, sk, loc, tau);
}
/* alias table of one cell: writes n entries of q, alias, full and offsets */
uint32_t or_alias_row_dump(const or_model* m, uint32_t cx, uint32_t cy, uint32_t* q,
                           uint16_t* alias, uint8_t* full, int8_t* dx, int8_t* dy)
{
    static __thread or_alias_row row;
    alias_build(m, cx, cy, &row);
    for (uint32_t o = 0; o < row.n; o++) {
        q[o] = row.q[o];
        alias[o] = row.alias[o];
        full[o] = row.full[o];
        dx[o] = row.dx[o];
        dy[o] = row.dy[o];
    }
    return row.n;
}
