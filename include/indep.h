/*
 * indep.h -- C ABI of the B300 (sm_103a) implementation of the Independent
 * algorithm for neutral biodiversity models (Langenstein 2021,
 * "Communication-free and Parallel Simulation of Neutral Biodiversity
 * Models").
 *
 * Every sampled individual's lineage is traced backwards in time on its own
 * (section "The Independent Algorithm"), driven by a counter-based RNG primed
 * on (seed, indexed location, time) (sections "Environmental RNG Priming" and
 * "Aligning the RNGs of Colliding Individuals"), with exponential inter-event
 * times drawn as memoryless sums inside re-prime intervals (section
 * "Memoryless sums of exponentials").  Lineages that meet draw identical
 * randomness afterwards; a device hash table culls the copies at common time
 * horizons (a device-side form of section "Deduplicating Redundant
 * Individuals" and of the water-level rounds of the appendix "The Independent
 * Water-Level Algorithm").  The species of an individual is the speciation
 * event its lineage ends in (section "A Neutral Coalescence-based
 * Simulation"); identities are dense ranks of the speciation keys
 * (location, IEEE-754 bits of the time) in ascending order.
 *
 * Conventions
 *  - Every entry point returns an ind_status; nothing throws or aborts.
 *  - The library owns all device state of a simulation; it allocates it on
 *    the simulation's stream through the process-wide allocator hook
 *    (ind_set_allocator), by default cudaMallocAsync.  The caller owns every
 *    buffer it passes in; input buffers are copied before the call returns.
 *  - All device work is issued on the stream given to sim_create (NULL = the
 *    legacy default stream).  Calls that return results to the host
 *    synchronise that stream.
 *  - Pointers documented as "host or device" may be either (unified virtual
 *    addressing); results are written with cudaMemcpyDefault.
 *  - Results are bit-identical for a given (landscape, dispersal, nu, seed,
 *    sample): they do not depend on tuning, batching, dedup cadence or the
 *    order in which the GPU executes lineages.
 */
#ifndef INDEP_H
#define INDEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ind_sim ind_sim;

typedef enum {
    IND_OK = 0,
    IND_ERR_ARG = -1,    /* invalid argument; nothing was changed */
    IND_ERR_OOM = -2,    /* the allocator failed; the object is unchanged */
    IND_ERR_CUDA = -3,   /* a CUDA runtime call failed (see ind_last_cuda_error) */
    IND_ERR_BUDGET = -4, /* sim_run used its round budget; call it again to resume */
    IND_ERR_STATE = -5,  /* call out of order (e.g. species before the run ended) */
    IND_ERR_DEVICE = -6  /* a device-side limit was hit (more than 2^20 draws in one
                            re-prime interval, 2^26 empty intervals crossed in one
                            search, or a full hash table); results are not valid */
} ind_status;

/* landscape kinds */
enum { IND_NONSPATIAL = 0, IND_TORUS = 1, IND_MAP = 2, IND_IMPLICIT = 3 };
/* dispersal kinds */
enum { IND_DISPERSAL_UNIFORM = 0, IND_DISPERSAL_GAUSSIAN = 1, IND_DISPERSAL_ALIAS_GAUSSIAN = 2 };

/* Landscape (section "Three Neutral scenarios").
 *  IND_NONSPATIAL: one deme of J = deme individuals (width = height = 1),
 *    dispersal uniform over all J indexed locations, the parent's own
 *    included; requires IND_DISPERSAL_UNIFORM.
 *  IND_TORUS: width x height cells of deme individuals each, wrapped;
 *    requires IND_DISPERSAL_GAUSSIAN.
 *  IND_MAP: width x height cells, deme_map[y * width + x] individuals in each
 *    (0 = not habitable), wrapped; requires IND_DISPERSAL_ALIAS_GAUSSIAN.
 *  IND_IMPLICIT: the spatially implicit scenario (section "Spatially
 *    Implicit"): a local community of J = deme individuals (width = height
 *    = 1), closed by a static metacommunity of meta_size individuals.  At
 *    an event of a local lineage the stream's draw 0 decides speciation
 *    (nu), draw 1 migration (probability `migration`), and draw 2 the
 *    parent's index: uniform over the metacommunity after a migration,
 *    else uniform over the J local individuals (the parent's own included).
 *    In the metacommunity, draw 0 decides speciation (meta_nu) and draw 1
 *    picks a uniform metacommunity parent; lineages never return.  Local
 *    individual i sits at location (0, 0, i); metacommunity individual i at
 *    x = i mod 2^20, y = 1, deme index i >> 20.  Only local individuals are
 *    sampled.  Requires IND_DISPERSAL_UNIFORM; 0 <= migration <= 1;
 *    1 <= meta_size <= 2^31; 0 < meta_nu <= 1; nu may be 0 here (but not
 *    together with migration = 0).
 * Limits: width, height <= 2^20; deme <= 2^23 - 1 (non-spatial J likewise);
 * width * height * deme < 2^32 (map: width * height * 255); lambda > 0 and
 * finite; delta_t a power of two in [2^-20, 2^20]; lambda * delta_t >= 2^-20.
 * A search that crosses 2^26 empty re-prime intervals, or draws 2^20 times in
 * one interval, stops the run with IND_ERR_DEVICE. */
typedef struct {
    int32_t kind;
    uint32_t width, height;
    uint32_t deme;
    const uint8_t* deme_map; /* IND_MAP only: host or device pointer, copied */
    double lambda;           /* turnover rate: events per unit time per lineage */
    double delta_t;          /* re-prime interval length */
    /* event-time sampler (both give Exp(lambda) inter-event times; they are
     * different random streams):
     *  IND_SAMPLER_EXP: points of a re-prime interval are running sums of
     *    Exp(lambda) draws (section "Memoryless sums of exponentials");
     *  IND_SAMPLER_POISSON: N ~ Poi(lambda delta_t) points placed uniformly
     *    in the interval (section "Homogeneous Poisson Point Process");
     *    requires lambda * delta_t <= 64. */
    int32_t event_sampler;
    /* IND_IMPLICIT only (ignored otherwise): */
    double migration;   /* probability that a local lineage's parent lives in the metacommunity */
    uint64_t meta_size; /* metacommunity individuals */
    double meta_nu;     /* speciation probability per event in the metacommunity */
} ind_landscape;

enum { IND_SAMPLER_EXP = 0, IND_SAMPLER_POISSON = 1 };

/* Dispersal (DispersalSampler of section "The Statically Checked Component
 * System"; the intra-deme index is uniform, CoalescenceSampler).
 *  IND_DISPERSAL_GAUSSIAN: each axis moves by round(sigma z), z ~ N(0, 1),
 *    sampled by inversion of the discretised normal CDF quantised to 2^-64;
 *    0 < sigma <= 64.
 *  IND_DISPERSAL_ALIAS_GAUSSIAN: per habitable cell, an alias table over the
 *    disk dx^2 + dy^2 <= radius^2 with weights
 *    round(2^32 exp(-(dx^2 + dy^2)/(2 sigma^2))) * deme(target); 1 <= radius
 *    <= 40. */
typedef struct {
    int32_t kind;
    double sigma;
    uint32_t radius;
} ind_dispersal;

typedef struct {
    uint64_t rounds;        /* horizon rounds executed so far */
    uint64_t raw_events;    /* events executed on the GPU, duplicates included */
    uint64_t unique_events; /* distinct (location, time) events; exact only when
                               counting was enabled (ind_tuning.count_unique) */
    uint64_t culled;        /* lineages removed by the horizon dedup */
    uint64_t n_sampled;     /* lineages started */
    uint64_t n_species;     /* species count (after sim_species) */
    uint64_t n_roots;       /* lineages that ended in a speciation event */
    double ms_total;        /* wall time of the sim_run calls (host clock) */
    double advance_ms;      /* summed advance-kernel time (profile = 1 only) */
    uint64_t advance_launches; /* advance-kernel launches timed (profile = 1 only) */
    double busiest_launch_ms;       /* profile = 1: the advance launch with the highest */
    uint64_t busiest_launch_events; /* event rate of the run: its time and events (all sims) */
    uint64_t critical_events; /* sum over rounds of the most events one lineage ran in the round:
                                 the dependent chain the rounds' durations are bound by (of the
                                 whole batch for sim_batch_run; 0 for served requests) */
    /* horizon-dedup inserts (exact only with ind_tuning.count_unique, else 0;
     * of the whole batch for sim_batch_run): all inserts, those that found
     * their slot already entered, and those another active lane of the same
     * warp inserted with the same slot in the same instruction */
    uint64_t dedup_inserts;
    uint64_t dedup_repeats;
    uint64_t dedup_warp_repeats;
} ind_run_stats;

/* Event stream (section "Reporting Coalescence Events Independently").
 * With an event log (sim_set_event_log), sim_run records every event it
 * executes, copies of not yet culled lineages included, and when the run
 * ends reduces the record on the device: sorted by (event time, location,
 * prior event time, lineage), the copies of one event are adjacent; the
 * first is kept (one entry per distinct event), and every later copy with
 * a prior time of its own is a lineage that dispersed into the location at
 * that time: a coalescence with the lineage of the first copy.  A lineage
 * removed by the horizon dedup leaves a copy of its pending event (with its
 * own prior time), so that no coalescence is lost to the dedup. */
#define IND_SPECIATION UINT64_MAX
typedef struct {
    uint64_t time_bits;  /* event time: IEEE-754 bits of tau >= 0 */
    uint64_t prior_bits; /* the executing lineage's previous event time (0: the present) */
    uint64_t loc;        /* location of the event */
    uint64_t target;     /* dispersal target, or IND_SPECIATION */
    uint32_t lineage;    /* a sampled individual (sampling order) whose lineage executes it */
    uint32_t reserved;
} ind_event;

typedef struct {
    uint64_t loc;       /* where the child dispersed to: the parent's location */
    uint64_t time_bits; /* the child's dispersal time */
    uint32_t parent;    /* sampled individual whose lineage was at loc */
    uint32_t child;     /* sampled individual whose lineage arrived */
} ind_coalescence;

/* Tuning of the engine.  None of it changes results (bit-identical). */
typedef struct {
    uint32_t block_threads;     /* advance-kernel threads per block: 64..512, multiple of 32 */
    uint32_t blocks_per_sm;     /* persistent grid = blocks_per_sm x SM count, 1..32 */
    uint32_t lineages_per_lane; /* lineages a warp claims per lane at a time, 1..64 */
    uint32_t rounds_per_check;  /* horizon rounds between host completion checks, 1..4096 */
    uint32_t use_graph;         /* 1: replay each chunk of rounds as a captured CUDA graph */
    uint32_t dedup;             /* 1: horizon dedup (default); 0: none */
    uint32_t count_unique;      /* 1: count distinct events exactly (slower, for measurement) */
    uint32_t profile;           /* 1: time every advance-kernel launch with CUDA events */
    uint32_t events_per_visit;  /* events a lane runs on its lineage between warp votes, 1..1024 */
    uint32_t coop_lineages;     /* at most this many active lineages: one warp per lineage (0: never); with
                                   more (advance_variant 1), the lineages with 256 or more events before
                                   the horizon still run one per warp when they fit the warp grid */
    uint32_t advance_variant;   /* more active lineages: 1 (default) = one lineage per lane, events in a
                                   loop; 0 = convergent state machine (one Philox block per lane per step,
                                   kept as an option: slower on B300 on every workload measured) */
    uint32_t reserved;
    /* horizon step of a simulation with n active lineages over S indexed
     * locations: lambda * step = max(floor, min(occupancy_step * S / n,
     * events_per_round / n)), floor = tail_events while n < busy_lineages
     * (the GPU is latency-bound and duplicates cost no time), else
     * min_events_per_lineage.  In a batch the level is then shared: a
     * simulation's lambda * step is raised to min(occupancy_step * S / n,
     * the largest lambda * step of the batch's live simulations) when that
     * is more, since a round lasts as long as its busiest simulation needs.
     * Where the live simulations mix landscape kinds, that level and
     * max_step_events are counted in time: a simulation of a kind whose
     * events cost more (relative costs 0.65 non-spatial and spatially
     * implicit, 0.84 torus, 1.04 habitat map, measured on B300) takes them
     * scaled by the least live kind's cost over its own.
     * None of this changes any result, only how much work a round does. */
    double events_per_round;       /* water level: target events per simulation per round */
    double min_events_per_lineage; /* lower bound of lambda x horizon step */
    double occupancy_step;         /* alpha: duplicate work per round stays near alpha / 2 */
    double tail_events;            /* lower bound of lambda x horizon step below busy_lineages */
    double busy_lineages;          /* active lineages that fill the GPU */
    double max_step_events;        /* upper bound of lambda x horizon step while several
                                      simulations share the rounds (no round waits long on one
                                      simulation's few lineages); a simulation alone in its batch
                                      is bounded 16 times higher */
} ind_tuning;

typedef struct {
    /* returns a device allocation of at least bytes, ordered on stream, or NULL */
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*release)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} ind_allocator;

/* Process-wide device allocator hook, used for all later allocations
 * (NULL restores cudaMallocAsync / cudaFreeAsync).  Not thread-safe with
 * concurrent library calls. */
ind_status ind_set_allocator(const ind_allocator* allocator);

/* Defaults of the tuning. */
void ind_default_tuning(ind_tuning* out);

/* Create a simulation: validates the arguments, copies the deme map,
 * derives the stream key from seed, and builds the dispersal tables on the
 * device (for IND_MAP: one alias row per habitable cell, 8 bytes per disk
 * offset).  nu is the speciation probability per event, 0 < nu <= 1 (IND_IMPLICIT:
 * the local community's, 0 <= nu <= 1).
 * cuda_stream is a cudaStream_t (NULL: legacy default stream). */
ind_status sim_create(const ind_landscape* landscape, const ind_dispersal* dispersal, double nu,
                      uint64_t seed, void* cuda_stream, ind_sim** out);

/* Choose the sampled individuals and reset all lineages to the present:
 * individual (cell, i) is sampled iff fraction >= 1 or the top 53 bits of its
 * sample draw (stream key of sample_seed, tag SAMPLE) are below
 * ceil(fraction 2^53).  Individuals are numbered in (cell row-major, i)
 * order.  0 < fraction <= 1.  *n_sampled receives the count (may be NULL). */
ind_status sim_sample(ind_sim* sim, double fraction, uint64_t sample_seed, uint64_t* n_sampled);

/* Isolated partitions (the IsolatedIndividuals and IsolatedLandscape
 * strategies of the paper's parallel Independent algorithm, section "The
 * Independent Algorithm" of its parallelisation chapter, configured as in
 * the appendix "Parallelism with Isolated Batches", and run at scale in
 * section "Biodiversity Simulation Limit Analysis"): the sampled
 * individuals of one simulation are split into n_parts disjoint parts, each
 * simulated on its own (one per GPU, or one after another) with no
 * communication; lineages of different parts that meet are simulated twice.
 * Because every lineage of the Independent algorithm depends only on
 * (seed, location, time), an individual's speciation key is the same in its
 * part as in the whole simulation, so the only exchange is a merge of the
 * parts' distinct keys into global species identities at the end
 * (ind_keys_unique, ind_keys_rank).
 *   IND_PARTITION_LANDSCAPE: part p holds the individuals of the cells in the
 *     rows y with floor(y n_parts / height) == p (horizontal bands; lineages
 *     that stay near their band rarely meet another part's);
 *   IND_PARTITION_INDIVIDUALS: part p holds the sampled individuals whose
 *     index j in the whole sample's order has j mod n_parts == p. */
#define IND_PARTITION_LANDSCAPE 0
#define IND_PARTITION_INDIVIDUALS 1

/* sim_sample restricted to part `part` (0 <= part < n_parts) of the sample
 * under `scheme`: the part's individuals in the whole sample's order.
 * n_parts = 1 is sim_sample.  IND_ERR_ARG for part >= n_parts, n_parts = 0 or
 * an unknown scheme. */
ind_status sim_sample_partition(ind_sim* sim, double fraction, uint64_t sample_seed, uint32_t part,
                                uint32_t n_parts, int32_t scheme, uint64_t* n_sampled);

/* The distinct speciation keys among n (location, time-bits) pairs, sorted
 * ascending by (location, time bits), into out_loc / out_time (n entries of
 * room each) and their count into *n_out (host).  Inputs and outputs are
 * device pointers, owned by the caller; n <= 2^31.  Scratch comes from the
 * allocator hook (IND_ERR_OOM if it fails).  Work is issued on `stream` and
 * finished before return.  Section "A Neutral Coalescence-based
 * Simulation": a species is a distinct speciation event. */
ind_status ind_keys_unique(const uint64_t* key_loc, const uint64_t* key_time, uint64_t n, uint64_t* out_loc,
                           uint64_t* out_time, uint64_t* n_out, void* stream);

/* The global species identity of each of n keys: its index among n_ref
 * distinct reference keys sorted ascending (the output of ind_keys_unique
 * over every part's distinct keys), into rank_out[n].  Device pointers,
 * caller-owned; a key missing from the reference gives IND_ERR_ARG (its
 * entry is UINT64_MAX).  Issued on `stream`, finished before return. */
ind_status ind_keys_rank(const uint64_t* key_loc, const uint64_t* key_time, uint64_t n, const uint64_t* ref_loc,
                         const uint64_t* ref_time, uint64_t n_ref, uint64_t* rank_out, void* stream);

/* Enable the event log of the next run (capacity: raw events the device may
 * hold, duplicates and one entry per deduplicated lineage included,
 * 1..2^31) or disable it (0).  Costs 36 bytes per
 * raw event plus 16 per lineage; a run that executes more events than the
 * capacity fails with IND_ERR_DEVICE.  sim_run and sim_batch_run log; in a
 * batch, every simulation has a log or none does (else IND_ERR_ARG), the
 * batch shares one record of the summed capacities (at most 2^31), and each
 * simulation receives its own events and coalescences, its lineages
 * numbered as it samples them.  srv_submit rejects a simulation with a log
 * (IND_ERR_ARG). */
ind_status sim_set_event_log(ind_sim* sim, uint64_t capacity);

/* After a logged run: the distinct events in (time, location) order and the
 * coalescences in the same order.  Up to cap / co_cap entries are written
 * (host or device pointers; NULL: counts only); *n_events and
 * *n_coalescences (either may be NULL) receive the totals.  IND_ERR_STATE
 * before the run has finished or without a log. */
ind_status sim_events(ind_sim* sim, ind_event* out, uint64_t cap, uint64_t* n_events, ind_coalescence* co_out,
                      uint64_t co_cap, uint64_t* n_coalescences);

/* Run horizon rounds until every lineage has speciated or round_budget
 * rounds were executed in this call (0 = unlimited); IND_ERR_BUDGET means
 * "not finished yet" and the next call resumes.  out may be NULL. */
ind_status sim_run(ind_sim* sim, uint64_t round_budget, ind_run_stats* out);

/* After a finished run: species identity per sampled individual (dense rank
 * of its speciation key, 0 .. n_species-1) into species_id_out[n_sampled]
 * (host or device; may be NULL), and the count into *n_species_out (may be
 * NULL). */
ind_status sim_species(ind_sim* sim, uint64_t* species_id_out, uint64_t* n_species_out);

/* After a finished run: the speciation key of every sampled individual:
 * location loc = x | y << 20 | i << 40 and the IEEE-754 bits of the
 * speciation time, into arrays of n_sampled entries (host or device). */
ind_status sim_species_keys(ind_sim* sim, uint64_t* key_loc_out, uint64_t* key_time_out);

/* Tuning of a simulation (copied); NULL restores the defaults. */
ind_status sim_set_tuning(ind_sim* sim, const ind_tuning* tuning);

/* Cumulative statistics of a simulation. */
ind_status sim_stats(const ind_sim* sim, ind_run_stats* out);

/* Upper bound of the device bytes a simulation of this shape holds after
 * sim_create + sim_sample(fraction) + sim_run (admission control);
 * 0 for invalid arguments. */
size_t sim_mem_estimate(const ind_landscape* landscape, const ind_dispersal* dispersal,
                        double fraction);

/* Free a simulation and its device state (stream-ordered). NULL is a no-op. */
void sim_destroy(ind_sim* sim);

/* Run n sampled simulations together in one persistent advance kernel per
 * round until all have finished, then resolve their species.  Each sim must
 * be sampled and not yet run; they may have different landscapes, sizes,
 * nu and dispersal.  Work is issued on the stream of sims[0]; tuning NULL =
 * sims[0]'s tuning.  per_sim (n entries, may be NULL) receives each
 * simulation's statistics.  Afterwards sim_species works on each sim. */
ind_status sim_batch_run(ind_sim** sims, uint32_t n, const ind_tuning* tuning,
                         ind_run_stats* per_sim);

/* ------------------------------------------------------------------------
 * Continuous-batching server.
 * Simulations (requests) are submitted while others run.  At every step the
 * server admits queued requests in arrival order while their
 * sim_mem_estimate fits in the HBM budget and a slot is free, appends their
 * lineages to the resident batch (each request keeps its own horizon, so a
 * newcomer starts at the present while others are deep in the past), runs a
 * chunk of horizon rounds of one persistent advance kernel over all resident
 * lineages, and retires the requests that finished: their species are
 * resolved on a second stream, overlapping the next rounds, and become
 * available through sim_species / sim_species_keys.  Results are
 * bit-identical to running each request alone.
 * ------------------------------------------------------------------------ */
typedef struct ind_server ind_server;

typedef struct {
    uint64_t submitted, admitted, finished;  /* requests so far */
    uint64_t queued, resident;               /* requests waiting / on the GPU */
    uint64_t resident_lineages;              /* active lineages after the last step */
    uint64_t bytes_admitted;                 /* sum of sim_mem_estimate of resident requests */
    uint64_t rounds;                         /* horizon rounds run */
    uint64_t raw_events;                     /* events executed by retired requests */
    uint64_t lineage_capacity;               /* resident-lineage capacity of the buffers */
} ind_server_stats;

/* The server's default tuning: ind_default_tuning with a higher water level
 * for requests with many lineages (occupancy_step 1, min_events_per_lineage
 * 1, events_per_round 2^24), since a shared round lasts as long as the
 * heaviest lineage in it runs.  Results do not depend on it. */
void srv_default_tuning(ind_tuning* tuning);

/* hbm_budget: bytes that resident requests may hold (their sim_mem_estimate
 * summed); the lineage buffers are sized from it.  max_sims: resident
 * requests at most (1..65536).  tuning NULL = srv_default_tuning.  All work runs on
 * cuda_stream (resolution of finished requests on a stream of the server's
 * own that waits for it). */
ind_status srv_create(uint64_t hbm_budget, uint32_t max_sims, const ind_tuning* tuning, void* cuda_stream,
                      ind_server** out);

/* Queue a created and sampled simulation that has not run yet; the server
 * does not take ownership (destroy it after it finished or after
 * srv_destroy).  *ticket (may be NULL) receives the submission number. */
ind_status srv_submit(ind_server* srv, ind_sim* sim, uint64_t* ticket);

/* Admit what fits, run up to `rounds` horizon rounds (>= 1) if anything is
 * resident, then retire finished requests: up to cap tickets of requests
 * finished in this step go to finished[] (host), their count to
 * *n_finished.  Tickets beyond cap are reported by later calls. */
ind_status srv_step(ind_server* srv, uint32_t rounds, uint64_t* finished, uint32_t cap, uint32_t* n_finished);

ind_status srv_stats(const ind_server* srv, ind_server_stats* out);

/* Free the server's device state.  Requests still resident are abandoned
 * (their sim_species returns IND_ERR_STATE). NULL is a no-op. */
void srv_destroy(ind_server* srv);

/* Synthetic habitat map (seeded site percolation): cell (x, y) is habitable
 * iff the top 53 bits of the first draw of its map stream (stream key of
 * map_seed, location x | y << 20, time 0, tag MAP) are below
 * ceil(p_habitable 2^53); its deme is then 1 + mulhi64(second draw,
 * max_deme).  deme_out: width * height bytes, row-major, host or device;
 * 1 <= max_deme <= 255.  Work runs on cuda_stream; returns after it ends. */
ind_status ind_habitat(uint64_t map_seed, uint32_t width, uint32_t height, double p_habitable,
                       uint32_t max_deme, uint8_t* deme_out, void* cuda_stream);

/* Conformance probe of the device arithmetic (no counterpart in the paper;
 * used by the tests): for each 64-bit input v[i], exp_q58_out[i] receives the
 * fixed-point -ln U of U = ((v[i] >> 11) + 1) 2^-53 in units of 2^-58, and
 * philox_out[4i..4i+3] the Philox4x32-10 block with key (lo, hi of v[i]) and
 * counter (lo, hi of v[i+1 mod n], lo, hi of v[i+2 mod n]).  Either output may
 * be NULL; all pointers host or device; 1 <= n <= 2^30. */
ind_status ind_selftest(const uint64_t* in, uint64_t n, uint64_t* exp_q58_out, uint32_t* philox_out,
                        void* cuda_stream);

/* Conformance probe of the event-time searches (no counterpart in the
 * paper; used by the tests).  For each i, out[i] receives the first point
 * strictly after tau[i] of the event process at location loc[i] of
 * simulation m (its seed, sampler, lambda and delta_t; sections "Memoryless
 * sums of exponentials" and "Homogeneous Poisson Point Process" under
 * "Exponential inter-event Times"), computed by search form `form`: 0 and 1 the
 * one-lane searches as the one-lane kernel runs them (one or two draw blocks
 * per step; integer sums for lambda = 1 and integer Poisson points), 2 the
 * warp-cooperative general search, 3 the short warp search in binary64, 4
 * the short warp search as the tail kernel runs it (integer sums for lambda
 * = 1), 5 the one-lane search in binary64 throughout.  Every form returns
 * the same value; a negative value reports a search
 * beyond the interval limits (IND_ERR_DEVICE in a run).  tau[i] >= 0
 * finite; loc[i] any packed location.  Pointers host or device, owned by
 * the caller; 1 <= n <= 2^26; runs on m's stream and returns after it. */
ind_status sim_selftest_search(ind_sim* m, int form, const uint64_t* loc, const double* tau, uint64_t n,
                               double* out);

/* The alias row of habitable cell (x, y) of a map simulation, as the device
 * built it (inspection and tests; the dispersal of the section "Spatially
 * Explicit Scenario with Maps", sampled through one alias table per
 * habitable cell as in the paper's map benchmarks).  Entry o of the row is
 * column o of the cell's integer
 * Vose table over the dispersal kernel's offsets (row-major (dy, dx) within
 * the radius), packed in 64 bits: threshold q (bits 0-31; column o is taken
 * iff the 32 low bits of the draw are below q), the alias column's offset
 * dx (bits 32-38) and dy (39-45) as 7-bit two's complement, the deme of
 * column o's target cell (46-53) and of the alias column's target cell
 * (54-61), and bit 63 set when column o is always taken (its alias is then
 * itself).  *n_out
 * receives the number of columns; with out == NULL that is all the call
 * does.  out (host or device, caller-owned) holds cap >= *n_out entries.
 * IND_ERR_ARG for a simulation that is not a map, a cell outside the map or
 * without habitat, or a short buffer. */
ind_status sim_alias_row(ind_sim* m, uint32_t x, uint32_t y, uint64_t* out, uint32_t cap, uint32_t* n_out);

/* Species ranking that allocates nothing (the paper has no counterpart: it
 * exists for callers that must not allocate device memory while they run,
 * e.g. a process that plans all of its device memory at start-up, or code
 * running inside an allocator of its own that it cannot re-enter).
 * Computes, for n individuals with speciation keys (key_loc[i],
 * key_time[i]), the dense species identity of each (rank of its key among
 * the distinct keys in ascending (location, time bits) order) into
 * species_out[i] and the number of distinct keys into *n_species_out: the
 * same values sim_species gives for those keys.
 *  - key_loc, key_time, species_out: device-accessible pointers of n entries;
 *    n_species_out: host or device pointer (may be NULL).
 *  - n <= 65536; larger n returns IND_ERR_ARG without doing anything.
 *  - Its scratch is one fixed device array of about 2.5 MiB that every GPU
 *    loading this library holds until the process exits; no cudaMalloc,
 *    cudaFree or allocating library routine is called.
 *  - The first call on a device looks up that array's device address (with
 *    the device current); make that first call before any stream capture.
 *  - All calls share the array and it keeps the last call's contents: calls
 *    whose work overlaps on the GPU race and give wrong results.
 *  - Work runs on cuda_stream; returns after it ends if n_species_out is set. */
ind_status ind_species_rank_static(const uint64_t* key_loc, const uint64_t* key_time, uint64_t n,
                                   uint64_t* species_out, uint64_t* n_species_out, void* cuda_stream);

/* Human-readable status name; never NULL. */
const char* ind_status_string(ind_status status);

/* The last CUDA error code seen by the library (cudaError_t as int). */
int ind_last_cuda_error(void);

/* Number of library kernel launches since the process started (for
 * accounting). */
uint64_t ind_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* INDEP_H */
