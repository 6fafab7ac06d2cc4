/*
 * pa.h -- C ABI of the GB300 population-annealing engine for the 2D
 * ferromagnetic Ising model (Barash, Weigel, Borovsky, Janke, Shchur,
 * "GPU accelerated population annealing algorithm", arXiv:1703.03676), with
 * the further models the paper's conclusion points to: the +-J spin glass
 * (pa_create_couplings), the simple cubic lattice (pa_config.dim = 3) and
 * the q-state Potts model (pa_config.potts_q).
 *
 * One pa_ctx is one PA run (Sec. 2.1): R replicas of a periodic L x L Ising
 * lattice (Eq. hamiltonian, J = 1) start from random spins at beta0 = 0 and
 * are annealed to beta_f. Every temperature step resamples the population
 * with the nearest-integer copy numbers of Eq. resampling-factors (normaliser
 * Eq. Q), runs theta checkerboard Metropolis sweeps per replica (Sec. 3,
 * "Spin updates", Fig. 1) and measures the population (Eq. observables,
 * Eq. free-energy, Eq. entropy). Steps are fixed (beta_i = i * dbeta) or
 * adaptive (Sec. 2.3); multi-histogram reweighting follows Sec. 2.4.
 *
 * Conventions shared by every entry point:
 *  - All pointers named host_* or typed as host arrays are host memory owned
 *    by the caller; the context owns all device memory it allocates.
 *  - No call aborts, traps or prints. Every call returns a pa_status; a
 *    failed call leaves the context valid for pa_destroy and for reading the
 *    rows completed before the failure.
 *  - Results are a pure function of pa_config: they do not depend on the
 *    stream, on CUDA-graph use, on the thread-group shape or on batching.
 *  - Work is enqueued on the stream given to pa_create (NULL: a stream the
 *    context creates). Calls that return data synchronise that stream.
 */
#ifndef PA_GB300_H
#define PA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pa_ctx pa_ctx;

typedef enum {
    PA_OK = 0,
    PA_DONE = 1,          /* pa_step: beta_f already reached, nothing done      */
    PA_EAGAIN = 2,        /* pa_step_async: the previous step is still running  */
    PA_EINVAL = -1,       /* invalid argument or configuration                  */
    PA_ENOMEM = -2,       /* device or host allocation failed                   */
    PA_ECAPACITY = -3,    /* R_i exceeded the population capacity               */
    PA_EEXTINCT = -4,     /* R_i == 0                                           */
    PA_ETIMEOUT = -5,     /* a bounded device wait ran out                      */
    PA_ECUDA = -6,        /* a CUDA runtime call failed                         */
    PA_ESTATE = -7,       /* call not valid in the context's current state      */
    PA_ESTALLED = -8      /* adaptive step found no positive step size          */
} pa_status;

/* PA_SPIN_INT8: one byte per spin. PA_SPIN_BITS32: 32 same-colour sites of
 * one replica per word (synchronous multi-spin coding). Both draw one
 * Philox4x32-10 word per attempt and give identical results (the Potts
 * model uses PA_SPIN_INT8 with states 0..q-1 and two words per attempt).
 * PA_SPIN_MSC32: the paper's asynchronous multi-spin coding (Sec. 4): bit j
 * of a site's word is replica 32g + j, and the 32 replicas' random numbers
 * come from the linear congruential generator r <- 1664525 r + 1013904223
 * (mod 2^32) seeded per (group g, site b, sweep u, colour c) by the Philox
 * word at counter (2u + c, b>>2, 5, g), lane b&3; replica bit j uses the
 * (j+1)-th output. A different random-number contract (its own oracle
 * mode); L in {4, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64, 96, 128}; not in
 * batches.
 * PA_SPIN_REPLICA8: the paper's replica-parallel layout (Sec. 3): one thread
 * per replica walks the lattice, byte spins stored with the replica index
 * fastest; the generic fallback for models without a domain decomposition.
 * Same contract as PA_SPIN_INT8 / PA_SPIN_BITS32 (identical results). */
typedef enum { PA_SPIN_INT8 = 0, PA_SPIN_BITS32 = 1, PA_SPIN_MSC32 = 2, PA_SPIN_REPLICA8 = 3 } pa_spin_format;

typedef enum { PA_HIST_E = 0, PA_HIST_M = 1, PA_HIST_ESUM = 2 } pa_hist_kind;

/* Run parameters (Sec. 3 "Further optimization and parameters": R, theta,
 * beta0, beta_f, the seed; plus the step rule of Sec. 2.1 / 2.3). */
typedef struct {
    int32_t L;              /* lattice edge, even, 4 <= L <= 1024. PA_SPIN_BITS32
                               needs L in {8, 16, 32, 64, 128, 256, 512}         */
    int32_t theta;          /* Metropolis sweeps per temperature step, >= 1       */
    int64_t R;              /* target population size, >= 1                      */
    double beta0;           /* must be 0 (Z_beta0 = 2^N, Eq. free-energy)         */
    double beta_f;          /* final inverse temperature, 0 < beta_f <= 50        */
    double dbeta;           /* > 0: fixed step; <= 0: adaptive step (Sec. 2.3)    */
    double overlap;         /* adaptive target alpha*, 0 < alpha* < 1             */
    uint64_t seed;          /* Philox4x32-10 key (low word, high word)            */
    int32_t spin_format;    /* pa_spin_format                                     */
    int32_t record_histograms; /* != 0: keep H_E and H_M of every step            */
    int64_t capacity;       /* population buffer size; 0 -> ceil(1.05 R) + 1024   */
    int32_t group_threads;  /* threads per replica in the sweep: 1..32 (power of
                               two dividing the plane's words) or 256 (one
                               replica per CTA, bit-packed); 0 -> default       */
    int32_t use_graph;      /* != 0: pa_run captures the fixed schedule as one
                               CUDA graph                                       */
    int32_t profile;        /* != 0: time every kernel phase with CUDA events     */
    int32_t dim;            /* 0 or 2: the L x L square lattice (Sec. 3); 3: the
                               L x L x L simple cubic lattice, N = L^3, with
                               PA_SPIN_BITS32 and L in {8, 16, 32, 64} only
                               (one of the further models the paper's
                               conclusion names; energy levels k = (E + 3N)/4
                               = 0 .. 3N/2, so every histogram has 3N/2 + 1
                               entries; magnetisation levels use the first
                               N + 1)                                           */
    int32_t potts_q;        /* 0: Ising spins; 2..8: the q-state Potts model,
                               H = -sum over bonds of delta(s_i, s_j) (a further
                               model the paper's conclusion names), square
                               lattice, PA_SPIN_INT8 only (byte states 0..q-1).
                               Energy levels k = E + 2N = 0 .. 2N (histograms of
                               2N + 1 entries); the "magnetisation" M is the
                               number of sites in the most populated state
                               (levels m = M); Z at beta0 = 0 is q^N. The
                               update proposes a uniform other state and
                               accepts by Metropolis on dE = n(s) - n(s')   */
    int32_t block_warps;    /* warps per CTA of the warp-group sweeps (group_threads
                               <= 32): 1, 2, 4 or 8; 0 -> 8 (fewer when one
                               warp's replicas need much shared memory). With
                               group_threads == 0 and block_warps == 0 the
                               launch shape is the one pa_autotune chose for
                               runs like this one in this process, if any,
                               else a fixed rule                            */
} pa_config;

/* One output row (Sec. 3 "Further optimization and parameters": beta, e, C,
 * m, m^2, m^4, beta F / N, S / N, R, ln Q), plus the number of distinct
 * families (initial replicas that still have descendants). */
typedef struct {
    double beta, e, C, abs_m, m2, m4, betaF_per_N, S_per_N, lnQ;
    int64_t R;
    int64_t families;
} pa_obs;

/* Per-step bookkeeping for tests: what the resampling of step `step` used. */
typedef struct {
    double beta;            /* beta_i                                             */
    double delta;           /* beta step used in Q and tau_hat                    */
    double S;               /* sum_k H_{i-1}[k] exp(-4 delta (k - kmin)), pairwise */
    int64_t R;              /* R_i                                                */
    int64_t R_prev;         /* R_{i-1}                                            */
    int32_t kmin_prev;      /* lowest occupied energy level of population i-1     */
    int32_t kmin, kmax;     /* occupied level range of population i               */
    int32_t pad;
    uint64_t T4, T8;        /* Metropolis thresholds ceil(exp(-4/8 beta_i) 2^32)  */
    int64_t families;
} pa_step_info;

/* Create a run and generate its beta0 population (row 0). `cuda_stream` is
 * a cudaStream_t borrowed for the context's lifetime, or NULL.
 * A population of at most 16384 slots of capacity takes two launches per
 * temperature step (resampling, sweep), each launched with programmatic
 * dependent launch so that it is scheduled while the one before it runs and
 * starts work when that one completes; the environment variable PA_PDL=0,
 * read here, launches them one after the other instead (same results).
 * Errors: PA_EINVAL (bad config), PA_ENOMEM, PA_ECUDA. */
pa_status pa_create(const pa_config *cfg, void *cuda_stream, pa_ctx **out);

/* Create a run of the +-J (Edwards-Anderson) model: quenched couplings
 * shared by every replica, H = -sum_{x,y} (Jr[y L + x] s(x,y) s(x+1,y) +
 * Jd[y L + x] s(x,y) s(x,y+1)) with every J = +1 or -1 (host arrays of
 * L*L int8 each; all +1 is the ferromagnet). The paper's method applies
 * unchanged (Sec. 1, Sec. 6: disordered systems): a neighbour is aligned
 * when J s_i s_j = +1, so dE = 4n - 8 and the acceptance rule, Q and the
 * resampling are as for the ferromagnet. The number of negative couplings
 * must be even (then (E + 2N)/4 is an integer). PA_SPIN_BITS32 and
 * PA_SPIN_INT8 only. */
pa_status pa_create_couplings(const pa_config *cfg, const int8_t *Jr, const int8_t *Jd, void *cuda_stream,
                              pa_ctx **out);

/* Create a run that follows a given schedule beta_1 < ... < beta_n (host
 * array betas[n], 0 < beta_i <= 50), with step i using
 * delta_i = beta_i - beta_{i-1} in Q and tau_hat. Sec. 2.3: with M runs the
 * adaptive schedule is decided in the first run and kept for the others
 * (pass that run's row betas). cfg->dbeta, overlap and beta_f are ignored.
 * Steps run like adaptive ones (one histogram readback per step). */
pa_status pa_create_scheduled(const pa_config *cfg, const double *betas, int64_t n, void *cuda_stream,
                              pa_ctx **out);

/* Combine M independent runs (Sec. 2.2, Eq. weighted-average): rows is the
 * host array of M x n rows (run-major) of runs of N = L*L spins sharing the
 * same betas. At each beta the weights are exp(-beta F_m) normalised, with
 * -beta F_m = -N (beta F / N)_m; e, |m|, m^2, m^4 are averaged; C comes from
 * the weighted <e> and <e^2> = C_m / (beta^2 N) + e_m^2 (beta > 0); the
 * combined -beta F = ln((1/M) sum_m Z_m); S/N = beta e - beta F / N; R and
 * families are summed; lnQ is NaN. Host-only (no GPU needed). PA_EINVAL if
 * the betas differ by more than 1e-12 relative. */
pa_status pa_weighted_average(const pa_obs *rows, int32_t m, int64_t n, int32_t N, pa_obs *out);

/* One temperature step (Sec. 2.1 steps 2-4). Fixed steps only enqueue work;
 * adaptive steps synchronise once to read the previous histogram.
 * Returns PA_DONE if beta_f was already reached. Device-side failures
 * (capacity, extinction) are reported by this call or the next one that
 * synchronises. */
pa_status pa_step(pa_ctx *ctx);

/* Non-blocking pa_step: enqueues the next step and returns PA_OK, or
 * PA_EAGAIN without doing anything if an adaptive run still waits for the
 * previous step's histogram (it streams to pinned host memory as soon as the
 * step ends), or PA_DONE once the last step is enqueued. Fixed steps never
 * return PA_EAGAIN. */
pa_status pa_step_async(pa_ctx *ctx);

/* Steps until beta_f and synchronises. With use_graph the remaining fixed
 * schedule runs as one CUDA-graph launch. */
pa_status pa_run(pa_ctx *ctx);

/* Enqueue the rest of the schedule and return without waiting (adaptive
 * runs still synchronise once per step). A fixed schedule started from step
 * 0 with use_graph runs as one CUDA-graph launch, captured on first use and
 * reused after pa_reset. */
pa_status pa_launch(pa_ctx *ctx);

/* Start the run again from step 0 with a new seed, keeping every device
 * allocation (and a captured graph): histograms, records and the status are
 * cleared and the beta0 population is regenerated from `seed`. */
pa_status pa_reset(pa_ctx *ctx, uint64_t seed);

/* Wait for enqueued work and report any device-side failure. */
pa_status pa_sync(pa_ctx *ctx);

/* Number of completed rows (row 0 is beta0). Synchronises. */
pa_status pa_num_rows(pa_ctx *ctx, int64_t *n_rows);

/* Copy up to `cap` rows into host `rows`; *n_rows gets the number copied. */
pa_status pa_observables(pa_ctx *ctx, pa_obs *rows, int64_t cap, int64_t *n_rows);

/* Step bookkeeping of completed step `step` (0 <= step < rows). */
pa_status pa_step_info_get(pa_ctx *ctx, int64_t step, pa_step_info *out);

/* Histogram of nlev entries into host `out` (cap >= nlev), where nlev =
 * N + 1 on the square lattice (N = L*L), 3N/2 + 1 on the simple cubic one
 * (N = L^3) and 2N + 1 for the Potts model (levels k = E + 2N):
 * PA_HIST_E: energy levels k = (E + dim N)/4 of step `step`;
 * PA_HIST_M: magnetisation levels m = (M + N)/2 of step `step` (entries
 * above N are 0);
 * PA_HIST_ESUM: sum of the energy histograms of steps 0..last (Sec. 2.4;
 * `step` ignored). Per-step kinds need record_histograms, else PA_ESTATE
 * (the latest step is always available). */
pa_status pa_histogram(pa_ctx *ctx, int64_t step, int32_t kind, int64_t *out, int64_t cap);

/* Current population in natural layout: host_out[r*N + y*L + x] = +1 / -1
 * (simple cubic: host_out[r*N + (z*L + y)*L + x]; Potts: the state 0..q-1)
 * for replica slot r < *n (cap is in replicas). */
pa_status pa_population(pa_ctx *ctx, int8_t *host_out, int64_t cap, int64_t *n);

/* 64-bit FNV-1a hash of the current population in the layout of
 * pa_population (one byte per spin, 0x01 for +1 and 0xff for -1, replica
 * after replica): a fingerprint for parity checks. */
pa_status pa_population_hash(pa_ctx *ctx, uint64_t *out);

/* Current per-replica energies, magnetisations and family ids. */
pa_status pa_replicas(pa_ctx *ctx, int32_t *E, int32_t *M, int64_t *family, int64_t cap, int64_t *n);

/* Multi-histogram reweighting (Sec. 2.4, Eq. MHReq1) over all completed
 * rows, evaluated at n inverse temperatures: out[t] gets beta, e, C,
 * beta F / N, S / N and the magnetisation moments |m|, m^2, m^4 (Sec. 2.4
 * notes the generalisation to magnetisations: the Boltzmann weight depends
 * on E only, so sum_M Omega(E, M) f(M) = Omega(E) (sum of f(M) over every
 * sample at level E) / Hsum(E)); lnQ is NaN, R and families 0. */
pa_status pa_mhr(pa_ctx *ctx, const double *betas, int64_t n, pa_obs *out);

/* The per-level magnetisation sums behind pa_mhr, over all measured replicas
 * of all completed steps: out[5k + 0] = sum |M|, out[5k + 1..2] = sum M^2
 * (low, high 64 bits), out[5k + 3..4] = sum M^4 (low, high), for energy
 * levels k = 0..nlev-1 (cap >= 5 nlev; nlev as for pa_histogram). */
pa_status pa_mag_sums(pa_ctx *ctx, uint64_t *out, int64_t cap);

/* ln Omega(E_k), E_k = 4k - dim N, for k = 0..nlev-1 from Eq. MHReq1 (-inf
 * where never visited; cap >= nlev as for pa_histogram). */
pa_status pa_ln_dos(pa_ctx *ctx, double *out, int64_t cap);

/* Accumulated device time in ms of each kernel phase (needs profile != 0):
 * [0] tables (Q and copy tables), [1] counts, [2] scan, [3] parent scatter,
 * [4] sweep, [5] stats, [6] init; launches[p] gets the launch count. A run
 * whose capacity is at most 16384 replicas resamples in one single-CTA
 * launch per step, counted under [0] (tables, copy numbers, scan and
 * parents, plus the previous step's statistics when the whole schedule is
 * enqueued at once by pa_run or pa_launch). The events themselves add a few
 * microseconds per launch: a small run's profiled time is well above its
 * unprofiled one. */
pa_status pa_phase_times(pa_ctx *ctx, double ms[7], int64_t launches[7]);

/* Number of this library's kernels launched for the run since pa_create
 * (a replay of the captured schedule counts every kernel node it runs). */
pa_status pa_kernel_launches(pa_ctx *ctx, int64_t *n);

/* The sweep launch shape chosen for this run (threads per replica, CTA size,
 * persistent CTAs). */
pa_status pa_launch_shape(pa_ctx *ctx, int32_t *group_threads, int32_t *block_threads, int32_t *grid_blocks);

/* Checkpoint at the current step boundary (Sec. 2.1 steps are independent
 * given the population: the random numbers are counter-based). Writes the
 * configuration, the host schedule and records, and the device state
 * (population, levels, families, current histograms, running sums) into
 * host_buf; *used gets the byte count. host_buf == NULL only reports the
 * size. Synchronises. PA_EINVAL if cap is too small. */
pa_status pa_checkpoint(pa_ctx *ctx, void *host_buf, size_t cap, size_t *used);

/* Resume from a checkpoint into a context created with the same
 * configuration (the seed, use_graph and profile may differ; the seed of
 * the checkpoint is used). Later steps are bit-identical to an
 * uninterrupted run. PA_EINVAL if the checkpoint does not match. */
pa_status pa_restore(pa_ctx *ctx, const void *host_buf, size_t n);

/* Device bytes a run with this configuration allocates (admission). */
size_t pa_footprint_bytes(const pa_config *cfg);

/* Default-initialise a config (every field zero except capacity rules). */
void pa_config_default(pa_config *cfg);

void pa_destroy(pa_ctx *ctx);
const char *pa_strerror(pa_status s);

/* Text of the last CUDA failure seen by a call on this thread (the CUDA
 * error name and the engine source line), or "" if none. */
const char *pa_last_error_message(void);

/* ---- autotuner ------------------------------------------------------------
 * The sweep's launch shape (threads per replica, warps per CTA) changes
 * only the speed of a run, never its results. pa_autotune times every shape
 * a run like cfg accepts on a two-step probe with cfg's lattice, format,
 * model and population size, and keeps the fastest; later pa_create calls in
 * the process whose config leaves the shape open (group_threads == 0 and
 * block_warps == 0) and that share the choice's key use it. Batches tune
 * their runs' threads per replica the same way (key batched = 1). Not part
 * of the paper (its kernels have a fixed shape): a deployment aid. */
typedef struct {
    int32_t L, spin_format, dim, potts_q;
    int32_t r_log2;         /* floor(log2 R): populations within a factor of 2 share a choice */
    int32_t batched;        /* 1: runs of a batch (the batched sweep), 0: runs alone */
    int32_t sms;            /* multiprocessors of the device                     */
    char gpu[64];           /* device name (no '|' or newline), NUL-terminated   */
} pa_tune_key;

typedef struct {
    int32_t group_threads;  /* chosen threads per replica                         */
    int32_t block_warps;    /* chosen warps per CTA (0: the default)              */
    double attempts_per_ns; /* sweep rate of the choice on its probe              */
    int32_t candidates;     /* shapes timed; 0 when read from a cache             */
    int32_t pad;
} pa_tune_choice;

/* The key of runs like cfg on the current device (name and SM count from
 * the CUDA runtime). Errors: PA_EINVAL, PA_ECUDA (no device). */
pa_status pa_tune_key_of(const pa_config *cfg, int32_t batched, pa_tune_key *out);

/* Tune (or recall) the launch shape of runs like cfg. The choice is kept
 * in the process and, with a cache file (cache_path, else the environment
 * variable PA_TUNE_CACHE, else none), read from and written to that text
 * file: one line per key, "v1|L|format|dim|potts_q|r_log2|batched|sms|gpu|
 * group_threads|block_warps|attempts_per_ns"; a known key is returned
 * without probing (candidates = 0). The probes allocate, run and free small
 * runs on `cuda_stream`. */
pa_status pa_autotune(const pa_config *cfg, const char *cache_path, void *cuda_stream, pa_tune_choice *out);

/* The cache file alone (host only, no device needed): store replaces the
 * line of the same key (written through a temporary file and a rename);
 * lookup sets *found to 1 and fills *out if the key is present, else 0.
 * Malformed lines are ignored. PA_EINVAL for a bad path, key or choice. */
pa_status pa_tune_cache_store(const char *path, const pa_tune_key *key, const pa_tune_choice *choice);
pa_status pa_tune_cache_lookup(const char *path, const pa_tune_key *key, pa_tune_choice *out, int32_t *found);

/* ---- batches of independent runs ---------------------------------------
 * Many independent fixed-schedule runs (batched runs; Sec. 2.2 notes
 * that independent runs combine by free-energy weights) stepped together:
 * every bookkeeping phase of a temperature step is one launch for all runs
 * (when every run's capacity is at most 16384, one launch of one CTA per run
 * for all of them, as a run alone takes one such CTA).
 * A run that fills the device alone (group_threads 256, one replica per
 * CTA at L = 128, 256, 512; or a warp-group run whose capacity needs at
 * least as many CTAs as the device keeps resident) is swept by its own sweep
 * kernel, the one it runs alone with. The other runs' sweep work queue
 * ((run, replica batch) items) is cut into segments of runs sharing (L,
 * group_threads), each ordered by descending work per replica and swept by
 * a persistent kernel compiled for that shape. The segments' kernels and
 * the own kernels (in turn on four streams) run on parallel branches of
 * the graph, so they overlap at their tails. The whole schedule
 * is one CUDA graph, captured on the first launch and reused after
 * pa_batch_reset.
 * Each run's results are those of the same pa_config run alone, bit for
 * bit. Runs must use fixed steps (dbeta > 0), bit-packed spins on the
 * square lattice and L <= 512 (L = 512: group_threads 256 only); group_threads == 0 picks the
 * threads per replica by a timed probe per L (cached per process), and an
 * unsupported group_threads gives PA_EINVAL. */
typedef struct pa_batch pa_batch;

/* Create n runs (their beta0 populations are generated). Errors as pa_create. */
pa_status pa_batch_create(const pa_config *cfgs, int32_t n, void *cuda_stream, pa_batch **out);
/* Enqueue every run's whole schedule (one graph launch) without waiting.
 * PA_ESTATE unless every run is at step 0. */
pa_status pa_batch_launch(pa_batch *b);
/* Wait for the batch; returns the first failing run's status (others keep
 * going and keep their rows). */
pa_status pa_batch_sync(pa_batch *b);
/* pa_batch_launch + pa_batch_sync. */
pa_status pa_batch_run(pa_batch *b);
/* Back to step 0 with seeds[i] for run i (host array of n seeds). */
pa_status pa_batch_reset(pa_batch *b, const uint64_t *seeds);
/* Borrow run i as a pa_ctx for read-only calls (observables, histograms,
 * population, MHR); stepping calls on it return PA_ESTATE and pa_destroy on
 * it does nothing. Valid until pa_batch_destroy. */
pa_status pa_batch_get(pa_batch *b, int32_t i, pa_ctx **out);
/* Accumulated device time per phase of the batched steps (needs profile in
 * any of the configs): [0] tables, [1] counts, [2] scan, [3] parent,
 * [4] plan + sweep, [5] stats. In a batch whose runs all have capacity
 * <= 16384, [0] is the one-CTA resampling of every run (with the previous
 * step's statistics), [1]-[3] stay empty and [5] is the last step's
 * statistics only. launches[p] counts the phase's launches. */
pa_status pa_batch_phase_times(pa_batch *b, double ms[7], int64_t launches[7]);
/* Threads per replica used for run i and the persistent grid size of the
 * sweep kernel that runs it (its own kernel, or its segment's kernel). */
pa_status pa_batch_shape(pa_batch *b, int32_t i, int32_t *group_threads, int32_t *sweep_blocks);
void pa_batch_destroy(pa_batch *b);

/* ---- serving ------------------------------------------------------------
 * A request loop with continuous batching (serving): requests
 * arrive at given times; arrived requests are admitted in arrival order
 * while fewer than max_active runs are resident and the sum of the
 * resident runs' pa_footprint_bytes stays within hbm_budget (a request
 * larger than the whole budget is admitted alone, once nothing else is
 * resident). A request that does not fit may be passed by up to max_bypass
 * later requests that do (0: strict arrival order); after that nothing more
 * is admitted before it, so a large request is never starved. Every
 * admitted run gets its own stream and stays resident on the device until
 * it finishes; the loop advances each run with pa_step_async, so the
 * kernels of different runs overlap on the GPU while others wait for their
 * host-side step decision, and a finished run frees its memory for the next
 * request. Runs allocate and free their device memory stream-ordered and
 * reuse pinned host buffers, so admitting or retiring a run does not
 * synchronise the device. Results are those of each request run alone. */
typedef struct {
    double arrival_s;       /* seconds after the loop starts                     */
    pa_config cfg;
} pa_request;

typedef struct {
    double admit_s;         /* seconds after the start: admitted (created)       */
    double finish_s;        /* all steps done and rows available                 */
    double attempts;        /* L^2 theta sum_{i>=1} R_i                          */
    int64_t steps;          /* temperature steps taken                           */
    int64_t footprint;      /* device bytes of the run                           */
    int32_t status;         /* pa_status of the run (PA_OK on success)           */
    int32_t pad;
} pa_request_result;

typedef struct {
    uint64_t hbm_budget;    /* bytes of resident runs, 0: no limit               */
    int32_t max_active;     /* resident runs at once, >= 1                       */
    int32_t keep;           /* != 0: return the finished contexts in out_ctx
                               (their memory stays allocated; the caller
                               destroys them) instead of destroying them        */
    double time_scale;      /* multiplies every arrival time (> 0)               */
    int32_t max_bypass;     /* later requests that may pass one that does not fit
                               (>= 0; 0: strict arrival order)                  */
    int32_t pad;
} pa_serve_options;

/* Serve n requests sorted by arrival time; returns when all are finished.
 * out[n] (host) gets per-request times and status; out_ctx[n] (host, only
 * with keep) the contexts. Returns PA_OK even if some requests failed (see
 * out[i].status); PA_EINVAL on bad arguments. */
pa_status pa_serve(const pa_request *reqs, int32_t n, const pa_serve_options *opt, pa_request_result *out,
                   pa_ctx **out_ctx);

/* ---- kernel-level entry points (device pointers, for tests) ----------- */

/* Philox4x32-10 on the device: out[4r..4r+3] = Philox(ctr[4r..4r+3], key =
 * (seed lo, seed hi)) for r < n. `dev_ctr` and `dev_out` are device
 * pointers of 4n uint32 each. Synchronous on `cuda_stream`. */
pa_status pa_philox_device(const uint32_t *dev_ctr, int64_t n, uint64_t seed, uint32_t *dev_out,
                           void *cuda_stream);

/* Nearest-integer resampling of one population on the device (Sec. 2.1,
 * Eq. resampling-factors, with the copy tables of Eq. Q): copy numbers
 * r_j = F[k_j] + [x_j < U[k_j]], where k_j = dev_levels[j] is the energy
 * level of old slot j and x_j the RESAMPLE word of slot j at step `step`
 * (Philox counter (step, j>>2, 2, 0), lane j&3, key = seed); their
 * exclusive scan; and dev_parent[o] = j for the r_j new slots o of each j,
 * in old-slot order. Device inputs: dev_levels[n_old] (0 <= k < n_levels),
 * dev_F[n_levels] = floor(tau_hat_k), dev_U[n_levels] = ceil(frac 2^32).
 * Device output: dev_parent[parent_cap]. Host output: *n_new = R_i.
 * Any F values are accepted (copy numbers and their sums are formed in 64
 * bits, so no total wraps); 1 <= n_old <= 2^31 and
 * 1 <= parent_cap <= 2^31. Scratch (about 8 bytes per old slot) is
 * allocated and freed inside the call. PA_ECAPACITY if R_i > parent_cap:
 * dev_parent is then left unwritten and *n_new is R_i, or 0 when the
 * copies of one 1024-slot tile alone already exceed parent_cap.
 * PA_EEXTINCT if R_i = 0, PA_EINVAL on bad sizes. Synchronous on
 * `cuda_stream` (NULL: the legacy default stream). */
pa_status pa_resample(const int32_t *dev_levels, int64_t n_old, const uint32_t *dev_F, const uint64_t *dev_U,
                      int64_t n_levels, uint64_t seed, int64_t step, uint32_t *dev_parent, int64_t parent_cap,
                      int64_t *n_new, void *cuda_stream);

/* Allocation-free pa_resample, for callers that must not allocate device
 * memory once they are running: a server whose device memory is fixed by
 * an admission budget, a host program whose device memory belongs to
 * another allocator (a framework's caching allocator) that a raw cudaMalloc
 * would bypass, or a loop where cudaMalloc/cudaFree would synchronise the
 * device and stall other streams. The paper has no counterpart: it is an
 * interface variant of pa_resample, with the same arguments, results and
 * errors. Its scratch is one static device array of the library
 * (PA_RESAMPLE_NOALLOC_MAX_OLD old slots: about 2 MiB, held on every GPU
 * that loads the library until the process exits); the caller still
 * provides the input and output buffers. n_old > PA_RESAMPLE_NOALLOC_MAX_OLD
 * returns PA_EINVAL (see pa_last_error_message). The first call on a device
 * looks up the array's device address with that device current; make that
 * first call before any stream capture. All calls share the one array, so
 * calls whose work overlaps on the GPU (several streams or threads at once)
 * race and give wrong results: serialise them. No call allocates or frees
 * device memory. */
#define PA_RESAMPLE_NOALLOC_MAX_OLD 262144
pa_status pa_resample_noalloc(const int32_t *dev_levels, int64_t n_old, const uint32_t *dev_F,
                              const uint64_t *dev_U, int64_t n_levels, uint64_t seed, int64_t step,
                              uint32_t *dev_parent, int64_t parent_cap, int64_t *n_new, void *cuda_stream);

/* The replica copy of the resampling step (Sec. 3, the resampling kernel's
 * copy of each selected replica) as a standalone kernel, for measuring it
 * against HBM bandwidth (the engine fuses this copy into the sweep's load):
 * dev_dst[o * words + w] = dev_src[dev_parent[o] * words + w] for
 * o < n_new, w < words. dev_src holds n_src replicas of `words` uint32
 * words (words a multiple of 4; dev_src and dev_dst 16-byte aligned, not
 * overlapping); dev_parent holds n_new old-slot indices. A parent >= n_src is
 * skipped (nothing read or written for that slot) and the call returns
 * PA_EINVAL after the copy. Allocates and frees a 4-byte flag. Synchronous
 * on `cuda_stream`; ms, if not NULL, gets the kernel's device time. */
pa_status pa_gather(const uint32_t *dev_src, int64_t n_src, const uint32_t *dev_parent, int64_t n_new, int32_t words,
                    uint32_t *dev_dst, void *cuda_stream, double *ms);

/* Throughput ceiling of the random-number generator alone: a persistent
 * kernel that evaluates Philox4x32-10 on `blocks_per_thread` counters per
 * thread over the whole device and XOR-folds the words (one store per
 * thread into the device buffer `dev_sink`, >= 4 bytes per thread of a
 * 152 x 2048-thread grid). *words_per_ns gets 4 x counters / elapsed ns.
 * Synchronous on `cuda_stream`. */
pa_status pa_measure_rng_peak(int64_t blocks_per_thread, uint32_t *dev_sink, void *cuda_stream,
                              double *words_per_ns);

/* Measured issue rate of one integer instruction class over the whole
 * device, the denominators behind the sweep's roofline: every thread of a
 * 152 x 2048-thread grid (SM count x 2048) runs eight independent dependency
 * chains for `iters` iterations (rounded down to a multiple of 4, >= 4) of
 *   pipe 0: 32x32->64 product by a constant, halves XORed (the
 *           Philox4x32-10 round, Sec. 3; the multiplies are counted),
 *   pipe 1: three-input logic op (the Philox XOR, the bit-sliced neighbour
 *           count), three per chain and iteration,
 *   pipe 2: 32-bit multiply-add (the accept-bit insert; the LCG of Sec. 4).
 * *lane_ops_per_ns gets instructions x threads / elapsed ns of the second of
 * two launches (the first warms up). `dev_sink` is a device buffer of >= 4
 * bytes per thread. Synchronous on `cuda_stream`; PA_EINVAL for a bad pipe
 * or iteration count. */
pa_status pa_measure_pipe_peak(int pipe, int64_t iters, uint32_t *dev_sink, void *cuda_stream,
                               double *lane_ops_per_ns);

/* Self-test of the bounded wait behind the sweep's bulk prefetch (the
 * one-replica-per-CTA sweep at L = 128 loads the next replica with a bulk
 * copy completed on a shared-memory barrier, and gives up with PA_ETIMEOUT
 * after a bounded number of polls instead of spinning on). One 32-thread
 * CTA arms the same barrier for `bytes` bytes (16..4096, a multiple of 16)
 * of a device pattern; with copy != 0 it issues the copy, with copy == 0
 * nothing ever delivers them. Every thread polls at most `tries` times
 * (>= 1). Returns PA_OK when the bytes landed and equal the pattern,
 * PA_ETIMEOUT when the wait ran out (nothing is left in flight and the
 * context stays usable), PA_ECUDA if they landed but differ, PA_EINVAL for
 * bad arguments. Allocates and frees its buffers; synchronous on
 * `cuda_stream`. */
pa_status pa_selftest_bulk_wait(int32_t bytes, int32_t copy, int32_t tries, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PA_GB300_H */
