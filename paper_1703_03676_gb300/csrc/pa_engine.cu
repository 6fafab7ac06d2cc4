// Host side of the population-annealing engine and the C ABI of include/pa.h.
//
// The host owns what is sequential and FP64 (Sec. 2.1-2.4): the inverse
// temperature schedule, the Metropolis thresholds ceil(exp(-4 beta) 2^32) and
// ceil(exp(-8 beta) 2^32), the level weights t[d] = exp(-4 delta d), the
// adaptive bisection on the histogram overlap (Sec. 2.3), ln Q, the
// free energy and entropy (Eq. free-energy, Eq. entropy), the observables
// (Eq. observables) from exact integer moment sums, and the multi-histogram
// estimate of the density of states (Eq. MHReq1). Every other step of the
// method runs in the kernels of pa_kernels.cu.
//
// This file must be compiled with -ffp-contract=off so that the FP64 tables
// are evaluated exactly as written (no fused multiply-add).
#include "../../include/pa.h"
#include "pa_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <cstring>
#include <thread>
#include <map>
#include <mutex>
#include <new>
#include <vector>

using pa::RunDev;
using pa::StepDev;

namespace {

constexpr long long kMaxAdaptiveSteps = 1 << 16;
constexpr long long kMaxRecordedHistSteps = 4096;

inline __int128 i128_of(const unsigned long long* p)
{
    return (__int128)(((unsigned __int128)p[1] << 64) | p[0]);
}

// smallest power of two >= n
inline long long pad_pow2(long long n)
{
    long long p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Pairwise tree (sum = left half + right half) over T[k] = H[k] w[k - kmin]
// for k in [kmin, kmax], zero elsewhere, on [lo, lo + n) with n a power of
// two. Subtrees outside [kmin, kmax] are exactly +0.0.
double tree_sum(const std::vector<long long>& H, const std::vector<double>& w, int kmin, int kmax, long long lo,
                long long n)
{
    if (lo + n <= kmin || lo > kmax) return 0.0;
    if (n == 1) return (double)H[(size_t)lo] * w[(size_t)(lo - kmin)];
    const double a = tree_sum(H, w, kmin, kmax, lo, n / 2);
    const double b = tree_sum(H, w, kmin, kmax, lo + n / 2, n / 2);
    return a + b;
}

// level weights exp(-(estep delta) d), d = 0..nd-1 (libm exp, one call each);
// estep is the energy between adjacent levels (4 Ising, 1 Potts)
void level_weights(double delta, int nd, std::vector<double>& w, int estep = 4)
{
    w.resize((size_t)nd);
    const double f = (double)estep * delta;
    for (int d = 0; d < nd; d++) w[(size_t)d] = std::exp(-(f * (double)d));
}

uint64_t threshold(double beta, double dE)
{
    return (uint64_t)std::ceil(std::ldexp(std::exp(-dE * beta), 32));
}

}  // namespace

struct pa_ctx {
    pa_config cfg{};
    RunDev h{};
    pa::Launch ln{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int N = 0;
    bool adaptive = false;
    long long n_fixed = 0;        // fixed schedule: number of steps
    long long max_steps = 0;      // record capacity (steps 0..max_steps)
    long long hist_steps = 0;     // steps with recorded histograms
    long long enq_step = 0;       // last step enqueued (0 = init)
    long long done_rows = 0;      // rows whose records are on the host
    bool done = false;            // beta_f reached
    pa_status failed = PA_OK;     // sticky device failure
    bool in_batch = false;        // stepped by a pa_batch, read-only for the caller
    std::vector<double> sched;    // given schedule beta_1..beta_n (empty: none)
    std::vector<double> betas;    // beta_i for i = 0..enq_step
    std::vector<double> deltas;   // step size used by step i (0 for i = 0)
    std::vector<uint64_t> T4, T8;
    std::vector<StepDev> recs;    // host copies of rec[0..done_rows)
    std::vector<void*> allocs;
    void* h_stage = nullptr;      // pinned staging for adaptive uploads
    size_t h_stage_bytes = 0;
    // adaptive runs: record, status and energy histogram of the last enqueued
    // step stream into pinned memory; ev_ready marks their arrival
    void* h_down = nullptr;
    size_t h_down_bytes = 0;
    cudaEvent_t ev_ready = nullptr;
    unsigned* d_key = nullptr;    // Philox key in device memory
    cudaGraphExec_t graph = nullptr;  // steps 1..n of the fixed schedule
    bool capturing = false;
    // profiling: (start, end) event pairs per kernel launch and its phase
    std::vector<cudaEvent_t> ev;  // plain launches, destroyed once read
    std::vector<int> ev_phase;
    std::vector<cudaEvent_t> gev; // owned by the graph, read after each launch
    std::vector<int> gev_phase;
    bool gev_pending = false;
    double phase_ms[7] = {0, 0, 0, 0, 0, 0, 0};
    long long phase_n[7] = {0, 0, 0, 0, 0, 0, 0};
    long long n_kern = 0;         // kernels of this library launched for the run
    long long graph_kern = 0;     // kernels in one launch of `graph`
    bool small_rs = false;        // capacity <= kSmallCap: one-CTA resampling launch per step
    bool pdl = false;             // small_rs steps: each launch may be scheduled while the one before
                                  // it runs (programmatic dependent launch; off with PA_PDL=0 and
                                  // when profiling events sit between the launches)
    bool stats_pending = false;   // statistics of the last enqueued step not yet launched
};

namespace {

thread_local char g_last_error[256] = "";

pa_status from_cuda(cudaError_t e, int line)
{
    if (e == cudaSuccess) return PA_OK;
    std::snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at pa_engine.cu:%d", cudaGetErrorName(e),
                  cudaGetErrorString(e), line);
    if (e == cudaErrorMemoryAllocation) return PA_ENOMEM;
    return PA_ECUDA;
}

#define PA_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return from_cuda(e_, __LINE__); \
    } while (0)

bool bits_L_ok(int L)
{
    return L == 8 || L == 16 || L == 32 || L == 64 || L == 128 || L == 256 || L == 512;
}

// simple cubic lattice, bit-packed: one L x L layer of a colour plane fills
// whole words (L^2 / 64 >= 1), a replica fits one CTA's shared memory
bool bits3_L_ok(int L)
{
    return L == 8 || L == 16 || L == 32 || L == 64;
}

bool msc_L_ok(int L)
{
    switch (L) {
    case 4: case 6: case 8: case 10: case 12: case 16: case 20: case 24: case 32: case 48: case 64: case 96:
    case 128: return true;
    default: return false;
    }
}

pa_status validate(const pa_config& c)
{
    if (c.L < 4 || c.L > 1024 || (c.L & 1)) return PA_EINVAL;
    if (c.theta < 1 || c.R < 1 || c.R > (1ll << 31)) return PA_EINVAL;
    if (c.beta0 != 0.0) return PA_EINVAL;
    if (!(c.beta_f > 0.0) || !(c.beta_f <= 50.0)) return PA_EINVAL;
    if (c.spin_format != PA_SPIN_INT8 && c.spin_format != PA_SPIN_BITS32 && c.spin_format != PA_SPIN_MSC32 &&
        c.spin_format != PA_SPIN_REPLICA8)
        return PA_EINVAL;
    if (c.spin_format == PA_SPIN_MSC32 && !msc_L_ok(c.L)) return PA_EINVAL;
    if (c.spin_format == PA_SPIN_BITS32 && !bits_L_ok(c.L)) return PA_EINVAL;
    if (!(c.dbeta > 0.0)) {
        if (!(c.overlap > 0.0 && c.overlap < 1.0)) return PA_EINVAL;
    } else {
        const double n = std::floor(c.beta_f / c.dbeta + 0.5);
        if (n < 1 || n > 1e7) return PA_EINVAL;
    }
    if (c.capacity < 0 || (c.capacity > 0 && c.capacity < c.R)) return PA_EINVAL;
    if (c.group_threads < 0 || (c.group_threads & (c.group_threads - 1))) return PA_EINVAL;
    if (c.group_threads > 32 && !(c.group_threads == 256 && c.spin_format == PA_SPIN_BITS32)) return PA_EINVAL;
    if (c.block_warps != 0 && c.block_warps != 1 && c.block_warps != 2 && c.block_warps != 4 && c.block_warps != 8)
        return PA_EINVAL;
    if (c.dim != 0 && c.dim != 2 && c.dim != 3) return PA_EINVAL;
    if (c.potts_q != 0 && (c.potts_q < 2 || c.potts_q > 8 || c.spin_format != PA_SPIN_INT8 || c.dim == 3))
        return PA_EINVAL;
    if (c.dim == 3 && (c.spin_format != PA_SPIN_BITS32 || !bits3_L_ok(c.L))) return PA_EINVAL;
    return PA_OK;
}

int dim_of(const pa_config& c)
{
    return c.dim == 3 ? 3 : 2;
}

// sites of the L x L torus, or of the L x L x L one (dim 3)
long long sites_of(const pa_config& c)
{
    return dim_of(c) == 3 ? (long long)c.L * c.L * c.L : (long long)c.L * c.L;
}

long long capacity_of(const pa_config& c)
{
    return c.capacity > 0 ? c.capacity : (long long)std::ceil((double)c.R * 1.05) + 1024;
}

int words_of(const pa_config& c)
{
    const long long N = sites_of(c);
    if (c.spin_format == PA_SPIN_BITS32) return (int)(N / 32);
    if (c.spin_format == PA_SPIN_MSC32) return (int)N;  // per group of 32 replicas
    if (c.spin_format == PA_SPIN_REPLICA8) return 0;    // site-major bytes, sized separately
    return (int)(((N + 15) / 16) * 4);  // bytes padded to 16, in words
}

// Byte spins of the square-lattice ferromagnet on a lattice the bit-packed
// kernels support are swept by those kernels (each replica packed into
// shared memory on load, unpacked on store); the population stays one byte
// per site in HBM.
bool packed_bytes(const pa_config& c, bool couplings)
{
    return c.spin_format == PA_SPIN_INT8 && c.potts_q == 0 && dim_of(c) == 2 && !couplings && bits_L_ok(c.L);
}

// a thread count the bit-packed square-lattice kernels accept for L
bool bits_group_valid(int L, int g)
{
    const int wp = L * L / 64;
    if (g < 1 || (g & (g - 1))) return false;
    if (g == 256) return wp % 256 == 0;
    return wp % g == 0 || (g <= 32 && g % wp == 0 && g / wp <= 8);
}

// threads per replica: enough to fill the device, a power of two dividing
// the plane's words (bit-packed) or the Philox blocks per plane (bytes)
int auto_group(const pa_config& c, bool bits_kernel)
{
    const long long N = sites_of(c);
    if (bits_kernel) {
        const long long wp = N / 64;
        // L >= 128: one replica per 256-thread CTA (measured faster than warp
        // groups: 1431 vs 1376 attempts/ns at L = 128, 1382 vs 1267 at L = 256)
        if (wp >= 256) return 256;
        int g = 32;
        while (g > 1 && wp % g) g >>= 1;
        // square lattices with few words per replica and a population too
        // small to occupy the device: up to 8 threads share each word's
        // Philox blocks, until the run has ~16 warps per SM
        if (dim_of(c) == 2)
            while (g < 32 && g < 8 * wp && c.R * 2 * g <= 152ll * 16 * 32) g <<= 1;
        return g;
    }
    const long long qp = (N / 2 + 3) / 4;
    int g = 1;
    while (g < 32 && g * 2 <= qp) g <<= 1;
    return g;
}

struct Sizes {
    long long cap, ntiles, steps, hist_steps;
    int N, words;
    int nlev;  // energy levels k = (E + dim N)/4 = 0 .. dim N/2; also the length of each histogram
};

Sizes sizes_of(const pa_config& c)
{
    Sizes s{};
    s.N = (int)sites_of(c);
    // Ising: (E + dim N)/4 = 0 .. dim N/2; Potts: E + 2N = 0 .. 2N
    s.nlev = (c.potts_q ? 2 * s.N : dim_of(c) * s.N / 2) + 1;
    s.cap = capacity_of(c);
    s.ntiles = (s.cap + pa::kTile - 1) / pa::kTile;
    s.words = words_of(c);
    if (c.dbeta > 0.0) s.steps = (long long)std::floor(c.beta_f / c.dbeta + 0.5);
    else s.steps = kMaxAdaptiveSteps;
    s.hist_steps = c.record_histograms ? std::min(s.steps + 1, kMaxRecordedHistSteps) : 0;
    return s;
}

size_t footprint(const pa_config& c)
{
    const Sizes s = sizes_of(c);
    const size_t N1 = (size_t)s.nlev;
    size_t b = 0;
    if (c.spin_format == PA_SPIN_REPLICA8) b += 2 * (((size_t)s.N * (size_t)s.cap + 3) / 4) * 4;
    else b += 2 * (size_t)(c.spin_format == PA_SPIN_MSC32 ? (s.cap + 31) / 32 : s.cap) * s.words * 4;  // pop
    b += 2 * (size_t)s.cap * 4 * 3;                 // elev, mlev, fam
    b += (size_t)s.cap * 4 * 3;                     // parent, cnt, loc
    b += 2 * (size_t)s.ntiles * 4;                  // tile sums / offsets
    b += 2 * 2 * N1 * 4;                            // H
    b += N1 * 8 * 3 + N1 * 4;                       // Hsum, tw, U, F
    b += N1 * 8 * 5;                                // magnetisation sums per level
    b += (size_t)(dim_of(c) == 3 ? 3 : (c.potts_q ? 6 : 2)) * (size_t)(s.steps + 1) * 4;  // thresholds
    b += (size_t)(s.steps + 1) * sizeof(StepDev);   // records
    b += (size_t)s.hist_steps * 2 * N1 * 4;         // recorded histograms
    b += 64;                                        // status + work
    return b;
}

// Device buffers of a run are stream-ordered allocations on the run's
// stream (cudaMallocAsync / cudaFreeAsync): creating or destroying a run
// does not synchronise the device, so runs resident beside it (serving,
// batches) keep running. pa_create synchronises its own stream once after
// allocating, before the host uploads its tables.
template <class T>
pa_status dev_alloc(pa_ctx* c, T** p, size_t count)
{
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMallocAsync(&q, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PA_ENOMEM : PA_ECUDA;
    }
    c->allocs.push_back(q);
    *p = (T*)q;
    return PA_OK;
}

#define PA_TRY(x)                        \
    do {                                 \
        pa_status s_ = (x);              \
        if (s_ != PA_OK) return s_;      \
    } while (0)

// Pinned host staging buffers, kept for reuse by later runs of the process
// (size classes of powers of two): freeing pinned memory synchronises the
// device, which would stall every other run's stream.
std::mutex g_pinned_mu;
std::multimap<size_t, void*> g_pinned_free;

size_t pinned_class(size_t bytes)
{
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
}

void* pinned_alloc(size_t bytes)
{
    const size_t cls = pinned_class(bytes);
    {
        std::lock_guard<std::mutex> g(g_pinned_mu);
        auto it = g_pinned_free.find(cls);
        if (it != g_pinned_free.end()) {
            void* p = it->second;
            g_pinned_free.erase(it);
            return p;
        }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, cls) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_release(void* p, size_t bytes)
{
    std::lock_guard<std::mutex> g(g_pinned_mu);
    g_pinned_free.emplace(pinned_class(bytes), p);
}

// ---------------------------------------------------------------- profiling
pa_status prof_record(pa_ctx* c, int phase)
{
    if (!c->cfg.profile) return PA_OK;
    cudaEvent_t a;
    PA_CUDA(cudaEventCreate(&a));
    // inside a capture the record must become a graph node (external event)
    PA_CUDA(cudaEventRecordWithFlags(a, c->stream, c->capturing ? cudaEventRecordExternal : 0u));
    if (c->capturing) {
        c->gev.push_back(a);
        c->gev_phase.push_back(phase);
    } else {
        c->ev.push_back(a);
        c->ev_phase.push_back(phase);
    }
    return PA_OK;
}

pa_status prof_begin(pa_ctx* c, int phase, cudaEvent_t* out)
{
    *out = nullptr;
    return prof_record(c, phase);
}

pa_status prof_end(pa_ctx* c)
{
    return prof_record(c, -1);
}

// accumulate the elapsed time of every completed (start, end) pair
pa_status prof_collect(pa_ctx* c)
{
    for (size_t i = 0; i + 1 < c->ev.size(); i += 2) {
        float ms = 0.f;
        PA_CUDA(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
        c->phase_ms[c->ev_phase[i]] += ms;
        c->phase_n[c->ev_phase[i]] += 1;
    }
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    c->ev_phase.clear();
    if (c->gev_pending) {
        for (size_t i = 0; i + 1 < c->gev.size(); i += 2) {
            float ms = 0.f;
            PA_CUDA(cudaEventElapsedTime(&ms, c->gev[i], c->gev[i + 1]));
            c->phase_ms[c->gev_phase[i]] += ms;
            c->phase_n[c->gev_phase[i]] += 1;
        }
        c->gev_pending = false;
    }
    return PA_OK;
}

#define PA_PHASE(ctx, ph, launch)                      \
    do {                                               \
        cudaEvent_t ev_;                               \
        PA_TRY(prof_begin(ctx, ph, &ev_));             \
        PA_CUDA(launch);                               \
        (ctx)->n_kern++;                               \
        PA_TRY(prof_end(ctx));                         \
    } while (0)

// ---------------------------------------------------------------- steps
// One temperature step. Small populations (capacity <= kSmallCap) resample
// in one single-CTA launch; larger ones in four (tables, counts, scan,
// parent). The statistics of the step run at once when stats_now (the host
// may read them next), else they are deferred into the next step's first
// launch (a whole schedule enqueued at once; its last step has stats_now).
pa_status enqueue_kernels(pa_ctx* c, int step, bool stats_now)
{
    const RunDev& h = c->h;
    if (c->small_rs) {
        PA_PHASE(c, 0, pa::launch_resample_small(h, step, c->stats_pending, c->stream, c->pdl));
    } else {
        if (c->stats_pending) PA_PHASE(c, 5, pa::launch_stats(nullptr, h, step - 1, c->stream));
        PA_PHASE(c, 0, pa::launch_tables(nullptr, h, step, c->stream));
        PA_PHASE(c, 1, pa::launch_counts(nullptr, h, c->ln, step, c->stream));
        PA_PHASE(c, 2, pa::launch_scan(nullptr, h, step, c->stream));
        PA_PHASE(c, 3, pa::launch_parent(nullptr, h, c->ln, step, c->stream));
    }
    c->stats_pending = false;
    PA_PHASE(c, 4, pa::launch_sweep(nullptr, h, c->ln, step, c->stream, c->pdl));
    if (stats_now) PA_PHASE(c, 5, pa::launch_stats(nullptr, h, step, c->stream));
    else c->stats_pending = true;
    return PA_OK;
}

// Pull records rec[done_rows .. enq_step] to the host (synchronises).
pa_status pull_records(pa_ctx* c)
{
    PA_CUDA(cudaStreamSynchronize(c->stream));
    if (c->cfg.profile) PA_TRY(prof_collect(c));
    int st = 0;
    PA_CUDA(cudaMemcpy(&st, c->h.status, sizeof(int), cudaMemcpyDeviceToHost));
    long long last = c->enq_step;
    if (st != 0) {
        c->failed = (pa_status)st;
        // the failing step left its record incomplete; keep the steps before it
        long long good = c->done_rows;
        std::vector<StepDev> tmp((size_t)(last + 1));
        PA_CUDA(cudaMemcpy(tmp.data(), c->h.rec, sizeof(StepDev) * (size_t)(last + 1), cudaMemcpyDeviceToHost));
        for (long long i = std::max<long long>(good, 1); i <= last; i++) {
            if (tmp[(size_t)i].R > c->h.cap || tmp[(size_t)i].R == 0) {
                last = i - 1;
                break;
            }
        }
    }
    if (last + 1 > c->done_rows) {
        const size_t n = (size_t)(last + 1 - c->done_rows);
        c->recs.resize((size_t)(last + 1));
        PA_CUDA(cudaMemcpy(c->recs.data() + c->done_rows, c->h.rec + c->done_rows, sizeof(StepDev) * n,
                           cudaMemcpyDeviceToHost));
        c->done_rows = last + 1;
    }
    return c->failed;
}

// Host FP64 of the adaptive step (Sec. 2.3): overlap alpha(delta) of the
// histogram H of population i-1 (levels ascending), bisection to alpha*.
double overlap_alpha(const std::vector<long long>& H, int kmin, int kmax, long long R, long long Rprev,
                     double delta, long long P, int estep)
{
    std::vector<double> w;
    level_weights(delta, kmax - kmin + 1, w, estep);
    const double S = tree_sum(H, w, kmin, kmax, 0, P);
    double acc = 0.0;
    for (int k = kmin; k <= kmax; k++) {
        const double tau = ((double)R * w[(size_t)(k - kmin)]) / S;
        acc += (double)H[(size_t)k] * std::min(1.0, tau);
    }
    return acc / (double)Rprev;
}

pa_status enqueue_readback(pa_ctx* c);

pa_status enqueue_step(pa_ctx* c, bool wait = true, bool defer_stats = false)
{
    if (c->done) return PA_DONE;
    const long long i = c->enq_step + 1;
    if (i > c->max_steps) return PA_ESTATE;
    double beta, delta;
    bool final_step;
    if (!c->adaptive) {
        delta = c->cfg.dbeta;
        beta = 0.0 + (double)i * c->cfg.dbeta;
        final_step = (i == c->n_fixed);
    } else {
        // population i-1: its record, status and histogram (staged readback)
        if (wait) {
            PA_CUDA(cudaEventSynchronize(c->ev_ready));
        } else {
            const cudaError_t q = cudaEventQuery(c->ev_ready);
            if (q == cudaErrorNotReady) return PA_EAGAIN;
            if (q != cudaSuccess) return from_cuda(q, __LINE__);
        }
        const StepDev& pr = *(const StepDev*)c->h_down;
        const int dstatus = *(const int*)((const char*)c->h_down + sizeof(StepDev));
        if (dstatus != 0) {
            c->failed = (pa_status)dstatus;
            return c->failed;
        }
        const uint32_t* hr = (const uint32_t*)((const char*)c->h_down + sizeof(StepDev) + 16);
        const int kmin = pr.kmin, kmax = pr.kmax;
        const int nl = kmax - kmin + 1;
        std::vector<long long> H((size_t)c->h.nlev, 0);
        for (int k = kmin; k <= kmax; k++) H[(size_t)k] = hr[(size_t)k];
        const long long P = pad_pow2(c->h.nlev);
        const double bprev = c->betas[(size_t)(i - 1)];
        const double dmax = c->cfg.beta_f - bprev;
        const double target = c->cfg.overlap;
        if (!c->sched.empty()) {
            // given schedule (Sec. 2.3: the first run's steps, reused)
            beta = c->sched[(size_t)(i - 1)];
            delta = beta - bprev;
            final_step = (i == (long long)c->sched.size());
        } else if (overlap_alpha(H, kmin, kmax, c->cfg.R, pr.R, dmax, P, c->h.estep) >= target) {
            delta = dmax;
            final_step = true;
            beta = c->cfg.beta_f;
        } else {
            double lo = 0.0, hi = dmax;
            for (int it = 0; it < 60; it++) {
                const double mid = 0.5 * (lo + hi);
                if (overlap_alpha(H, kmin, kmax, c->cfg.R, pr.R, mid, P, c->h.estep) >= target) lo = mid;
                else hi = mid;
            }
            if (!(lo > 0.0)) return PA_ESTALLED;
            delta = lo;
            final_step = false;
            beta = bprev + delta;
        }
        // level weights for this step and its thresholds
        std::vector<double> w;
        level_weights(delta, nl, w, c->h.estep);
        uint32_t thr[2];
        const uint64_t t4 = threshold(beta, 4.0), t8 = threshold(beta, 8.0);
        thr[0] = (uint32_t)(t4 - 1);
        thr[1] = (uint32_t)(t8 - 1);
        char* st = (char*)c->h_stage;
        std::memcpy(st, w.data(), sizeof(double) * (size_t)nl);
        std::memcpy(st + sizeof(double) * (size_t)nl, thr, sizeof(thr));
        PA_CUDA(cudaMemcpyAsync(c->h.tw, st, sizeof(double) * (size_t)nl, cudaMemcpyHostToDevice, c->stream));
        PA_CUDA(cudaMemcpyAsync(c->h.thr + 2 * i, st + sizeof(double) * (size_t)nl, sizeof(thr),
                                cudaMemcpyHostToDevice, c->stream));
        if (c->h.thr12) {
            uint32_t* t12 = (uint32_t*)(st + sizeof(double) * (size_t)nl + sizeof(thr));
            *t12 = (uint32_t)(threshold(beta, 12.0) - 1);
            PA_CUDA(cudaMemcpyAsync(c->h.thr12 + i, t12, 4, cudaMemcpyHostToDevice, c->stream));
        }
        if (c->h.thrp) {
            uint32_t* tp = (uint32_t*)(st + sizeof(double) * (size_t)nl + sizeof(thr) + 16);
            for (int d = 1; d <= 4; d++) tp[d - 1] = (uint32_t)(threshold(beta, (double)d) - 1);
            PA_CUDA(cudaMemcpyAsync(c->h.thrp + 4 * i, tp, 16, cudaMemcpyHostToDevice, c->stream));
        }
        c->T4.push_back(t4);
        c->T8.push_back(t8);
    }
    PA_TRY(enqueue_kernels(c, (int)i, !defer_stats || final_step || c->adaptive));
    c->betas.push_back(beta);
    c->deltas.push_back(delta);
    c->enq_step = i;
    if (final_step) c->done = true;
    if (c->adaptive && !final_step) PA_TRY(enqueue_readback(c));
    return PA_OK;
}

// Adaptive runs: stage what the next step decision needs.
pa_status enqueue_readback(pa_ctx* c)
{
    if (!c->adaptive) return PA_OK;
    const long long i = c->enq_step;
    char* d = (char*)c->h_down;
    PA_CUDA(cudaMemcpyAsync(d, c->h.rec + i, sizeof(StepDev), cudaMemcpyDeviceToHost, c->stream));
    PA_CUDA(cudaMemcpyAsync(d + sizeof(StepDev), c->h.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PA_CUDA(cudaMemcpyAsync(d + sizeof(StepDev) + 16, c->h.H[i & 1], sizeof(uint32_t) * (size_t)c->h.nlev,
                            cudaMemcpyDeviceToHost, c->stream));
    PA_CUDA(cudaEventRecord(c->ev_ready, c->stream));
    return PA_OK;
}

// ---------------------------------------------------------------- rows
void make_row(const pa_ctx* c, long long i, double sum_lnQ, double lnQ, pa_obs* o)
{
    const StepDev& r = c->recs[(size_t)i];
    const double beta = c->betas[(size_t)i];
    const double fR = (double)r.R, fN = (double)c->N;
    const __int128 sE = i128_of(r.sums + 0), sE2 = i128_of(r.sums + 2), sAM = i128_of(r.sums + 4),
                   sM2 = i128_of(r.sums + 6), sM4 = i128_of(r.sums + 8);
    const __int128 num = (__int128)r.R * sE2 - sE * sE;
    o->beta = beta;
    o->e = (double)sE / (fR * fN);
    o->C = beta * beta * (double)num / (fR * fR * fN);
    o->abs_m = (double)sAM / (fR * fN);
    o->m2 = (double)sM2 / (fR * fN * fN);
    o->m4 = (double)sM4 / (fR * fN * fN * fN * fN);
    // Z at beta0 = 0 counts every configuration: 2^N spins, q^N Potts states
    o->betaF_per_N = -(fN * std::log(c->h.potts_q ? (double)c->h.potts_q : 2.0) + sum_lnQ) / fN;
    o->S_per_N = beta * o->e - o->betaF_per_N;
    o->lnQ = lnQ;
    o->R = r.R;
    o->families = (int64_t)r.fam;
}

double lnQ_of(const pa_ctx* c, long long i)
{
    if (i == 0) return 0.0;
    const StepDev& r = c->recs[(size_t)i];
    const double Emin = (double)(-c->h.eoff + (long long)c->h.estep * r.kmin_prev);
    return (std::log(r.S) - std::log((double)r.R_prev)) - c->deltas[(size_t)i] * Emin;
}

void all_rows(const pa_ctx* c, std::vector<pa_obs>& rows)
{
    rows.resize((size_t)c->done_rows);
    double sum = 0.0;
    for (long long i = 0; i < c->done_rows; i++) {
        const double q = lnQ_of(c, i);
        sum += q;
        make_row(c, i, sum, q, &rows[(size_t)i]);
    }
}

// Back to step 0 with a new seed: clear histograms, records and status,
// then generate and measure the beta0 population (Sec. 2.1 step 1).
pa_status reset_run(pa_ctx* c, uint64_t seed)
{
    RunDev& h = c->h;
    const size_t N1 = (size_t)h.nlev;
    PA_CUDA(cudaStreamSynchronize(c->stream));
    if (c->cfg.profile) PA_TRY(prof_collect(c));
    unsigned* key = (unsigned*)c->h_stage;  // pinned; idle after the sync
    key[0] = (unsigned)(seed & 0xffffffffu);
    key[1] = (unsigned)(seed >> 32);
    PA_CUDA(cudaMemcpyAsync(c->d_key, key, 8, cudaMemcpyHostToDevice, c->stream));
    PA_CUDA(cudaMemsetAsync(h.H[0], 0, 2 * N1 * 4, c->stream));
    PA_CUDA(cudaMemsetAsync(h.H[1], 0, 2 * N1 * 4, c->stream));
    PA_CUDA(cudaMemsetAsync(h.Hsum, 0, N1 * 8, c->stream));
    PA_CUDA(cudaMemsetAsync(h.Msum, 0, 5 * N1 * 8, c->stream));
    PA_CUDA(cudaMemsetAsync(h.rec, 0, sizeof(StepDev) * (size_t)(c->max_steps + 1), c->stream));
    PA_CUDA(cudaMemsetAsync(h.status, 0, 16, c->stream));
    PA_CUDA(cudaMemsetAsync(h.work, 0, 16, c->stream));
    c->cfg.seed = seed;
    c->failed = PA_OK;
    c->betas.assign(1, 0.0);
    c->deltas.assign(1, 0.0);
    if (c->adaptive) {
        c->T4.resize(1);
        c->T8.resize(1);
    }
    c->recs.clear();
    c->done_rows = 0;
    c->enq_step = 0;
    c->done = false;
    c->stats_pending = false;
    cudaEvent_t ev;
    PA_TRY(prof_begin(c, 6, &ev));
    PA_CUDA(pa::launch_init(nullptr, h, c->ln, c->stream));
    PA_TRY(prof_end(c));
    PA_TRY(prof_begin(c, 5, &ev));
    PA_CUDA(pa::launch_stats(nullptr, h, 0, c->stream));
    PA_TRY(prof_end(c));
    c->n_kern += 2;
    return enqueue_readback(c);
}

// Enqueue the remaining schedule without waiting. A fixed schedule started
// from step 0 runs as one CUDA graph (captured on first use, reused after
// pa_reset since every kernel reads the seed from device memory).
pa_status launch_rest(pa_ctx* c)
{
    if (c->failed != PA_OK) return c->failed;
    if (c->done) return PA_OK;
    if (!c->adaptive && c->cfg.use_graph && c->enq_step == 0) {
        if (!c->graph) {
            cudaStream_t cap = nullptr;
            PA_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaStream_t saved = c->stream;
            c->stream = cap;
            c->capturing = true;
            cudaGraph_t g = nullptr;
            pa_status st = PA_OK;
            const long long k0 = c->n_kern;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = PA_ECUDA;
            while (st == PA_OK && !c->done) st = enqueue_step(c, true, true);
            if (st == PA_DONE) st = PA_OK;
            const cudaError_t ce = cudaStreamEndCapture(cap, &g);
            c->stream = saved;
            c->capturing = false;
            c->graph_kern = c->n_kern - k0;  // captured, not launched yet
            c->n_kern = k0;
            if (st == PA_OK && ce != cudaSuccess) st = PA_ECUDA;
            if (st == PA_OK && cudaGraphInstantiate(&c->graph, g, 0) != cudaSuccess) st = PA_ECUDA;
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            if (st != PA_OK) {
                cudaGetLastError();
                for (cudaEvent_t e : c->gev) cudaEventDestroy(e);
                c->gev.clear();
                c->gev_phase.clear();
                c->betas.resize(1);
                c->deltas.resize(1);
                c->enq_step = 0;
                c->done = false;
                c->graph = nullptr;
                c->stats_pending = false;
                return st;
            }
        } else {
            // replay: the host schedule is the same as at capture
            while (!c->done) {
                const long long i = c->enq_step + 1;
                c->betas.push_back(0.0 + (double)i * c->cfg.dbeta);
                c->deltas.push_back(c->cfg.dbeta);
                c->enq_step = i;
                if (i == c->n_fixed) c->done = true;
            }
        }
        PA_CUDA(cudaGraphLaunch(c->graph, c->stream));
        c->n_kern += c->graph_kern;
        if (c->cfg.profile) c->gev_pending = true;
        return PA_OK;
    }
    pa_status st = PA_OK;
    while (st == PA_OK) st = enqueue_step(c, true, true);
    return st == PA_DONE ? PA_OK : st;
}

pa_status free_all(pa_ctx* c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->gev) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFreeAsync(p, c->stream);
    if (c->h_stage) pinned_release(c->h_stage, c->h_stage_bytes);
    if (c->h_down) pinned_release(c->h_down, c->h_down_bytes);
    if (c->ev_ready) cudaEventDestroy(c->ev_ready);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    return PA_OK;
}

}  // namespace

// ============================================== allocation-free resampling
// Scratch of pa_resample_noalloc: one static device array, laid out as
// [key 16 B | R_i 8 B | status 4 B | tile sums | tile offsets | r_j | local
// offsets], every part 256-byte aligned. Host code cannot use the array's
// name as a device address: the address comes from cudaGetSymbolAddress,
// looked up once per device with that device current.
namespace {
constexpr long long kNoAllocMaxOld = PA_RESAMPLE_NOALLOC_MAX_OLD;
constexpr long long kNoAllocTiles = (kNoAllocMaxOld + pa::kTile - 1) / pa::kTile;
constexpr size_t kOffKey = 0, kOffN = 256, kOffStatus = 512, kOffTileSum = 768;
constexpr size_t kOffTileOff = ((kOffTileSum + kNoAllocTiles * 4 + 255) / 256) * 256;
constexpr size_t kOffCnt = ((kOffTileOff + kNoAllocTiles * 4 + 255) / 256) * 256;
constexpr size_t kOffLoc = kOffCnt + (size_t)kNoAllocMaxOld * 4;
constexpr size_t kNoAllocBytes = kOffLoc + (size_t)kNoAllocMaxOld * 4;
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kMaxDevices] = {};

pa_status noalloc_scratch(unsigned char** out)
{
    int dev = 0;
    PA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "pa_resample_noalloc: device index %d is not below the supported %d devices", dev, kMaxDevices);
        return PA_EINVAL;
    }
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        PA_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_addr[dev];
    return PA_OK;
}
}  // namespace

// ======================================================================= ABI
extern "C" {

void pa_config_default(pa_config* cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->L = 16;
    cfg->theta = 10;
    cfg->R = 1000;
    cfg->beta_f = 1.0;
    cfg->dbeta = 0.01;
    cfg->overlap = 0.85;
    cfg->seed = 1;
    cfg->spin_format = PA_SPIN_BITS32;
    cfg->use_graph = 1;
}

const char* pa_last_error_message(void)
{
    return g_last_error;
}

const char* pa_strerror(pa_status s)
{
    switch (s) {
    case PA_OK: return "ok";
    case PA_DONE: return "beta_f reached";
    case PA_EINVAL: return "invalid argument";
    case PA_ENOMEM: return "out of memory";
    case PA_ECAPACITY: return "population exceeded its capacity";
    case PA_EEXTINCT: return "population died out";
    case PA_ETIMEOUT: return "bounded device wait timed out";
    case PA_ECUDA: return "CUDA runtime error";
    case PA_ESTATE: return "invalid state for this call";
    case PA_ESTALLED: return "adaptive step found no positive step size";
    case PA_EAGAIN: return "previous step not finished yet";
    }
    return "unknown status";
}

size_t pa_footprint_bytes(const pa_config* cfg)
{
    if (!cfg || validate(*cfg) != PA_OK) return 0;
    return footprint(*cfg);
}

namespace {
pa_status create_impl(const pa_config* cfg, void* cuda_stream, const int8_t* Jr, const int8_t* Jd, pa_ctx** out);
}

pa_status pa_create(const pa_config* cfg, void* cuda_stream, pa_ctx** out)
{
    return create_impl(cfg, cuda_stream, nullptr, nullptr, out);
}

pa_status pa_create_couplings(const pa_config* cfg, const int8_t* Jr, const int8_t* Jd, void* cuda_stream,
                              pa_ctx** out)
{
    if (!Jr || !Jd) return PA_EINVAL;
    return create_impl(cfg, cuda_stream, Jr, Jd, out);
}

}  // extern "C"

namespace {

// +-J couplings as the kernels read them: for colour c and plane site b at
// (x, y), the bonds to its neighbours in the order same-h, row, up, down
// (same-h is the left bond when x is odd, the right bond when x is even).
void bond_tables(int L, const int8_t* Jr, const int8_t* Jd, std::vector<uint32_t>& masks,
                 std::vector<uint8_t>& bytes)
{
    const int N = L * L, HB = L / 2, NP = N / 2, WP = N / 64;
    bytes.assign((size_t)8 * NP, 0);
    masks.assign((size_t)8 * (WP > 0 ? WP : 1), 0u);
    for (int c = 0; c < 2; c++)
        for (int b = 0; b < NP; b++) {
            const int y = b / HB, h = b % HB, x = 2 * h + ((c + y) & 1);
            const int right = Jr[y * L + x] < 0, left = Jr[y * L + (x + L - 1) % L] < 0;
            const int down = Jd[y * L + x] < 0, up = Jd[((y + L - 1) % L) * L + x] < 0;
            const int dir[4] = {(x & 1) ? left : right, (x & 1) ? right : left, up, down};
            for (int d = 0; d < 4; d++) {
                bytes[(size_t)(d * 2 + c) * NP + b] = (uint8_t)dir[d];
                if (WP > 0 && dir[d]) masks[(size_t)(d * 2 + c) * WP + (b >> 5)] |= 1u << (b & 31);
            }
        }
}

pa_status create_impl(const pa_config* cfg, void* cuda_stream, const int8_t* Jr, const int8_t* Jd, pa_ctx** out)
{
    if (!cfg || !out) return PA_EINVAL;
    *out = nullptr;
    PA_TRY(validate(*cfg));
    if (Jr) {
        if (cfg->spin_format != PA_SPIN_BITS32 && cfg->spin_format != PA_SPIN_INT8) return PA_EINVAL;
        long long neg = 0;
        if (dim_of(*cfg) != 2 || cfg->potts_q) return PA_EINVAL;  // +-J bonds: square-lattice Ising only
        const long long N = (long long)cfg->L * cfg->L;
        for (long long i = 0; i < N; i++) {
            if ((Jr[i] != 1 && Jr[i] != -1) || (Jd[i] != 1 && Jd[i] != -1)) return PA_EINVAL;
            neg += (Jr[i] < 0) + (Jd[i] < 0);
        }
        if (neg & 1) return PA_EINVAL;  // (E + 2N)/4 must be an integer
    }
    pa_ctx* c = new (std::nothrow) pa_ctx();
    if (!c) return PA_ENOMEM;
    c->cfg = *cfg;
    auto fail = [&](pa_status s) {
        free_all(c);
        delete c;
        return s;
    };
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(PA_ECUDA);
        c->own_stream = true;
    }
    const Sizes s = sizes_of(*cfg);
    c->N = s.N;
    c->adaptive = !(cfg->dbeta > 0.0);
    c->n_fixed = c->adaptive ? 0 : s.steps;
    c->max_steps = s.steps;
    c->hist_steps = s.hist_steps;
    RunDev& h = c->h;
    h.L = cfg->L;
    h.N = s.N;
    h.half = cfg->L / 2;
    h.words = s.words;
    h.wp = s.N / 64;
    h.theta = cfg->theta;
    h.fmt = cfg->spin_format;
    int tuned_g = 0, tuned_bw = 0;
    if (!cfg->group_threads && !cfg->block_warps && !pa::tuned_shape(*cfg, 0, &tuned_g, &tuned_bw)) tuned_g = 0;
    const int want_g = cfg->group_threads ? cfg->group_threads : tuned_g;
    h.packed = packed_bytes(*cfg, Jr != nullptr) ? 1 : 0;
    if (h.packed && want_g && !bits_group_valid(cfg->L, want_g))
        h.packed = 0;  // a group shape only the byte kernels have
    h.gt = want_g ? want_g : auto_group(*cfg, h.packed || h.fmt == PA_SPIN_BITS32);
    h.bw = cfg->block_warps ? cfg->block_warps : tuned_bw;
    if (h.fmt == PA_SPIN_MSC32 || h.fmt == PA_SPIN_REPLICA8) h.gt = 1;  // not thread groups
    if (h.fmt == PA_SPIN_BITS32 && (s.N / 64) % h.gt) {
        // several threads per word: square lattice, at most 8 per word, warp groups
        const int wp = s.N / 64;
        if (dim_of(*cfg) != 2 || h.gt > 32 || h.gt % wp || h.gt / wp > 8) return fail(PA_EINVAL);
    }
    h.R = cfg->R;
    h.cap = s.cap;
    h.ntiles = (int)s.ntiles;
    h.record_hist = cfg->record_histograms ? 1 : 0;
    h.hist_steps = (int)s.hist_steps;
    h.nsteps = (int)s.steps;
    h.unit = 1u;
    h.dim = dim_of(*cfg);
    h.nlev = s.nlev;
    h.potts_q = cfg->potts_q;
    h.estep = cfg->potts_q ? 1 : 4;
    h.eoff = (long long)h.dim * s.N;  // Ising dim N; Potts (square lattice) 2N
    c->small_rs = s.cap <= pa::kSmallCap;
    {
        const char* e = std::getenv("PA_PDL");
        c->pdl = c->small_rs && !cfg->profile && !(e && e[0] == '0');
    }
    const size_t N1 = (size_t)s.nlev;
    pa_status st = PA_OK;
#define PA_ALLOC(p, n)                            \
    do {                                          \
        st = dev_alloc(c, &(p), (n));             \
        if (st != PA_OK) return fail(st);         \
    } while (0)
    const size_t pop_words = cfg->spin_format == PA_SPIN_REPLICA8
                                 ? ((size_t)s.N * (size_t)s.cap + 3) / 4
                                 : (cfg->spin_format == PA_SPIN_MSC32 ? (size_t)((s.cap + 31) / 32) : (size_t)s.cap) *
                                       (size_t)s.words;
    for (int b = 0; b < 2; b++) {
        PA_ALLOC(h.pop[b], pop_words);
        PA_ALLOC(h.elev[b], (size_t)s.cap);
        PA_ALLOC(h.mlev[b], (size_t)s.cap);
        PA_ALLOC(h.fam[b], (size_t)s.cap);
        PA_ALLOC(h.H[b], 2 * N1);
    }
    PA_ALLOC(h.parent, (size_t)s.cap);
    PA_ALLOC(h.cnt, (size_t)s.cap);
    PA_ALLOC(h.loc, (size_t)s.cap);
    PA_ALLOC(h.tile_sum, (size_t)s.ntiles);
    PA_ALLOC(h.tile_off, (size_t)s.ntiles);
    PA_ALLOC(h.Hsum, N1);
    PA_ALLOC(h.Msum, 5 * N1);
    PA_ALLOC(h.tw, N1);
    PA_ALLOC(h.F, N1);
    PA_ALLOC(h.U, N1);
    PA_ALLOC(h.thr, 2 * (size_t)(s.steps + 1));
    if (h.dim == 3) PA_ALLOC(h.thr12, (size_t)(s.steps + 1));
    if (h.potts_q) PA_ALLOC(h.thrp, 4 * (size_t)(s.steps + 1));
    PA_ALLOC(h.rec, (size_t)(s.steps + 1));
    if (s.hist_steps) PA_ALLOC(h.hist_rec, (size_t)s.hist_steps * 2 * N1);
    PA_ALLOC(h.status, 4);
    PA_ALLOC(h.work, 4);
    PA_ALLOC(c->d_key, 4);
    h.key = c->d_key;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(PA_ECUDA);  // allocations ready
    if (Jr) {
        std::vector<uint32_t> masks;
        std::vector<uint8_t> bytes;
        bond_tables(cfg->L, Jr, Jd, masks, bytes);
        if (cfg->spin_format == PA_SPIN_BITS32) {
            uint32_t* d = nullptr;
            PA_ALLOC(d, masks.size());
            if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
                cudaMemcpy(d, masks.data(), masks.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(PA_ECUDA);
            h.bonds = d;
        } else {
            uint8_t* d = nullptr;
            PA_ALLOC(d, bytes.size());
            if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
                cudaMemcpy(d, bytes.data(), bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(PA_ECUDA);
            h.bonds8 = d;
        }
    }
#undef PA_ALLOC
    // staging for adaptive uploads (level weights + thresholds)
    c->h_stage_bytes = N1 * sizeof(double) + 64;
    if (!(c->h_stage = pinned_alloc(c->h_stage_bytes))) return fail(PA_ENOMEM);
    if (c->adaptive) {
        c->h_down_bytes = sizeof(StepDev) + 16 + 4 * N1;
        if (!(c->h_down = pinned_alloc(c->h_down_bytes))) return fail(PA_ENOMEM);
        if (cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) != cudaSuccess) return fail(PA_ECUDA);
    }
    c->T4.push_back(1ull << 32);
    c->T8.push_back(1ull << 32);
    if (!c->adaptive) {
        // all thresholds and the (fixed) level weights up front
        std::vector<uint32_t> thr(2 * (size_t)(s.steps + 1), 0xffffffffu), thr12((size_t)(s.steps + 1), 0xffffffffu);
        std::vector<uint32_t> thrp(4 * (size_t)(s.steps + 1), 0xffffffffu);
        for (long long i = 1; i <= s.steps; i++) {
            const double beta = 0.0 + (double)i * cfg->dbeta;
            const uint64_t t4 = threshold(beta, 4.0), t8 = threshold(beta, 8.0);
            thr[2 * (size_t)i] = (uint32_t)(t4 - 1);
            thr[2 * (size_t)i + 1] = (uint32_t)(t8 - 1);
            thr12[(size_t)i] = (uint32_t)(threshold(beta, 12.0) - 1);
            for (int d = 1; d <= 4; d++) thrp[4 * (size_t)i + (size_t)(d - 1)] = (uint32_t)(threshold(beta, (double)d) - 1);
            c->T4.push_back(t4);
            c->T8.push_back(t8);
        }
        std::vector<double> w;
        level_weights(cfg->dbeta, (int)N1, w, h.estep);
        if (cudaMemcpy(h.thr, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h.tw, w.data(), N1 * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
            (h.thr12 && cudaMemcpy(h.thr12, thr12.data(), thr12.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
            (h.thrp && cudaMemcpy(h.thrp, thrp.data(), thrp.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess))
            return fail(PA_ECUDA);
    }
    if (pa::plan_sweep(h, &c->ln) != cudaSuccess) {
        cudaGetLastError();
        return fail(PA_EINVAL);
    }
    {
        const pa_status rs = reset_run(c, cfg->seed);
        if (rs != PA_OK) return fail(rs);
    }
    c->enq_step = 0;
    *out = c;
    return PA_OK;
}

}  // namespace

extern "C" {

pa_status pa_create_scheduled(const pa_config* cfg, const double* betas, int64_t n, void* cuda_stream,
                              pa_ctx** out)
{
    if (!cfg || !betas || !out || n < 1 || n > kMaxAdaptiveSteps) return PA_EINVAL;
    double prev = 0.0;
    for (int64_t i = 0; i < n; i++) {
        if (!(betas[i] > prev) || !(betas[i] <= 50.0)) return PA_EINVAL;
        prev = betas[i];
    }
    pa_config c = *cfg;
    c.dbeta = 0.0;  // stepped like an adaptive run, with the given betas
    c.overlap = 0.5;
    c.beta_f = betas[n - 1];
    PA_TRY(pa_create(&c, cuda_stream, out));
    (*out)->sched.assign(betas, betas + n);
    return PA_OK;
}

// Eq. weighted-average over M runs sharing the inverse temperatures.
pa_status pa_weighted_average(const pa_obs* rows, int32_t m, int64_t n, int32_t N, pa_obs* out)
{
    if (!rows || !out || m < 1 || n < 1 || N < 1) return PA_EINVAL;
    std::vector<double> lw((size_t)m), w((size_t)m);
    for (int64_t i = 0; i < n; i++) {
        const double beta = rows[i].beta;
        for (int32_t r = 0; r < m; r++) {
            const pa_obs& o = rows[(size_t)r * (size_t)n + (size_t)i];
            if (std::fabs(o.beta - beta) > 1e-12 * std::max(1.0, std::fabs(beta))) return PA_EINVAL;
            lw[(size_t)r] = -(double)N * o.betaF_per_N;
        }
        double top = lw[0];
        for (int32_t r = 1; r < m; r++) top = std::max(top, lw[(size_t)r]);
        double Z = 0.0;
        for (int32_t r = 0; r < m; r++) {
            w[(size_t)r] = std::exp(lw[(size_t)r] - top);
            Z += w[(size_t)r];
        }
        for (int32_t r = 0; r < m; r++) w[(size_t)r] /= Z;
        double e = 0.0, am = 0.0, m2 = 0.0, m4 = 0.0, e2 = 0.0, Cavg = 0.0;
        int64_t R = 0, fam = 0;
        for (int32_t r = 0; r < m; r++) {
            const pa_obs& o = rows[(size_t)r * (size_t)n + (size_t)i];
            const double wi = w[(size_t)r];
            e += wi * o.e;
            am += wi * o.abs_m;
            m2 += wi * o.m2;
            m4 += wi * o.m4;
            if (beta > 0.0) e2 += wi * (o.C / (beta * beta * N) + o.e * o.e);
            Cavg += wi * o.C;
            R += o.R;
            fam += o.families;
        }
        pa_obs& d = out[i];
        d.beta = beta;
        d.e = e;
        d.C = beta > 0.0 ? beta * beta * N * (e2 - e * e) : Cavg;
        d.abs_m = am;
        d.m2 = m2;
        d.m4 = m4;
        d.betaF_per_N = -(top + std::log(Z) - std::log((double)m)) / (double)N;
        d.S_per_N = beta * e - d.betaF_per_N;
        d.lnQ = NAN;
        d.R = R;
        d.families = fam;
    }
    return PA_OK;
}

pa_status pa_step(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    if (c->in_batch) return PA_ESTATE;
    if (c->failed != PA_OK) return c->failed;
    return enqueue_step(c);
}

pa_status pa_step_async(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    if (c->in_batch) return PA_ESTATE;
    if (c->failed != PA_OK) return c->failed;
    return enqueue_step(c, false);
}

pa_status pa_sync(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    return pull_records(c);
}

pa_status pa_run(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    if (c->in_batch) return PA_ESTATE;
    PA_TRY(launch_rest(c));
    return pull_records(c);
}

pa_status pa_launch(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    if (c->in_batch) return PA_ESTATE;
    return launch_rest(c);
}

pa_status pa_reset(pa_ctx* c, uint64_t seed)
{
    if (!c) return PA_EINVAL;
    if (c->in_batch) return PA_ESTATE;
    return reset_run(c, seed);
}

pa_status pa_num_rows(pa_ctx* c, int64_t* n)
{
    if (!c || !n) return PA_EINVAL;
    pa_status st = pull_records(c);
    *n = c->done_rows;
    return st == PA_OK || st == PA_ECAPACITY || st == PA_EEXTINCT ? PA_OK : st;
}

pa_status pa_observables(pa_ctx* c, pa_obs* rows, int64_t cap, int64_t* n)
{
    if (!c || !n || (cap > 0 && !rows)) return PA_EINVAL;
    pa_status st = pull_records(c);
    if (st != PA_OK && st != PA_ECAPACITY && st != PA_EEXTINCT) return st;
    std::vector<pa_obs> all;
    all_rows(c, all);
    const long long m = std::min<long long>(cap, (long long)all.size());
    for (long long i = 0; i < m; i++) rows[i] = all[(size_t)i];
    *n = m;
    return PA_OK;
}

pa_status pa_step_info_get(pa_ctx* c, int64_t step, pa_step_info* out)
{
    if (!c || !out) return PA_EINVAL;
    pull_records(c);
    if (step < 0 || step >= c->done_rows) return PA_EINVAL;
    const StepDev& r = c->recs[(size_t)step];
    out->beta = c->betas[(size_t)step];
    out->delta = c->deltas[(size_t)step];
    out->S = r.S;
    out->R = r.R;
    out->R_prev = r.R_prev;
    out->kmin_prev = r.kmin_prev;
    out->kmin = r.kmin;
    out->kmax = r.kmax;
    out->pad = 0;
    out->T4 = c->T4[(size_t)step];
    out->T8 = c->T8[(size_t)step];
    out->families = (int64_t)r.fam;
    return PA_OK;
}

pa_status pa_histogram(pa_ctx* c, int64_t step, int32_t kind, int64_t* out, int64_t cap)
{
    if (!c || !out || cap < c->h.nlev) return PA_EINVAL;
    pull_records(c);
    const size_t N1 = (size_t)c->h.nlev;
    if (kind == PA_HIST_ESUM) {
        std::vector<unsigned long long> t(N1);
        PA_CUDA(cudaMemcpy(t.data(), c->h.Hsum, N1 * 8, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < N1; k++) out[k] = (int64_t)t[k];
        return PA_OK;
    }
    if (kind != PA_HIST_E && kind != PA_HIST_M) return PA_EINVAL;
    if (step < 0 || step >= c->done_rows) return PA_EINVAL;
    std::vector<uint32_t> t(N1);
    const uint32_t* src = nullptr;
    if (c->h.hist_rec && step < c->hist_steps) src = c->h.hist_rec + (size_t)step * 2 * N1;
    else if (step == c->done_rows - 1 && c->failed == PA_OK) src = c->h.H[step & 1];
    else return PA_ESTATE;
    PA_CUDA(cudaMemcpy(t.data(), src + (kind == PA_HIST_M ? N1 : 0), N1 * 4, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < N1; k++) out[k] = (int64_t)t[k];
    return PA_OK;
}

pa_status pa_population(pa_ctx* c, int8_t* host_out, int64_t cap, int64_t* n)
{
    if (!c || !n) return PA_EINVAL;
    pa_status st = pull_records(c);
    if (st != PA_OK) return PA_ESTATE;
    const long long last = c->done_rows - 1;
    const long long R = c->recs[(size_t)last].R;
    const int L = c->cfg.L, N = c->N, half = L / 2;
    const long long m = std::min<long long>(cap, R);
    if (c->h.fmt == PA_SPIN_REPLICA8) {
        const size_t rc = (size_t)c->h.cap;
        std::vector<uint8_t> buf((size_t)N * rc);
        if (m > 0) PA_CUDA(cudaMemcpy(buf.data(), c->h.pop[last & 1], buf.size(), cudaMemcpyDeviceToHost));
        for (long long r = 0; r < m; r++)
            for (int y = 0; y < L; y++)
                for (int x = 0; x < L; x++) {
                    const int col = (x + y) & 1, b = y * half + (x >> 1);
                    const int up = buf[(size_t)(col * (N / 2) + b) * rc + (size_t)r];
                    host_out[(size_t)r * N + (size_t)y * L + x] = up ? 1 : -1;
                }
        *n = m;
        return PA_OK;
    }
    if (c->h.fmt == PA_SPIN_MSC32) {
        std::vector<uint32_t> buf((size_t)((m + 31) / 32) * (size_t)N);
        if (m > 0)
            PA_CUDA(cudaMemcpy(buf.data(), c->h.pop[last & 1], buf.size() * 4, cudaMemcpyDeviceToHost));
        for (long long r = 0; r < m; r++) {
            const uint32_t* w = buf.data() + (size_t)(r / 32) * N;
            for (int y = 0; y < L; y++)
                for (int x = 0; x < L; x++) {
                    const int col = (x + y) & 1, b = y * half + (x >> 1);
                    const int up = (w[col * (N / 2) + b] >> (r % 32)) & 1u;
                    host_out[(size_t)r * N + (size_t)y * L + x] = up ? 1 : -1;
                }
        }
        *n = m;
        return PA_OK;
    }
    std::vector<uint32_t> buf((size_t)m * c->h.words);
    if (m > 0)
        PA_CUDA(cudaMemcpy(buf.data(), c->h.pop[last & 1], buf.size() * 4, cudaMemcpyDeviceToHost));
    const int layers = c->h.dim == 3 ? L : 1;  // z-layers of the simple cubic lattice
    for (long long r = 0; r < m; r++) {
        const uint32_t* w = buf.data() + (size_t)r * c->h.words;
        const uint8_t* bytes = (const uint8_t*)w;
        for (int z = 0; z < layers; z++)
            for (int y = 0; y < L; y++)
                for (int x = 0; x < L; x++) {
                    const int col = (x + y + z) & 1, b = (z * L + y) * half + (x >> 1);
                    int up;
                    if (c->h.fmt == PA_SPIN_BITS32) up = (w[col * (N / 64) + (b >> 5)] >> (b & 31)) & 1u;
                    else up = bytes[col * (N / 2) + b];
                    // Potts: the state 0..q-1 itself
                    host_out[(size_t)r * N + ((size_t)z * L + y) * L + x] =
                        c->h.potts_q ? (int8_t)up : (int8_t)(up ? 1 : -1);
                }
    }
    *n = m;
    return PA_OK;
}

pa_status pa_replicas(pa_ctx* c, int32_t* E, int32_t* M, int64_t* family, int64_t cap, int64_t* n)
{
    if (!c || !n) return PA_EINVAL;
    pa_status st = pull_records(c);
    if (st != PA_OK) return PA_ESTATE;
    const long long last = c->done_rows - 1;
    const long long R = c->recs[(size_t)last].R;
    const long long m = std::min<long long>(cap, R);
    std::vector<int32_t> ev((size_t)m), mv((size_t)m);
    std::vector<uint32_t> fv((size_t)m);
    if (m > 0) {
        PA_CUDA(cudaMemcpy(ev.data(), c->h.elev[last & 1], (size_t)m * 4, cudaMemcpyDeviceToHost));
        PA_CUDA(cudaMemcpy(mv.data(), c->h.mlev[last & 1], (size_t)m * 4, cudaMemcpyDeviceToHost));
        PA_CUDA(cudaMemcpy(fv.data(), c->h.fam[last & 1], (size_t)m * 4, cudaMemcpyDeviceToHost));
    }
    for (long long r = 0; r < m; r++) {
        if (E) E[r] = (int32_t)((long long)c->h.estep * ev[(size_t)r] - c->h.eoff);
        if (M) M[r] = c->h.potts_q ? mv[(size_t)r] : 2 * mv[(size_t)r] - c->N;
        if (family) family[r] = fv[(size_t)r];
    }
    *n = m;
    return PA_OK;
}

// Eq. MHReq1: Omega(E) = sum_i P_i(E) / sum_i R_i exp(beta_i F_i - beta_i E),
// evaluated in logarithms: ln Omega_k = ln Hsum_k - LSE_i(ln R_i + beta_i F_i
// - beta_i E_k) with beta_i F_i = -(N ln 2 + sum_{l<=i} ln Q_l); row 0 (an
// exact beta = 0 sample) included.
pa_status pa_ln_dos(pa_ctx* c, double* out, int64_t cap)
{
    if (!c || !out || cap < c->h.nlev) return PA_EINVAL;
    pa_status st = pull_records(c);
    if (st != PA_OK && st != PA_ECAPACITY && st != PA_EEXTINCT) return st;
    const size_t N1 = (size_t)c->h.nlev;
    std::vector<unsigned long long> hs(N1);
    PA_CUDA(cudaMemcpy(hs.data(), c->h.Hsum, N1 * 8, cudaMemcpyDeviceToHost));
    std::vector<pa_obs> rows;
    all_rows(c, rows);
    const size_t nr = rows.size();
    std::vector<double> lnR(nr), bF(nr), b(nr);
    for (size_t i = 0; i < nr; i++) {
        lnR[i] = std::log((double)rows[i].R);
        bF[i] = rows[i].betaF_per_N * (double)c->N;
        b[i] = rows[i].beta;
    }
    std::vector<double> a(nr);
    for (size_t k = 0; k < N1; k++) {
        if (hs[k] == 0) {
            out[k] = -INFINITY;
            continue;
        }
        const double Ek = (double)(-c->h.eoff + (long long)c->h.estep * (long long)k);
        double m = -INFINITY;
        for (size_t i = 0; i < nr; i++) {
            a[i] = lnR[i] + bF[i] - b[i] * Ek;
            m = std::max(m, a[i]);
        }
        double s = 0.0;
        for (size_t i = 0; i < nr; i++) s += std::exp(a[i] - m);
        out[k] = std::log((double)hs[k]) - (m + std::log(s));
    }
    return PA_OK;
}

pa_status pa_mag_sums(pa_ctx* c, uint64_t* out, int64_t cap)
{
    if (!c || !out || cap < 5 * (int64_t)c->h.nlev) return PA_EINVAL;
    pa_status st = pull_records(c);
    if (st != PA_OK && st != PA_ECAPACITY && st != PA_EEXTINCT) return st;
    PA_CUDA(cudaMemcpy(out, c->h.Msum, 5 * (size_t)c->h.nlev * 8, cudaMemcpyDeviceToHost));
    return PA_OK;
}

// Reweighted rows: energy moments from Omega(E); magnetisation moments from
// sum_M Omega(E, M) f(M) = Omega(E) (sum of f(M) at level E) / Hsum(E), the
// Boltzmann weight depending on E only.
pa_status pa_mhr(pa_ctx* c, const double* betas, int64_t n, pa_obs* out)
{
    if (!c || (n > 0 && (!betas || !out))) return PA_EINVAL;
    const size_t N1 = (size_t)c->h.nlev;
    std::vector<double> lno(N1);
    PA_TRY(pa_ln_dos(c, lno.data(), (int64_t)N1));
    std::vector<unsigned long long> hs(N1), ms(5 * N1);
    PA_CUDA(cudaMemcpy(hs.data(), c->h.Hsum, N1 * 8, cudaMemcpyDeviceToHost));
    PA_CUDA(cudaMemcpy(ms.data(), c->h.Msum, 5 * N1 * 8, cudaMemcpyDeviceToHost));
    std::vector<double> mic(3 * N1, 0.0);
    for (size_t k = 0; k < N1; k++) {
        if (!hs[k]) continue;
        const double cnt = (double)hs[k];
        const unsigned __int128 m2 = ((unsigned __int128)ms[5 * k + 2] << 64) | ms[5 * k + 1];
        const unsigned __int128 m4 = ((unsigned __int128)ms[5 * k + 4] << 64) | ms[5 * k + 3];
        mic[3 * k + 0] = (double)ms[5 * k] / cnt;
        mic[3 * k + 1] = (double)m2 / cnt;
        mic[3 * k + 2] = (double)m4 / cnt;
    }
    const double fN = (double)c->N;
    for (int64_t t = 0; t < n; t++) {
        const double beta = betas[t];
        double m = -INFINITY;
        for (size_t k = 0; k < N1; k++) {
            if (!std::isfinite(lno[k])) continue;
            const double Ek = (double)(-c->h.eoff + (long long)c->h.estep * (long long)k);
            m = std::max(m, lno[k] - beta * Ek);
        }
        double Z = 0.0, e1 = 0.0, e2 = 0.0, a1 = 0.0, a2 = 0.0, a4 = 0.0;
        for (size_t k = 0; k < N1; k++) {
            if (!std::isfinite(lno[k])) continue;
            const double Ek = (double)(-c->h.eoff + (long long)c->h.estep * (long long)k);
            const double w = std::exp(lno[k] - beta * Ek - m);
            Z += w;
            e1 += w * Ek;
            e2 += w * Ek * Ek;
            a1 += w * mic[3 * k];
            a2 += w * mic[3 * k + 1];
            a4 += w * mic[3 * k + 2];
        }
        e1 /= Z;
        e2 /= Z;
        const double lnZ = m + std::log(Z);
        pa_obs& o = out[t];
        o.beta = beta;
        o.e = e1 / fN;
        o.C = beta * beta * (e2 - e1 * e1) / fN;
        o.abs_m = a1 / Z / fN;
        o.m2 = a2 / Z / (fN * fN);
        o.m4 = a4 / Z / (fN * fN * fN * fN);
        o.betaF_per_N = -lnZ / fN;
        o.S_per_N = beta * o.e - o.betaF_per_N;
        o.lnQ = NAN;
        o.R = 0;
        o.families = 0;
    }
    return PA_OK;
}

pa_status pa_phase_times(pa_ctx* c, double ms[7], int64_t launches[7])
{
    if (!c || !ms || !launches) return PA_EINVAL;
    PA_CUDA(cudaStreamSynchronize(c->stream));
    if (c->cfg.profile) PA_TRY(prof_collect(c));
    for (int p = 0; p < 7; p++) {
        ms[p] = c->phase_ms[p];
        launches[p] = c->phase_n[p];
    }
    return PA_OK;
}

pa_status pa_kernel_launches(pa_ctx* c, int64_t* n)
{
    if (!c || !n) return PA_EINVAL;
    *n = c->n_kern;
    return PA_OK;
}

pa_status pa_launch_shape(pa_ctx* c, int32_t* gt, int32_t* bt, int32_t* gb)
{
    if (!c) return PA_EINVAL;
    if (gt) *gt = c->h.gt;
    if (bt) *bt = c->ln.sweep_threads;
    if (gb) *gb = c->ln.sweep_blocks;
    return PA_OK;
}

void pa_destroy(pa_ctx* c)
{
    if (!c || c->in_batch) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

pa_status pa_philox_device(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out, void* stream)
{
    if (n < 0 || (n > 0 && (!ctr || !out))) return PA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PA_CUDA(pa::launch_philox(ctr, n, pa::PhiloxKey{(unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)}, out, s));
    PA_CUDA(cudaStreamSynchronize(s));
    return PA_OK;
}

pa_status pa_resample(const int32_t* lev, int64_t n_old, const uint32_t* F, const uint64_t* U, int64_t n_levels,
                      uint64_t seed, int64_t step, uint32_t* parent, int64_t cap, int64_t* n_new, void* stream)
{
    if (!lev || !F || !U || !parent || !n_new || n_old < 1 || n_old > (1ll << 31) || n_levels < 1 || cap < 1 ||
        cap > (1ll << 31) || step < 0 || step > 0xffffffffll)
        return PA_EINVAL;
    *n_new = 0;
    cudaStream_t s = (cudaStream_t)stream;
    const long long tiles = (n_old + pa::kTile - 1) / pa::kTile;
    // scratch: key, counts, local offsets, tile sums/offsets, R_i, status
    unsigned* key = nullptr;
    uint32_t *cnt = nullptr, *loc = nullptr, *tsum = nullptr, *toff = nullptr;
    long long* nn = nullptr;
    int* st = nullptr;
    pa_status out = PA_OK;
    auto grab = [&](void** p, size_t b) {
        if (out == PA_OK && cudaMalloc(p, b) != cudaSuccess) {
            cudaGetLastError();
            out = PA_ENOMEM;
        }
    };
    grab((void**)&key, 16);
    grab((void**)&cnt, (size_t)n_old * 4);
    grab((void**)&loc, (size_t)n_old * 4);
    grab((void**)&tsum, (size_t)tiles * 4);
    grab((void**)&toff, (size_t)tiles * 4);
    grab((void**)&nn, 16);
    grab((void**)&st, 16);
    if (out == PA_OK) {
        const unsigned hk[2] = {(unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)};
        pa::ResampleArgs a{};
        a.n_old_dev = nullptr;
        a.n_old = n_old;
        a.lev = lev;
        a.F = F;
        a.U = (const unsigned long long*)U;
        a.key = key;
        a.step = (unsigned)step;
        a.cnt = cnt;
        a.loc = loc;
        a.tile_sum = tsum;
        a.tile_off = toff;
        a.parent = parent;
        a.cap = cap;
        a.n_new = nn;
        a.n_prev_out = nullptr;
        a.status = st;
        a.work = nullptr;
        long long hn = 0;
        int hs = 0;
        cudaError_t e = cudaMemcpyAsync(key, hk, 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, 16, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(nn, 0, 16, s);  // stays 0 if a tile alone exceeds cap
        if (e == cudaSuccess) e = pa::launch_resample(a, (int)tiles, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hn, nn, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) out = from_cuda(e, __LINE__);
        else if (hs != 0) out = (pa_status)hs;
        *n_new = hn;
    }
    cudaFree(key);
    cudaFree(cnt);
    cudaFree(loc);
    cudaFree(tsum);
    cudaFree(toff);
    cudaFree(nn);
    cudaFree(st);
    return out;
}

pa_status pa_resample_noalloc(const int32_t* lev, int64_t n_old, const uint32_t* F, const uint64_t* U,
                              int64_t n_levels, uint64_t seed, int64_t step, uint32_t* parent, int64_t cap,
                              int64_t* n_new, void* stream)
{
    if (!lev || !F || !U || !parent || !n_new || n_old < 1 || n_levels < 1 || cap < 1 || cap > (1ll << 31) ||
        step < 0 || step > 0xffffffffll)
        return PA_EINVAL;
    *n_new = 0;
    if (n_old > kNoAllocMaxOld) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "pa_resample_noalloc: n_old %lld exceeds the static scratch limit %lld", (long long)n_old,
                      kNoAllocMaxOld);
        return PA_EINVAL;
    }
    unsigned char* base = nullptr;
    PA_TRY(noalloc_scratch(&base));
    cudaStream_t s = (cudaStream_t)stream;
    const long long tiles = (n_old + pa::kTile - 1) / pa::kTile;
    unsigned* key = (unsigned*)(base + kOffKey);
    long long* nn = (long long*)(base + kOffN);
    int* st = (int*)(base + kOffStatus);
    pa::ResampleArgs a{};
    a.n_old_dev = nullptr;
    a.n_old = n_old;
    a.lev = lev;
    a.F = F;
    a.U = (const unsigned long long*)U;
    a.key = key;
    a.step = (unsigned)step;
    a.cnt = (uint32_t*)(base + kOffCnt);
    a.loc = (uint32_t*)(base + kOffLoc);
    a.tile_sum = (uint32_t*)(base + kOffTileSum);
    a.tile_off = (uint32_t*)(base + kOffTileOff);
    a.parent = parent;
    a.cap = cap;
    a.n_new = nn;
    a.n_prev_out = nullptr;
    a.status = st;
    a.work = nullptr;
    // the array keeps the previous call's contents: the status word and R_i
    // must start at zero (R_i stays 0 when one tile alone exceeds cap); every
    // other part is written before it is read
    const unsigned hk[2] = {(unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)};
    long long hn = 0;
    int hs = 0;
    PA_CUDA(cudaMemcpyAsync(key, hk, 8, cudaMemcpyHostToDevice, s));
    PA_CUDA(cudaMemsetAsync(st, 0, 4, s));
    PA_CUDA(cudaMemsetAsync(nn, 0, 8, s));
    PA_CUDA(pa::launch_resample(a, (int)tiles, s));
    PA_CUDA(cudaMemcpyAsync(&hn, nn, 8, cudaMemcpyDeviceToHost, s));
    PA_CUDA(cudaMemcpyAsync(&hs, st, 4, cudaMemcpyDeviceToHost, s));
    PA_CUDA(cudaStreamSynchronize(s));
    *n_new = hn;
    return hs != 0 ? (pa_status)hs : PA_OK;
}

pa_status pa_gather(const uint32_t* src, int64_t n_src, const uint32_t* parent, int64_t n_new, int32_t words,
                    uint32_t* dst, void* stream, double* ms)
{
    if (!src || !parent || !dst || n_src < 1 || n_new < 0 || words < 4 || words % 4 ||
        ((uintptr_t)src | (uintptr_t)dst) % 16)
        return PA_EINVAL;
    if (n_new == 0) {
        if (ms) *ms = 0.0;
        return PA_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PA_CUDA(cudaGetDevice(&dev));
    PA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned* bad = nullptr;
    PA_CUDA(cudaMalloc(&bad, 4));
    cudaEvent_t a = nullptr, b = nullptr;
    unsigned hbad = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, 4, s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = pa::launch_gather(src, parent, n_new, n_src, words, dst, bad, sms * 8, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float t = 0.f;
    if (e == cudaSuccess && ms) e = cudaEventElapsedTime(&t, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(bad);
    if (e != cudaSuccess) return from_cuda(e, __LINE__);
    if (ms) *ms = (double)t;
    return hbad ? PA_EINVAL : PA_OK;
}

pa_status pa_selftest_bulk_wait(int32_t bytes, int32_t copy, int32_t tries, void* stream)
{
    if (bytes < 16 || bytes > 4096 || bytes % 16 || tries < 1) return PA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* src = nullptr;  // pattern, then the kernel's result word
    PA_CUDA(cudaMalloc(&src, (size_t)bytes + 16));
    std::vector<uint32_t> pat((size_t)bytes / 4 + 4);
    for (size_t i = 0; i < pat.size(); i++) pat[i] = 0x9E3779B9u * (uint32_t)(i + 1);
    int res = 2;
    cudaError_t e = cudaMemcpyAsync(src, pat.data(), (size_t)bytes + 16, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = pa::launch_bulk_selftest(src, bytes, copy != 0, tries, (int*)(src + bytes / 4), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&res, src + bytes / 4, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(src);
    if (e != cudaSuccess) return from_cuda(e, __LINE__);
    if (res == pa::kStatusTimeout) return PA_ETIMEOUT;
    return res == 0 ? PA_OK : PA_ECUDA;
}

pa_status pa_measure_rng_peak(int64_t blocks_per_thread, uint32_t* sink, void* stream, double* words_per_ns)
{
    if (blocks_per_thread < 8 || !sink || !words_per_ns) return PA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PA_CUDA(cudaGetDevice(&dev));
    PA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, grid = sms * 8;  // 2048 resident threads per SM
    const long long blocks = blocks_per_thread & ~7ll;
    cudaEvent_t a, b;
    PA_CUDA(cudaEventCreate(&a));
    PA_CUDA(cudaEventCreate(&b));
    PA_CUDA(pa::launch_rng_peak(blocks, sink, grid, threads, s));  // warm-up
    PA_CUDA(cudaEventRecord(a, s));
    PA_CUDA(pa::launch_rng_peak(blocks, sink, grid, threads, s));
    PA_CUDA(cudaEventRecord(b, s));
    PA_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    PA_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *words_per_ns = 4.0 * (double)blocks * (double)grid * threads / ((double)ms * 1e6);
    return PA_OK;
}

pa_status pa_measure_pipe_peak(int pipe, int64_t iters, uint32_t* sink, void* stream, double* lane_ops_per_ns)
{
    if (pipe < 0 || pipe > 2 || iters < 4 || !sink || !lane_ops_per_ns) return PA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PA_CUDA(cudaGetDevice(&dev));
    PA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, grid = sms * 8;  // 2048 resident threads per SM
    const long long it = iters & ~3ll;
    cudaEvent_t a, b;
    PA_CUDA(cudaEventCreate(&a));
    PA_CUDA(cudaEventCreate(&b));
    PA_CUDA(pa::launch_pipe_peak(pipe, it, sink, grid, threads, s));  // warm-up
    PA_CUDA(cudaEventRecord(a, s));
    PA_CUDA(pa::launch_pipe_peak(pipe, it, sink, grid, threads, s));
    PA_CUDA(cudaEventRecord(b, s));
    PA_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    PA_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double per_iter = pipe == 1 ? 24.0 : 8.0;  // instructions per thread per iteration
    *lane_ops_per_ns = per_iter * (double)it * (double)grid * threads / ((double)ms * 1e6);
    return PA_OK;
}

}  // extern "C"

// ================================================================== batches
// Independent fixed-schedule runs stepped together (batched runs):
// each bookkeeping phase of a temperature step is one launch over all runs,
// and the sweep is one persistent kernel per segment of runs sharing a
// shape (L, threads per replica), pulling items from the segment's queue
// (descending work per replica); the segments run on parallel graph
// branches. The whole schedule is captured once as one CUDA graph.
struct pa_batch {
    std::vector<pa_ctx*> runs;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void*> allocs;
    pa::BatchDev bd{};
    pa::BatchLaunch ln{};
    int max_steps = 0;
    cudaGraphExec_t graph = nullptr;
    bool profile = false;
    std::vector<cudaEvent_t> ev;  // (start, end) per phase launch in the graph
    std::vector<int> ev_phase;
    bool ev_pending = false;
    double phase_ms[7] = {0, 0, 0, 0, 0, 0, 0};
    long long phase_n[7] = {0, 0, 0, 0, 0, 0, 0};
    std::vector<int> order;       // queue position -> run
    // runs of one replica per CTA: descriptors, sweep plans and last steps
    // (BatchLaunch points at these), and their index among the runs
    std::vector<pa::RunDev> own_h;
    std::vector<pa::Launch> own_ln;
    std::vector<int> own_last, own_run;
};

namespace {

// host side of a fixed schedule: the betas of every step the graph runs
void advance_fixed(pa_ctx* c)
{
    while (!c->done) {
        const long long i = c->enq_step + 1;
        c->betas.push_back(0.0 + (double)i * c->cfg.dbeta);
        c->deltas.push_back(c->cfg.dbeta);
        c->enq_step = i;
        if (i == c->n_fixed) c->done = true;
    }
}

void batch_free(pa_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (pa_ctx* c : b->runs) {
        if (!c) continue;
        c->in_batch = false;
        c->own_stream = false;
        pa_destroy(c);
    }
    for (void* p : b->allocs) cudaFreeAsync(p, b->stream);
    for (int i = 0; i < pa::kMaxBatchSegs; i++) {
        if (b->ln.side[i]) cudaStreamDestroy(b->ln.side[i]);
        if (b->ln.join[i]) cudaEventDestroy(b->ln.join[i]);
    }
    for (int i = 0; i < pa::kBatchOwnStreams; i++) {
        if (b->ln.own_side[i]) cudaStreamDestroy(b->ln.own_side[i]);
        if (b->ln.own_join[i]) cudaEventDestroy(b->ln.own_join[i]);
    }
    if (b->ln.fork) cudaEventDestroy(b->ln.fork);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

pa_status batch_record(pa_batch* b, int phase)
{
    if (!b->profile) return PA_OK;
    cudaEvent_t e;
    PA_CUDA(cudaEventCreate(&e));
    PA_CUDA(cudaEventRecordWithFlags(e, b->stream, cudaEventRecordExternal));
    b->ev.push_back(e);
    b->ev_phase.push_back(phase);
    return PA_OK;
}

pa_status batch_collect(pa_batch* b)
{
    if (!b->ev_pending) return PA_OK;
    for (size_t i = 0; i + 1 < b->ev.size(); i += 2) {
        float ms = 0.f;
        PA_CUDA(cudaEventElapsedTime(&ms, b->ev[i], b->ev[i + 1]));
        b->phase_ms[b->ev_phase[i]] += ms;
        b->phase_n[b->ev_phase[i]] += 1;
    }
    b->ev_pending = false;
    return PA_OK;
}

pa_status batch_capture(pa_batch* b)
{
    cudaStream_t cap = nullptr;
    PA_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = b->stream;
    b->stream = cap;
    pa_status st = PA_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = PA_ECUDA;
    for (int step = 1; st == PA_OK && step <= b->max_steps; step++) {
        for (int phase = 0; phase < 6 && st == PA_OK; phase++) {
            if (!pa::batch_phase_launches(b->ln, step, phase)) continue;
            st = batch_record(b, phase);
            if (st == PA_OK && pa::launch_batch_step(b->bd, b->ln, step, cap, phase, nullptr) != cudaSuccess)
                st = PA_ECUDA;
            if (st == PA_OK) st = batch_record(b, -1);
        }
    }
    const cudaError_t ce = cudaStreamEndCapture(cap, &g);
    b->stream = saved;
    if (st == PA_OK && ce != cudaSuccess) st = PA_ECUDA;
    if (st == PA_OK && cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) st = PA_ECUDA;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (st != PA_OK) {
        cudaGetLastError();
        for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
        b->ev.clear();
        b->ev_phase.clear();
        b->graph = nullptr;
    }
    return st;
}

}  // namespace

extern "C" {

pa_status pa_batch_create(const pa_config* cfgs, int32_t n, void* cuda_stream, pa_batch** out)
{
    if (!cfgs || !out || n < 1 || n > pa::kMaxBatchRuns) return PA_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; i++) {
        const pa_config& c = cfgs[i];
        PA_TRY(validate(c));
        if (!(c.dbeta > 0.0) || c.spin_format != PA_SPIN_BITS32 || c.L > 512 || dim_of(c) != 2)
            return PA_EINVAL;  // bit-packed square lattices only
        if (c.group_threads && !pa::batch_supports(c.L, c.group_threads)) return PA_EINVAL;
    }
    pa_batch* b = new (std::nothrow) pa_batch();
    if (!b) return PA_ENOMEM;
    auto fail = [&](pa_status s) {
        batch_free(b);
        delete b;
        return s;
    };
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(PA_ECUDA);
        b->own_stream = true;
    }
    b->profile = false;
    std::vector<RunDev> hr((size_t)n);
    for (int i = 0; i < n; i++) {
        pa_config c = cfgs[i];
        if (c.profile) b->profile = true;
        if (!c.group_threads) {
            pa_tune_choice tc{};
            const pa_status ts = pa::autotune_impl(&c, 1, nullptr, b->stream, &tc);
            if (ts != PA_OK) return fail(ts);
            c.group_threads = tc.group_threads;
        }
        c.use_graph = 0;
        c.profile = 0;
        pa_ctx* m = nullptr;
        const pa_status cs = pa_create(&c, b->stream, &m);
        if (cs != PA_OK) return fail(cs);
        m->in_batch = true;
        b->runs.push_back(m);
        hr[(size_t)i] = m->h;
        b->max_steps = std::max(b->max_steps, (int)m->n_fixed);
    }
    // queue order: runs grouped by shape (larger lattices first), each group
    // by descending work per replica (theta * N). A run that fills the device
    // alone (one replica per CTA, or a warp-group run whose sweep grid is all
    // the device keeps resident) is swept by its own sweep kernel, the one it
    // runs alone with; beside the others, its tail overlaps theirs. The other
    // runs of one shape form a segment, swept by one kernel.
    auto own = [&](int i) { return hr[(size_t)i].gt > 32 || b->runs[(size_t)i]->ln.sweep_full; };
    std::vector<int> order((size_t)n), tile_run, tile_first((size_t)n);
    for (int i = 0; i < n; i++) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const RunDev &a = hr[(size_t)x], &c = hr[(size_t)y];
        if (own(x) != own(y)) return own(x);  // own-kernel runs first: segments stay contiguous
        if (a.L != c.L) return a.L > c.L;
        if (a.gt != c.gt) return a.gt > c.gt;
        return (long long)a.theta * a.N > (long long)c.theta * c.N;
    });
    b->ln.nseg = 0;
    for (int q = 0; q < n; q++) {
        const int i = order[(size_t)q];
        const RunDev& a = hr[(size_t)i];
        if (own(i)) {
            b->own_h.push_back(a);
            b->own_ln.push_back(b->runs[(size_t)i]->ln);
            b->own_last.push_back((int)b->runs[(size_t)i]->n_fixed);
            b->own_run.push_back(i);
            continue;
        }
        pa::BatchSeg* last = b->ln.nseg ? &b->ln.seg[b->ln.nseg - 1] : nullptr;
        if (last && last->L == a.L && last->G == a.gt) {
            last->q1 = q + 1;
            continue;
        }
        if (b->ln.nseg == pa::kMaxBatchSegs) return fail(PA_EINVAL);
        b->ln.seg[b->ln.nseg++] = pa::BatchSeg{q, q + 1, a.L, a.gt, 0, 0};
    }
    for (int i = 0; i < b->ln.nseg; i++) {
        pa::BatchSeg& sg = b->ln.seg[i];
        long long units = 0;
        for (int q = sg.q0; q < sg.q1; q++) units += hr[(size_t)order[(size_t)q]].cap;
        if (pa::plan_batch_segment(&sg, units) != cudaSuccess) {
            cudaGetLastError();
            return fail(PA_EINVAL);
        }
    }
    b->ln.small = true;
    for (pa_ctx* m : b->runs) b->ln.small = b->ln.small && m->small_rs;
    b->ln.last = b->max_steps;
    b->ln.nown = (int)b->own_h.size();
    b->ln.own_h = b->own_h.data();
    b->ln.own_ln = b->own_ln.data();
    b->ln.own_last = b->own_last.data();
    const int ncs = std::min(b->ln.nown, pa::kBatchOwnStreams);
    if (b->ln.nseg + ncs > 1) {
        if (cudaEventCreateWithFlags(&b->ln.fork, cudaEventDisableTiming) != cudaSuccess) return fail(PA_ECUDA);
        for (int i = 0; i < b->ln.nseg; i++)
            if (cudaStreamCreateWithFlags(&b->ln.side[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ln.join[i], cudaEventDisableTiming) != cudaSuccess)
                return fail(PA_ECUDA);
        for (int i = 0; i < ncs; i++)
            if (cudaStreamCreateWithFlags(&b->ln.own_side[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ln.own_join[i], cudaEventDisableTiming) != cudaSuccess)
                return fail(PA_ECUDA);
    }
    for (int i = 0; i < n; i++) {
        tile_first[(size_t)i] = (int)tile_run.size();
        for (int t = 0; t < hr[(size_t)i].ntiles; t++) tile_run.push_back(i);
    }
    auto dalloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMallocAsync(p, std::max<size_t>(bytes, 16), b->stream) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        b->allocs.push_back(*p);
        return true;
    };
    RunDev* d_runs = nullptr;
    int *d_order = nullptr, *d_tile_run = nullptr, *d_tile_first = nullptr;
    long long* d_off = nullptr;
    unsigned* d_work = nullptr;
    if (!dalloc((void**)&d_runs, sizeof(RunDev) * (size_t)n) || !dalloc((void**)&d_order, 4 * (size_t)n) ||
        !dalloc((void**)&d_tile_run, 4 * tile_run.size()) || !dalloc((void**)&d_tile_first, 4 * (size_t)n) ||
        !dalloc((void**)&d_off, 8 * (size_t)(n + 1)) || !dalloc((void**)&d_work, 4 * pa::kMaxBatchSegs))
        return fail(PA_ENOMEM);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(PA_ECUDA);  // allocations ready
    if (cudaMemcpy(d_runs, hr.data(), sizeof(RunDev) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_order, order.data(), 4 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_tile_run, tile_run.data(), 4 * tile_run.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_tile_first, tile_first.data(), 4 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(PA_ECUDA);
    b->bd.runs = d_runs;
    b->bd.order = d_order;
    b->bd.tile_run = d_tile_run;
    b->bd.tile_first = d_tile_first;
    b->bd.item_off = d_off;
    b->bd.work = d_work;
    b->bd.nruns = n;
    b->bd.nseg = b->ln.nseg;
    b->ln.tiles = (int)tile_run.size();
    b->order = order;
    *out = b;
    return PA_OK;
}

pa_status pa_batch_launch(pa_batch* b)
{
    if (!b) return PA_EINVAL;
    for (pa_ctx* c : b->runs)
        if (c->enq_step != 0 || c->failed != PA_OK) return PA_ESTATE;
    if (!b->graph) PA_TRY(batch_capture(b));
    for (pa_ctx* c : b->runs) advance_fixed(c);
    PA_CUDA(cudaGraphLaunch(b->graph, b->stream));
    if (b->profile) b->ev_pending = true;
    return PA_OK;
}

pa_status pa_batch_sync(pa_batch* b)
{
    if (!b) return PA_EINVAL;
    PA_CUDA(cudaStreamSynchronize(b->stream));
    PA_TRY(batch_collect(b));
    pa_status first = PA_OK;
    for (pa_ctx* c : b->runs) {
        const pa_status st = pull_records(c);
        if (st != PA_OK && first == PA_OK) first = st;
    }
    return first;
}

pa_status pa_batch_run(pa_batch* b)
{
    PA_TRY(pa_batch_launch(b));
    return pa_batch_sync(b);
}

pa_status pa_batch_reset(pa_batch* b, const uint64_t* seeds)
{
    if (!b || !seeds) return PA_EINVAL;
    PA_CUDA(cudaStreamSynchronize(b->stream));
    PA_TRY(batch_collect(b));
    for (size_t i = 0; i < b->runs.size(); i++) PA_TRY(reset_run(b->runs[i], seeds[i]));
    return PA_OK;
}

pa_status pa_batch_get(pa_batch* b, int32_t i, pa_ctx** out)
{
    if (!b || !out || i < 0 || i >= (int32_t)b->runs.size()) return PA_EINVAL;
    *out = b->runs[(size_t)i];
    return PA_OK;
}

pa_status pa_batch_phase_times(pa_batch* b, double ms[7], int64_t launches[7])
{
    if (!b || !ms || !launches) return PA_EINVAL;
    PA_CUDA(cudaStreamSynchronize(b->stream));
    PA_TRY(batch_collect(b));
    for (int p = 0; p < 7; p++) {
        ms[p] = b->phase_ms[p];
        launches[p] = b->phase_n[p];
    }
    return PA_OK;
}

pa_status pa_batch_shape(pa_batch* b, int32_t i, int32_t* group_threads, int32_t* sweep_blocks)
{
    if (!b || i < 0 || i >= (int32_t)b->runs.size()) return PA_EINVAL;
    if (group_threads) *group_threads = b->runs[(size_t)i]->h.gt;
    if (sweep_blocks) {
        *sweep_blocks = 0;
        for (size_t j = 0; j < b->own_run.size(); j++)
            if (b->own_run[j] == i) *sweep_blocks = b->own_ln[j].sweep_blocks;
        for (int q = 0; q < (int)b->order.size(); q++)
            if (b->order[(size_t)q] == i)
                for (int s = 0; s < b->ln.nseg; s++)
                    if (q >= b->ln.seg[s].q0 && q < b->ln.seg[s].q1) *sweep_blocks = b->ln.seg[s].blocks;
    }
    return PA_OK;
}

void pa_batch_destroy(pa_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

}  // extern "C"

// ================================================================== serving
extern "C" pa_status pa_serve(const pa_request* reqs, int32_t n, const pa_serve_options* opt,
                              pa_request_result* out, pa_ctx** out_ctx)
{
    if (!reqs || !opt || !out || n < 0 || opt->max_active < 1 || !(opt->time_scale > 0.0) || opt->max_bypass < 0)
        return PA_EINVAL;
    if (opt->keep && !out_ctx) return PA_EINVAL;
    for (int32_t i = 0; i < n; i++) {
        if (i > 0 && reqs[i].arrival_s < reqs[i - 1].arrival_s) return PA_EINVAL;
        std::memset(&out[i], 0, sizeof(out[i]));
        out[i].status = PA_ESTATE;
        if (out_ctx) out_ctx[i] = nullptr;
    }
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    struct Active {
        int32_t idx;
        pa_ctx* ctx;
        size_t fp;
        bool enq_done;
    };
    std::vector<Active> active;
    std::vector<char> admitted((size_t)n, 0);
    size_t used = 0;
    int32_t head = 0, finished = 0;  // head: oldest request not admitted yet
    int32_t head_passed = 0;          // later requests admitted while the head waits
    while (finished < n) {
        bool progress = false;
        // admission: arrived requests in arrival order, within the concurrency
        // limit and the HBM budget; a request that does not fit may be passed
        // by up to max_bypass later ones, after which admission waits for it
        for (int32_t q = head; q < n && reqs[q].arrival_s * opt->time_scale <= now_s() &&
                               (int32_t)active.size() < opt->max_active;
             q++) {
            if (admitted[(size_t)q]) continue;
            const size_t fp = pa_footprint_bytes(&reqs[q].cfg);
            const bool fits = !opt->hbm_budget || active.empty() || used + fp <= opt->hbm_budget;
            if (!fits) {
                if (q == head && head_passed >= opt->max_bypass) break;
                continue;
            }
            pa_request_result& r = out[q];
            r.admit_s = now_s();
            r.footprint = (int64_t)fp;
            pa_ctx* c = nullptr;
            const pa_status st = pa_create(&reqs[q].cfg, nullptr, &c);
            if (st != PA_OK) {
                r.status = st;
                r.finish_s = now_s();
                finished++;
            } else {
                active.push_back({q, c, fp, false});
                used += fp;
            }
            admitted[(size_t)q] = 1;
            if (q != head) head_passed++;
            while (head < n && admitted[(size_t)head]) {
                head++;
                head_passed = 0;
            }
            progress = true;
        }
        // advance every resident run
        for (size_t a = 0; a < active.size();) {
            Active& A = active[a];
            bool retire = false;
            if (!A.enq_done) {
                const pa_status st = pa_step_async(A.ctx);
                if (st == PA_OK) {
                    progress = true;
                } else if (st == PA_DONE) {
                    A.enq_done = true;
                    progress = true;
                } else if (st != PA_EAGAIN) {
                    out[A.idx].status = st;
                    retire = true;
                }
            }
            if (A.enq_done && !retire) {
                const cudaError_t q = cudaStreamQuery(A.ctx->stream);
                if (q == cudaSuccess) {
                    out[A.idx].status = pull_records(A.ctx);
                    retire = true;
                } else if (q != cudaErrorNotReady) {
                    out[A.idx].status = from_cuda(q, __LINE__);
                    retire = true;
                }
            }
            if (retire) {
                pa_request_result& r = out[A.idx];
                r.finish_s = now_s();
                pa_ctx* c = A.ctx;
                r.steps = c->done_rows > 0 ? c->done_rows - 1 : 0;
                double att = 0.0;
                for (long long i = 1; i < c->done_rows; i++)
                    att += (double)c->N * (double)c->cfg.theta * (double)c->recs[(size_t)i].R;
                r.attempts = att;
                if (opt->keep) out_ctx[A.idx] = c;
                else pa_destroy(c);
                used -= A.fp;
                finished++;
                progress = true;
                active.erase(active.begin() + (long)a);
            } else {
                a++;
            }
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    return PA_OK;
}

// ================================================================ checkpoint
// A step boundary is the whole state of a run: the random numbers are
// counter-based, so the population, its levels and families, the
// histograms, the per-step records and the host schedule determine every
// later step. Layout: header, host vectors, then device arrays.
namespace {
constexpr uint64_t kCkptMagic = 0x3130334247415041ull;  // "PAGB3001"

struct CkptHeader {
    uint64_t magic;
    uint32_t version, config_bytes;
    pa_config cfg;
    int64_t step, R, n_betas, n_T, n_sched, hist_steps_saved;
    int32_t done, N;
};

size_t pop_bytes_of(const pa_ctx* c, long long R)
{
    switch (c->h.fmt) {
    case PA_SPIN_MSC32: return (size_t)((R + 31) / 32) * (size_t)c->N * 4;
    case PA_SPIN_REPLICA8: return (((size_t)c->N * (size_t)c->h.cap + 3) / 4) * 4;
    default: return (size_t)R * (size_t)c->h.words * 4;
    }
}

struct Writer {
    char* p;
    size_t cap, used;
    bool ok;
    void put(const void* src, size_t n)
    {
        if (p && used + n <= cap) std::memcpy(p + used, src, n);
        else if (p) ok = false;
        used += n;
    }
};
}  // namespace

extern "C" pa_status pa_checkpoint(pa_ctx* c, void* host_buf, size_t cap, size_t* used)
{
    if (!c || !used) return PA_EINVAL;
    if (c->in_batch) return PA_ESTATE;
    PA_TRY(pull_records(c));
    const long long i = c->enq_step;
    if (c->done_rows != i + 1) return PA_ESTATE;
    const StepDev& last = c->recs[(size_t)i];
    const long long R = last.R;
    const size_t N1 = (size_t)c->h.nlev;
    const long long hs = c->h.hist_rec ? std::min<long long>(i + 1, c->hist_steps) : 0;
    CkptHeader hd{};
    hd.magic = kCkptMagic;
    hd.version = 1;
    hd.config_bytes = sizeof(pa_config);
    hd.cfg = c->cfg;
    hd.step = i;
    hd.R = R;
    hd.n_betas = (int64_t)c->betas.size();
    hd.n_T = (int64_t)c->T4.size();
    hd.n_sched = (int64_t)c->sched.size();
    hd.hist_steps_saved = hs;
    hd.done = c->done ? 1 : 0;
    hd.N = c->N;
    Writer w{(char*)host_buf, host_buf ? cap : 0, 0, true};
    w.put(&hd, sizeof(hd));
    w.put(c->betas.data(), 8 * c->betas.size());
    w.put(c->deltas.data(), 8 * c->deltas.size());
    w.put(c->T4.data(), 8 * c->T4.size());
    w.put(c->T8.data(), 8 * c->T8.size());
    w.put(c->sched.data(), 8 * c->sched.size());
    w.put(c->recs.data(), sizeof(StepDev) * (size_t)(i + 1));
    const int cur = (int)(i & 1);
    struct Dev {
        const void* src;
        size_t bytes;
    };
    const Dev devs[] = {
        {c->h.pop[cur], pop_bytes_of(c, R)},
        {c->h.elev[cur], 4 * (size_t)R},
        {c->h.mlev[cur], 4 * (size_t)R},
        {c->h.fam[cur], 4 * (size_t)R},
        {c->h.H[cur], 8 * N1},
        {c->h.Hsum, 8 * N1},
        {c->h.Msum, 40 * N1},
        {c->h.hist_rec, 8 * N1 * (size_t)hs},
    };
    for (const Dev& d : devs) {
        if (!d.bytes) continue;
        if (w.p && w.used + d.bytes <= w.cap) {
            PA_CUDA(cudaMemcpy(w.p + w.used, d.src, d.bytes, cudaMemcpyDeviceToHost));
        } else if (w.p) {
            w.ok = false;
        }
        w.used += d.bytes;
    }
    *used = w.used;
    if (host_buf && !w.ok) return PA_EINVAL;
    return PA_OK;
}

extern "C" pa_status pa_restore(pa_ctx* c, const void* host_buf, size_t n)
{
    if (!c || !host_buf || n < sizeof(CkptHeader)) return PA_EINVAL;
    if (c->in_batch) return PA_ESTATE;
    CkptHeader hd;
    std::memcpy(&hd, host_buf, sizeof(hd));
    if (hd.magic != kCkptMagic || hd.version != 1 || hd.config_bytes != sizeof(pa_config) || hd.N != c->N)
        return PA_EINVAL;
    pa_config a = hd.cfg, b = c->cfg;
    a.seed = b.seed = 0;  // the seed travels with the checkpoint
    a.use_graph = b.use_graph = 0;
    a.profile = b.profile = 0;
    if (std::memcmp(&a, &b, sizeof(a)) != 0) return PA_EINVAL;
    if (hd.step < 0 || hd.step > c->max_steps || hd.R < 1 || hd.R > c->h.cap) return PA_EINVAL;
    const long long i = hd.step, R = hd.R;
    const size_t N1 = (size_t)c->h.nlev;
    const char* p = (const char*)host_buf + sizeof(hd);
    const char* end = (const char*)host_buf + n;
    auto take = [&](size_t bytes) -> const char* {
        if ((size_t)(end - p) < bytes) return nullptr;
        const char* q = p;
        p += bytes;
        return q;
    };
    const char* pb = take(8 * (size_t)hd.n_betas);
    const char* pd = take(8 * (size_t)hd.n_betas);
    const char* p4 = take(8 * (size_t)hd.n_T);
    const char* p8 = take(8 * (size_t)hd.n_T);
    const char* ps = take(8 * (size_t)hd.n_sched);
    const char* pr = take(sizeof(StepDev) * (size_t)(i + 1));
    if (!pb || !pd || !p4 || !p8 || !ps || !pr) return PA_EINVAL;
    // device state of population i
    PA_CUDA(cudaStreamSynchronize(c->stream));
    const int cur = (int)(i & 1);
    struct Dev {
        void* dst;
        size_t bytes;
    };
    const long long hs = c->h.hist_rec ? std::min<long long>(hd.hist_steps_saved, c->hist_steps) : 0;
    if (hd.hist_steps_saved != hs) return PA_EINVAL;
    const Dev devs[] = {
        {c->h.pop[cur], pop_bytes_of(c, R)},
        {c->h.elev[cur], 4 * (size_t)R},
        {c->h.mlev[cur], 4 * (size_t)R},
        {c->h.fam[cur], 4 * (size_t)R},
        {c->h.H[cur], 8 * N1},
        {c->h.Hsum, 8 * N1},
        {c->h.Msum, 40 * N1},
        {c->h.hist_rec, 8 * N1 * (size_t)hs},
    };
    for (const Dev& d : devs) {
        if (!d.bytes) continue;
        const char* src = take(d.bytes);
        if (!src) return PA_EINVAL;
        PA_CUDA(cudaMemcpy(d.dst, src, d.bytes, cudaMemcpyHostToDevice));
    }
    // records of steps 0..i; later ones cleared
    PA_CUDA(cudaMemset(c->h.rec, 0, sizeof(StepDev) * (size_t)(c->max_steps + 1)));
    PA_CUDA(cudaMemcpy(c->h.rec, pr, sizeof(StepDev) * (size_t)(i + 1), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemset(c->h.status, 0, 16));
    PA_CUDA(cudaMemset(c->h.work, 0, 16));
    const unsigned key[2] = {(unsigned)(hd.cfg.seed & 0xffffffffu), (unsigned)(hd.cfg.seed >> 32)};
    PA_CUDA(cudaMemcpy(c->d_key, key, 8, cudaMemcpyHostToDevice));
    // host state
    c->cfg.seed = hd.cfg.seed;
    c->betas.assign((const double*)pb, (const double*)pb + hd.n_betas);
    c->deltas.assign((const double*)pd, (const double*)pd + hd.n_betas);
    c->T4.assign((const uint64_t*)p4, (const uint64_t*)p4 + hd.n_T);
    c->T8.assign((const uint64_t*)p8, (const uint64_t*)p8 + hd.n_T);
    c->sched.assign((const double*)ps, (const double*)ps + hd.n_sched);
    c->recs.assign((const StepDev*)pr, (const StepDev*)pr + (i + 1));
    c->done_rows = i + 1;
    c->enq_step = i;
    c->done = hd.done != 0;
    c->failed = PA_OK;
    c->stats_pending = false;
    if (c->adaptive && !c->done) PA_TRY(enqueue_readback(c));
    return PA_OK;
}

// 64-bit FNV-1a over the current population in natural layout (one byte
// per spin: 0x01 for +1, 0xff for -1, replica after replica): a compact
// fingerprint for parity checks.
extern "C" pa_status pa_population_hash(pa_ctx* c, uint64_t* out)
{
    if (!c || !out) return PA_EINVAL;
    PA_TRY(pull_records(c));
    const long long R = c->recs[(size_t)(c->done_rows - 1)].R;
    std::vector<int8_t> pop((size_t)R * (size_t)c->N);
    int64_t n = 0;
    PA_TRY(pa_population(c, pop.data(), R, &n));
    uint64_t h = 0xcbf29ce484222325ull;
    for (int8_t v : pop) {
        h ^= (uint64_t)(uint8_t)v;
        h *= 0x100000001b3ull;
    }
    *out = h;
    return PA_OK;
}
