// Internal declarations shared by the engine's kernels and its host code.
//
// Layout of one run in HBM (all buffers sized by the population capacity
// `cap`, so R_i may fluctuate without reallocation):
//   pop[2]      spins, ping-pong between steps. Bit-packed format: per
//               replica 2 * N/64 uint32 words, colour plane 0 then plane 1,
//               site b of a plane at bit b&31 of word b>>5 (bit 1 = spin +1).
//               Byte format: per replica N bytes (0/1), plane 0 then plane 1,
//               padded to a multiple of 16 bytes.
//   elev/mlev   per-slot energy level k = (E+2N)/4 and magnetisation level
//               m = (M+N)/2 of the population in pop[] with the same index.
//   fam[2]      family id (index of the initial replica) per slot.
//   cnt, loc    copy numbers r_j and their exclusive prefix within a tile.
//   tile_sum/off  per-tile totals and their exclusive scan.
//   parent      old slot of every new slot.
//   H[2]        energy and magnetisation histograms (2 x (N+1) uint32),
//               ping-pong by step parity.
//   Hsum        running sum of energy histograms (Sec. 2.4).
//   Msum        per energy level, over all steps: sum |M|, sum M^2, sum M^4
//               (the last two as 128-bit lo/hi), for reweighting magnetisations.
//   bonds       +-J couplings as masks per neighbour direction (same-h, row,
//               up, down) and colour; null for the ferromagnet.
//   tw          level weights t[d] = exp(-4 delta d) (host-computed).
//   F, U        copy tables per energy level: floor(tau_hat), ceil(frac 2^32).
//   thr         per step: T4 - 1 and T8 - 1 (uint32).
//   rec         per-step records read back by the host.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pa {

constexpr int kTile = 1024;            // replicas per copy-count tile
constexpr int kTileThreads = 256;      // 4 replicas (one Philox block) per thread
constexpr int kOneCta = 1024;          // threads of the per-run single-CTA kernels
constexpr long long kSmallCap = 16384; // populations resampled by one CTA in one launch

// device status word values (mirror pa_status)
constexpr int kStatusCapacity = -3;
constexpr int kStatusExtinct = -4;
constexpr int kStatusTimeout = -5;
// bit-packed CTA-group sweeps of replicas up to this many words (the 128 x 128
// square lattice) keep a second shared-memory replica buffer that a bulk copy
// fills with the next replica (measured: +0.4% at L = 128, -0.5% at L = 256)
constexpr int kPrefetchMaxWords = 512;

struct StepDev {
    long long R;              // R_i
    long long R_prev;         // R_{i-1}
    double S;                 // pairwise normaliser used by this step
    int kmin_prev;            // lowest occupied level of population i-1
    int kmin, kmax;           // occupied levels of population i
    int pad0;
    unsigned long long fam;   // number of distinct families in population i
    // sum E, sum E^2, sum |M|, sum M^2, sum M^4 as signed 128-bit (lo, hi)
    unsigned long long sums[10];
};

struct RunDev {
    int L, N, half;           // lattice edge, sites, L/2
    int words;                // uint32 words per replica in pop[]
    int wp;                   // bit-packed words per colour plane (N/64)
    int theta;
    int fmt;                  // 0 byte spins, 1 bit-packed
    int packed;               // byte spins swept by the bit-packed kernels (packed in shared memory)
    int gt;                   // threads per replica in the sweep
    int bw;                   // warps per CTA of a warp-group sweep (0: 8)
    long long R, cap;
    const unsigned* key;      // Philox key (2 words) in device memory
    int ntiles;               // copy-count tiles covering cap
    int record_hist;
    int hist_steps;           // steps with a slot in hist_rec
    int nsteps;               // last step of a fixed schedule (batched runs stop there)
    unsigned unit;            // always 1; a run-time multiplier for the accept-bit insert
    int dim;                  // 2: L x L square lattice; 3: L x L x L simple cubic (N = L^dim)
    int potts_q;              // 0: Ising; 2..8: q-state Potts (byte states 0..q-1, square lattice)
    int estep;                // energy between adjacent levels: 4 (Ising), 1 (Potts)
    int nlev;                 // energy levels k = (E + eoff)/4 = 0 .. dim N/2, and the length of each histogram
    long long eoff;           // E_k = estep k - eoff (dim N for Ising, 2N for Potts)
    uint32_t* pop[2];
    int32_t* elev[2];
    int32_t* mlev[2];
    uint32_t* fam[2];
    uint32_t* parent;
    uint32_t* cnt;
    uint32_t* loc;
    uint32_t* tile_sum;
    uint32_t* tile_off;
    uint32_t* H[2];           // energy histogram (nlev) then magnetisation histogram (nlev, N + 1 used)
    unsigned long long* Hsum;
    unsigned long long* Msum;  // per energy level: sum |M|, sum M^2 (lo, hi), sum M^4 (lo, hi)
    const uint32_t* bonds;    // +-J model, bit-packed: masks [dir][colour][word], bit set = J < 0
    const uint8_t* bonds8;    // +-J model, byte spins: [dir][colour][site], 1 = J < 0
    double* tw;
    uint32_t* F;
    unsigned long long* U;
    uint32_t* thr;            // per step: T4 - 1, T8 - 1
    uint32_t* thr12;          // per step: T12 - 1 (simple cubic lattice only, else null)
    uint32_t* thrp;           // per step: T1 - 1 .. T4 - 1 for dE = 1..4 (Potts only, else null)
    StepDev* rec;
    uint32_t* hist_rec;       // (steps) x 2 x (N+1) when record_hist
    int* status;
    unsigned* work;           // persistent-kernel work counter
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 products with the published multipliers, high halves XORed with
// the other two counter words and the round key; Weyl key increments.
struct PhiloxKey {
    unsigned k0, k1;
};

__device__ __forceinline__ uint4 philox10(uint4 c, PhiloxKey key)
{
    unsigned k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ k0, (unsigned)p1,
                       (unsigned)(p0 >> 32) ^ c.w ^ k1, (unsigned)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// stream tags of the counter's fourth word
constexpr unsigned kTagInit = 0u, kTagSweep = 1u, kTagResample = 2u, kTagPotts = 6u;

// ---------------------------------------------------------------- resampling
// Arguments of the three resampling kernels (copy numbers, tile scan, parent
// scatter). The old population size is read from device memory (n_old_dev,
// as inside a captured run) or taken by value when n_old_dev is null.
struct ResampleArgs {
    const long long* n_old_dev;
    long long n_old;
    const int32_t* lev;              // energy level of every old slot
    const uint32_t* F;               // floor(tau_hat) per level
    const unsigned long long* U;     // ceil(frac(tau_hat) 2^32) per level
    const unsigned* key;             // Philox key (2 words, device)
    unsigned step;                   // temperature step i (RESAMPLE counter word 0)
    uint32_t* cnt;                   // r_j
    uint32_t* loc;                   // exclusive prefix of r_j within its tile
    uint32_t* tile_sum;
    uint32_t* tile_off;
    uint32_t* parent;                // new slot -> old slot
    long long cap;                   // capacity of parent
    long long* n_new;                // R_i (device)
    long long* n_prev_out;           // R_{i-1} echo (device, may be null)
    int* status;                     // set to kStatusCapacity / kStatusExtinct
    unsigned* work;                  // persistent-kernel counter reset for the sweep (may be null)
};

// ---------------------------------------------------------------- batches
// Many independent runs stepped together: one launch per phase for all runs.
constexpr int kMaxBatchRuns = 1024;
constexpr int kMaxBatchSegs = 16;     // (L, threads per replica) shapes of one batch
struct BatchDev {
    const RunDev* runs;       // device array of the runs' descriptors
    const int* order;         // runs in queue order (by shape, then descending work per replica)
    const int* tile_run;      // copy-count tile -> run
    const int* tile_first;    // first copy-count tile of each run
    long long* item_off;      // nruns + 1 offsets of each run's work items (queue order)
    unsigned* work;           // queue counter of each segment of the sweep
    int nruns;
    int nseg;                 // queue segments (runs of one shape)
};

// ---------------------------------------------------------------- launches
struct Launch {
    int sweep_blocks, sweep_threads;  // persistent sweep grid
    int count_blocks;                 // tiles over cap
    size_t sweep_smem;
    const void* sweep_cover;          // sweep instance with one fixed replica per group (grid holds the
                                      // whole capacity), or null
    bool sweep_full;                  // the grid is all the device keeps resident (a full population
                                      // has at least that many work items)
};

cudaError_t launch_init(const RunDev* d_run, const RunDev& h, const Launch& ln, cudaStream_t s);
cudaError_t launch_tables(const RunDev* d_run, const RunDev& h, int step, cudaStream_t s);
cudaError_t launch_counts(const RunDev* d_run, const RunDev& h, const Launch& ln, int step, cudaStream_t s);
cudaError_t launch_scan(const RunDev* d_run, const RunDev& h, int step, cudaStream_t s);
cudaError_t launch_parent(const RunDev* d_run, const RunDev& h, const Launch& ln, int step, cudaStream_t s);
// the same three kernels on plain arguments; tiles = blocks covering the
// largest old population the launch may see
cudaError_t launch_resample(const ResampleArgs& a, int tiles, cudaStream_t s);
// pdl: launch with programmatic serialization (the kernel may be scheduled
// while the previous kernel of the stream runs; it waits for that kernel's
// completion before touching memory)
cudaError_t launch_sweep(const RunDev* d_run, const RunDev& h, const Launch& ln, int step, cudaStream_t s,
                         bool pdl = false);
cudaError_t launch_stats(const RunDev* d_run, const RunDev& h, int step, cudaStream_t s);
// statistics of step-1 (optional), tables, copy numbers, offsets and parents
// of step `step` in one single-CTA launch (capacity <= kSmallCap)
cudaError_t launch_resample_small(const RunDev& h, int step, bool with_stats, cudaStream_t s, bool pdl = false);
cudaError_t launch_rng_peak(long long blocks, uint32_t* sink, int grid, int threads, cudaStream_t s);
// the bulk-copy path with a bounded wait, with or without the copy (out[0]:
// 0 landed and equal, kStatusTimeout wait ran out, 1 landed but different)
cudaError_t launch_bulk_selftest(const uint32_t* src, int bytes, bool copy, int tries, int* out, cudaStream_t s);
cudaError_t launch_pipe_peak(int pipe, long long iters, uint32_t* sink, int grid, int threads, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, long long n, PhiloxKey key, uint32_t* out, cudaStream_t s);
cudaError_t launch_gather(const uint32_t* src, const uint32_t* parent, long long n_new, long long n_src, int words,
                          uint32_t* dst, unsigned* bad, int grid, cudaStream_t s);

// one segment of the batched sweep: queue positions [q0, q1), shape (L, G)
struct BatchSeg {
    int q0, q1, L, G;
    int blocks;               // persistent CTAs (256 threads)
    size_t smem;
};
constexpr int kBatchOwnStreams = 4;  // side streams taking the own-kernel runs' sweeps in turn
struct BatchLaunch {
    int tiles;                // copy-count tiles over all runs
    bool small;               // every run's capacity <= kSmallCap: one-CTA resampling per run
    int last;                 // the batch's last step
    int nseg;
    BatchSeg seg[kMaxBatchSegs];
    cudaStream_t side[kMaxBatchSegs];  // one stream per segment (branches of the graph)
    cudaEvent_t fork, join[kMaxBatchSegs];
    // runs that fill the device alone (all runs of one replica per CTA, and
    // warp-group runs whose sweep grid is all the device keeps resident),
    // each swept by its own sweep kernel (the one it runs alone with), in
    // queue order
    int nown;
    const RunDev* own_h;    // their descriptors (host array of nown)
    const Launch* own_ln;   // their sweep plans
    const int* own_last;    // their last steps
    cudaStream_t own_side[kBatchOwnStreams];
    cudaEvent_t own_join[kBatchOwnStreams];
};
cudaError_t plan_batch_segment(BatchSeg* seg, long long units);
cudaError_t launch_batch_step(const BatchDev& b, const BatchLaunch& ln, int step, cudaStream_t s, int phase,
                              int* phase_of_launch);
bool batch_phase_launches(const BatchLaunch& ln, int step, int phase);
bool batch_supports(int L, int gt);

#ifdef PA_GB300_H
// Autotuner (pa_tune.cu): the launch shape chosen in this process for runs
// like cfg (batched != 0: the batched sweep), and the tuner itself.
bool tuned_shape(const pa_config& cfg, int batched, int* G, int* bw);
pa_status autotune_impl(const pa_config* cfg, int batched, const char* cache_path, void* stream, pa_tune_choice* out);
#endif

// Sweep launch shape: persistent CTAs for this run (group threads gt).
cudaError_t plan_sweep(const RunDev& h, Launch* ln);
const void* sweep_kernel(const RunDev& h, bool init);

}  // namespace pa
