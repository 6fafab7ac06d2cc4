// Device kernels of the population-annealing engine (2D Ising, sm_103a).
//
// One temperature step i >= 1 (Sec. 2.1 steps 2-4) is six launches:
//   k_tables  (1 CTA)   S = pairwise sum of H_{i-1}[k] t[k-kmin]  (Eq. Q) and
//                       the copy tables F = floor(tau_hat), U = ceil(frac 2^32)
//                       (Eq. resampling-factors)
//   k_counts            r_j = F[k_j] + [x_j < U[k_j]], tile-local prefix
//   k_scan    (1 CTA)   tile offsets, R_i, capacity check
//   k_parent            parent[o_j + c] = j for c < r_j
//   k_sweep             gather parent into shared memory, theta checkerboard
//                       Metropolis sweeps, E and M by popcount, histograms
//   k_stats   (1 CTA)   integer moments, occupied range, running histogram sum
// Everything except S and the copy tables is integer arithmetic; S and the
// tables use only IEEE +, x, / with round-to-nearest intrinsics in a fixed
// order, so every result is reproducible bit for bit.
//
// Every kernel returns at once if the run's status word is set, so a failure
// at step i leaves rows 0..i-1 intact and the rest of a captured graph inert.
#include "pa_internal.cuh"

#include <algorithm>
#include <cstdio>

namespace pa {

// ======================================================== programmatic dependent launch
// A kernel launched with the programmatic-serialization attribute may be
// scheduled while the kernel before it in the stream is still running.
// pdl_wait() returns once that kernel has completed and its writes are
// visible (for a kernel launched without the attribute there is nothing to
// wait for and it returns at once); every kernel that can be launched so
// calls it before touching memory. pdl_trigger() lets the next kernel of the
// stream be scheduled early: it is issued right after the wait, so at most
// one kernel waits ahead of the one that runs.
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ======================================================== bit-packed geometry
constexpr uint32_t row_first_mask(int hb)
{
    uint32_t m = 0;
    for (int p = 0; p < 32; p += hb) m |= 1u << p;
    return m;
}
constexpr uint32_t row_odd_mask(int hb)
{
    uint32_t m = 0;
    for (int p = 0; p < 32; p++)
        if ((p / hb) & 1) m |= 1u << p;
    return m;
}

// Colour plane c holds the N/2 sites with (x + y) & 1 == c; site (x, y) is
// bit b = y*L/2 + x/2 of its plane. All four neighbours lie in the other
// plane: (x, y+-1) at b +- L/2, and along the row the same b plus b+1 when x
// is odd or b-1 when x is even (cyclic within the row).
template <int L>
struct Geo {
    static constexpr int N = L * L;
    static constexpr int HB = L / 2;           // bits per plane row
    static constexpr int WP = N / 64;          // words per plane
    static constexpr int WORDS = N / 32;       // words per replica
    static constexpr bool WIDE = HB >= 32;     // a row spans whole words
    static constexpr int WR = WIDE ? HB / 32 : 1;
    static constexpr uint32_t FIRST = WIDE ? 0u : row_first_mask(HB);
    static constexpr uint32_t LAST = WIDE ? 0u : (row_first_mask(HB) << (HB - 1));
    static constexpr uint32_t ODD = WIDE ? 0u : row_odd_mask(HB);
};

// The four neighbour words of word w of plane c; O is the other plane.
template <int L>
__device__ __forceinline__ void neighbours(const uint32_t* __restrict__ O, int c, int w, uint32_t& same,
                                           uint32_t& side, uint32_t& up, uint32_t& down)
{
    using G = Geo<L>;
    same = O[w];
    if constexpr (G::WIDE) {
        up = O[w >= G::WR ? w - G::WR : w - G::WR + G::WP];
        down = O[w + G::WR < G::WP ? w + G::WR : w + G::WR - G::WP];
        const int y = w / G::WR;
        const int pos = w - y * G::WR;
        if ((c + y) & 1) {  // x odd: neighbours at h and h + 1
            const int wn = (pos == G::WR - 1) ? w - (G::WR - 1) : w + 1;
            side = __funnelshift_r(same, O[wn], 1);
        } else {            // x even: neighbours at h and h - 1
            const int wv = (pos == 0) ? w + (G::WR - 1) : w - 1;
            side = __funnelshift_l(O[wv], same, 1);
        }
    } else {
        // several rows per word; word-row parity is even (32/HB is even)
        const uint32_t prev = O[w > 0 ? w - 1 : G::WP - 1];
        const uint32_t next = O[w + 1 < G::WP ? w + 1 : 0];
        up = (same << G::HB) | (prev >> (32 - G::HB));
        down = (same >> G::HB) | (next << (32 - G::HB));
        const uint32_t plus = ((same >> 1) & ~G::LAST) | ((same << (G::HB - 1)) & G::LAST);
        const uint32_t minus = ((same << 1) & ~G::FIRST) | ((same >> (G::HB - 1)) & G::FIRST);
        // colour 0: odd rows have x odd; colour 1: even rows have x odd
        side = c ? ((plus & ~G::ODD) | (minus & G::ODD)) : ((plus & G::ODD) | (minus & ~G::ODD));
    }
}

// Word counts of a bit-packed replica: the L x L square lattice (D = 2) or
// the L x L x L simple cubic one (D = 3). Layer z of a simple cubic colour
// plane is laid out like a square-lattice plane (WPL words).
template <int L, int D>
struct Lat {
    static constexpr int N = D == 3 ? L * L * L : L * L;
    static constexpr int WP = N / 64;       // words per colour plane
    static constexpr int WORDS = N / 32;    // words per replica
    static constexpr int WPL = L * L / 64;  // words per colour plane and layer
};

// The six neighbour words of word w of plane c on the simple cubic lattice.
// Within layer z the sites of colour c have x = c + z + y (mod 2), so the
// in-layer neighbours are the square lattice's for colour (c + z) & 1; the
// other two are the same word of layers z - 1 and z + 1.
template <int L>
__device__ __forceinline__ void neighbours3(const uint32_t* __restrict__ O, int c, int w, uint32_t& same,
                                            uint32_t& side, uint32_t& up, uint32_t& down, uint32_t& zup,
                                            uint32_t& zdn)
{
    constexpr int WPL = Lat<L, 3>::WPL;
    const int z = w / WPL, wl = w - z * WPL;
    neighbours<L>(O + z * WPL, (c + z) & 1, wl, same, side, up, down);
    zup = O[(z == 0 ? L - 1 : z - 1) * WPL + wl];
    zdn = O[(z == L - 1 ? 0 : z + 1) * WPL + wl];
}

// Sets bit T of acc when x <= thr. The 32 accept bits of a word are
// disjoint, so the insert can be an addition: a predicated multiply-add by
// the run-time constant unit (always 1) issues on the FMA pipe, which the
// update leaves less busy than the integer/logic pipe the compares and
// neighbour logic occupy (a compile-time 1 would be folded back into a
// logic op).
template <int T>
__device__ __forceinline__ uint32_t accept_bit(uint32_t acc, uint32_t x, uint32_t thr, uint32_t unit)
{
    asm("{\n\t.reg .pred p;\n\tsetp.le.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %4, %0;\n\t}"
        : "+r"(acc)
        : "r"(x), "r"(thr), "r"(unit), "n"(1u << T));
    return acc;
}

// Bits 4q .. 4q+3 of acc4 (x <= T4-1) and acc8 (x <= T8-1) from Philox
// block c0 + q, then blocks q+1 .. NQ-1
template <int Q, int NQ = 8>
__device__ __forceinline__ void accept_blocks(uint32_t& acc4, uint32_t& acc8, unsigned c0, unsigned k, unsigned c2,
                                              uint32_t t4m1, uint32_t t8m1, uint32_t unit, PhiloxKey key)
{
    if constexpr (Q < NQ) {
        const uint4 x = philox10(make_uint4(c2, c0 + Q, kTagSweep, k), key);
        acc4 = accept_bit<4 * Q + 0>(acc4, x.x, t4m1, unit);
        acc8 = accept_bit<4 * Q + 0>(acc8, x.x, t8m1, unit);
        acc4 = accept_bit<4 * Q + 1>(acc4, x.y, t4m1, unit);
        acc8 = accept_bit<4 * Q + 1>(acc8, x.y, t8m1, unit);
        acc4 = accept_bit<4 * Q + 2>(acc4, x.z, t4m1, unit);
        acc8 = accept_bit<4 * Q + 2>(acc8, x.z, t8m1, unit);
        acc4 = accept_bit<4 * Q + 3>(acc4, x.w, t4m1, unit);
        acc8 = accept_bit<4 * Q + 3>(acc8, x.w, t8m1, unit);
        accept_blocks<Q + 1, NQ>(acc4, acc8, c0, k, c2, t4m1, t8m1, unit, key);
    }
}

// One Metropolis update of the 32 sites of word s (all of one colour).
// A site with n aligned neighbours flips with certainty if n <= 2 (dE <= 0),
// with x <= T4-1 if n = 3 and x <= T8-1 if n = 4, x the SWEEP word of the
// site: counter (2u + c, b>>2, 1, k), lane b&3. Only counter word 1 differs
// between the lanes of a warp, so the first-round products are warp-uniform.
// Bit-sliced counting of the disagreeing neighbours d1..d4 gives "at least
// two disagree" (n <= 2) and "none disagrees" (n = 4) for all 32 sites at
// once. Each site's word is compared with both thresholds into two words of
// accept bits, and the count picks between them for all 32 sites with two
// logic ops: cheaper than selecting a threshold per site.
__device__ __forceinline__ uint32_t metropolis_word(uint32_t s, uint32_t same, uint32_t side, uint32_t up,
                                                    uint32_t down, unsigned c0, unsigned k, unsigned c2,
                                                    uint32_t t4m1, uint32_t t8m1, uint32_t unit, PhiloxKey key)
{
    const uint32_t d1 = s ^ same, d2 = s ^ side, d3 = s ^ up, d4 = s ^ down;
    const uint32_t a = d1 ^ d2, b = d1 & d2, cc = d3 ^ d4, e = d3 & d4;
    const uint32_t ge2 = b | e | (a & cc);
    const uint32_t eq0 = ~(d1 | d2 | d3 | d4);
    uint32_t acc4 = 0, acc8 = 0;
    accept_blocks<0>(acc4, acc8, c0, k, c2, t4m1, t8m1, unit, key);
    return s ^ (ge2 | (acc4 & ~eq0) | (acc8 & eq0));
}

// The update of metropolis_word shared by S lanes (small lattices, where a
// population has too few words to occupy the GPU): lane `sub` of the S
// evaluates Philox blocks sub*8/S .. (sub+1)*8/S - 1 of the word (counter
// word 1 = 8w + block, as in metropolis_word) into its bits of the accept
// words, which the S lanes (adjacent lanes of the group, mask gmask) then
// OR together. Every lane returns the same new word.
template <int S>
__device__ __forceinline__ uint32_t metropolis_word_split(uint32_t s, uint32_t same, uint32_t side, uint32_t up,
                                                          uint32_t down, unsigned w8, int sub, unsigned k,
                                                          unsigned c2, uint32_t t4m1, uint32_t t8m1, uint32_t unit,
                                                          PhiloxKey key, unsigned gmask)
{
    constexpr int QPL = 8 / S;  // Philox blocks per lane
    const uint32_t d1 = s ^ same, d2 = s ^ side, d3 = s ^ up, d4 = s ^ down;
    const uint32_t a = d1 ^ d2, b = d1 & d2, cc = d3 ^ d4, e = d3 & d4;
    const uint32_t ge2 = b | e | (a & cc);
    const uint32_t eq0 = ~(d1 | d2 | d3 | d4);
    uint32_t acc4 = 0, acc8 = 0;
    accept_blocks<0, QPL>(acc4, acc8, w8 + (unsigned)(sub * QPL), k, c2, t4m1, t8m1, unit, key);
    acc4 <<= 4 * QPL * sub;
    acc8 <<= 4 * QPL * sub;
#pragma unroll
    for (int off = 1; off < S; off <<= 1) {
        acc4 |= __shfl_xor_sync(gmask, acc4, off);
        acc8 |= __shfl_xor_sync(gmask, acc8, off);
    }
    return s ^ (ge2 | (acc4 & ~eq0) | (acc8 & eq0));
}

// Bits 4q .. 4q+3 of acc4, acc8 and acc12 (x <= T4-1, T8-1, T12-1) from
// Philox block q, then blocks q+1 .. 7
template <int Q>
__device__ __forceinline__ void accept_blocks3(uint32_t& acc4, uint32_t& acc8, uint32_t& acc12, unsigned c0,
                                               unsigned k, unsigned c2, uint32_t t4m1, uint32_t t8m1,
                                               uint32_t t12m1, uint32_t unit, PhiloxKey key)
{
    if constexpr (Q < 8) {
        const uint4 x = philox10(make_uint4(c2, c0 + Q, kTagSweep, k), key);
        acc4 = accept_bit<4 * Q + 0>(acc4, x.x, t4m1, unit);
        acc8 = accept_bit<4 * Q + 0>(acc8, x.x, t8m1, unit);
        acc12 = accept_bit<4 * Q + 0>(acc12, x.x, t12m1, unit);
        acc4 = accept_bit<4 * Q + 1>(acc4, x.y, t4m1, unit);
        acc8 = accept_bit<4 * Q + 1>(acc8, x.y, t8m1, unit);
        acc12 = accept_bit<4 * Q + 1>(acc12, x.y, t12m1, unit);
        acc4 = accept_bit<4 * Q + 2>(acc4, x.z, t4m1, unit);
        acc8 = accept_bit<4 * Q + 2>(acc8, x.z, t8m1, unit);
        acc12 = accept_bit<4 * Q + 2>(acc12, x.z, t12m1, unit);
        acc4 = accept_bit<4 * Q + 3>(acc4, x.w, t4m1, unit);
        acc8 = accept_bit<4 * Q + 3>(acc8, x.w, t8m1, unit);
        acc12 = accept_bit<4 * Q + 3>(acc12, x.w, t12m1, unit);
        accept_blocks3<Q + 1>(acc4, acc8, acc12, c0, k, c2, t4m1, t8m1, t12m1, unit, key);
    }
}

// One Metropolis update of the 32 sites of word s on the simple cubic
// lattice: with n of the six neighbours aligned, dE = 4n - 12, so a site
// flips with certainty if at most 3 neighbours agree (3 or more disagree),
// else iff x <= T4-1, T8-1, T12-1 for 2, 1, 0 disagreeing neighbours; x is
// the SWEEP word of the site, as on the square lattice. The disagreeing
// neighbours are counted bit-sliced (two full adders of three, then the
// carries), 4 b2 + 2 b1 + b0.
__device__ __forceinline__ uint32_t metropolis_word3(uint32_t s, uint32_t n1, uint32_t n2, uint32_t n3,
                                                     uint32_t n4, uint32_t n5, uint32_t n6, unsigned c0,
                                                     unsigned k, unsigned c2, uint32_t t4m1, uint32_t t8m1,
                                                     uint32_t t12m1, uint32_t unit, PhiloxKey key)
{
    const uint32_t d1 = s ^ n1, d2 = s ^ n2, d3 = s ^ n3, d4 = s ^ n4, d5 = s ^ n5, d6 = s ^ n6;
    const uint32_t sa = d1 ^ d2 ^ d3, ca = (d1 & d2) | (d3 & (d1 ^ d2));
    const uint32_t sb = d4 ^ d5 ^ d6, cb = (d4 & d5) | (d6 & (d4 ^ d5));
    const uint32_t b0 = sa ^ sb, k0 = sa & sb;
    const uint32_t b1 = ca ^ cb ^ k0, b2 = (ca & cb) | (k0 & (ca ^ cb));
    const uint32_t ge3 = b2 | (b1 & b0);
    const uint32_t eq2 = ~b2 & b1 & ~b0, eq1 = ~b2 & ~b1 & b0, eq0 = ~(b2 | b1 | b0);
    uint32_t acc4 = 0, acc8 = 0, acc12 = 0;
    accept_blocks3<0>(acc4, acc8, acc12, c0, k, c2, t4m1, t8m1, t12m1, unit, key);
    return s ^ (ge3 | (acc4 & eq2) | (acc8 & eq1) | (acc12 & eq0));
}

// ======================================================== bulk copies
// One-dimensional bulk copy global -> shared memory through the tensor-memory
// accelerator (cp.async.bulk), completion tracked by an mbarrier in shared
// memory (expect-tx bytes; the barrier's phase flips when they have landed).
// Every wait is bounded: after kBulkWaitTries failed polls the caller gets
// false and reports a timeout instead of spinning on.
constexpr int kBulkWaitTries = 1 << 20;

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* m)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// issued by one thread: the barrier expects `bytes`, the copy delivers them
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* m)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order earlier generic accesses of dst
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}

// wait until the barrier has completed the phase with this parity
__device__ __forceinline__ bool mbar_wait(unsigned long long* m, unsigned parity, int tries = kBulkWaitTries)
{
    for (int i = 0; i < tries; i++) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(m)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// the next replica's load, issued by thread 0 once the current replica's
// first colour phase is done (src null: no next replica)
struct Prefetch {
    const uint32_t* src;
    uint32_t* dst;
    unsigned long long* mbar;
    unsigned bytes;
};

// ======================================================== shared epilogue
// 128-bit unsigned accumulation (lo, hi) with an explicit carry: integer
// addition is associative, so the total does not depend on the order.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* lohi, unsigned long long lo,
                                                unsigned long long hi)
{
    const unsigned long long old = atomicAdd(&lohi[0], lo);
    if (old + lo < old) hi += 1ull;
    if (hi) atomicAdd(&lohi[1], hi);
}

// Record a finished replica from its energy level kl, magnetisation level
// ml and magnetisation M: levels, histograms, family, and the per-level
// magnetisation sums used to reweight magnetisations (Sec. 2.4).
__device__ __forceinline__ void record_levels(const RunDev& r, int nxt, long long k, int kl, int ml, long long M,
                                              uint32_t family)
{
    r.elev[nxt][k] = kl;
    r.mlev[nxt][k] = ml;
    r.fam[nxt][k] = family;
    atomicAdd(&r.H[nxt][kl], 1u);
    atomicAdd(&r.H[nxt][r.nlev + ml], 1u);
    const unsigned long long aM = (unsigned long long)(M < 0 ? -M : M);
    const unsigned long long M2 = aM * aM;
    const unsigned __int128 M4 = (unsigned __int128)M2 * M2;
    unsigned long long* ms = r.Msum + 5 * (size_t)kl;
    atomicAdd(&ms[0], aM);
    atomic_add_u128(ms + 1, M2, 0ull);
    atomic_add_u128(ms + 3, (unsigned long long)M4, (unsigned long long)(M4 >> 64));
}

// Ising spins: anti-parallel bonds and up spins give kl = (E + dim N)/4 with
// E = 2*anti - dim N, ml = (M + N)/2 = ups and M = 2*ups - N.
__device__ __forceinline__ void record_replica(const RunDev& r, int nxt, long long k, unsigned anti, unsigned ups,
                                               uint32_t family)
{
    record_levels(r, nxt, k, (int)(anti >> 1), (int)ups, 2ll * (long long)ups - r.N, family);
}

template <int G>
__device__ __forceinline__ unsigned group_sum(unsigned v)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int WORDS, int G>
__device__ __forceinline__ void copy_words(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, int gl)
{
    if constexpr (WORDS % 4 == 0) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (int i = gl; i < WORDS / 4; i += G) d4[i] = s4[i];
    } else {
        for (int i = gl; i < WORDS; i += G) dst[i] = src[i];
    }
}

// A replica stored one byte per site (0/1, colour plane 0 then plane 1,
// site b of a plane at byte b) and the same replica bit-packed (site b of a
// plane at bit b&31 of word b>>5): word i of the packed image holds bytes
// 32i .. 32i+31 of the byte image, bit j = byte 32i + j.
__device__ __forceinline__ uint32_t nibble_of(uint32_t v)  // bytes 0..3 of v (each 0/1) -> bits 0..3
{
    return (v & 1u) | ((v >> 7) & 2u) | ((v >> 14) & 4u) | ((v >> 21) & 8u);
}

__device__ __forceinline__ uint32_t bytes_of(uint32_t n)  // bits 0..3 of n -> bytes 0..3 (0/1)
{
    return (n & 1u) | ((n & 2u) << 7) | ((n & 4u) << 14) | ((n & 8u) << 21);
}

template <int WORDS, int G>
__device__ __forceinline__ void pack_bytes(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, int gl)
{
    for (int i = gl; i < WORDS; i += G) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src + 8 * i);
        const uint4 a = s4[0], b = s4[1];
        dst[i] = nibble_of(a.x) | nibble_of(a.y) << 4 | nibble_of(a.z) << 8 | nibble_of(a.w) << 12 |
                 nibble_of(b.x) << 16 | nibble_of(b.y) << 20 | nibble_of(b.z) << 24 | nibble_of(b.w) << 28;
    }
}

template <int WORDS, int G>
__device__ __forceinline__ void unpack_bytes(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, int gl)
{
    for (int i = gl; i < WORDS; i += G) {
        const uint32_t w = src[i];
        uint4* d4 = reinterpret_cast<uint4*>(dst + 8 * i);
        d4[0] = make_uint4(bytes_of(w), bytes_of(w >> 4), bytes_of(w >> 8), bytes_of(w >> 12));
        d4[1] = make_uint4(bytes_of(w >> 16), bytes_of(w >> 20), bytes_of(w >> 24), bytes_of(w >> 28));
    }
}

// a replica of the population in pop[] (bit-packed, or bytes when kBytes)
// into the packed shared-memory image, and back
template <int L, int G, int D, bool kBytes>
__device__ __forceinline__ void load_replica(uint32_t* sp, const uint32_t* pop, long long slot, int gl)
{
    using Gm = Lat<L, D>;
    if constexpr (kBytes) pack_bytes<Gm::WORDS, G>(sp, pop + (size_t)slot * (Gm::N / 4), gl);
    else copy_words<Gm::WORDS, G>(sp, pop + (size_t)slot * Gm::WORDS, gl);
}

template <int L, int G, int D, bool kBytes>
__device__ __forceinline__ void store_replica(uint32_t* pop, long long slot, const uint32_t* sp, int gl)
{
    using Gm = Lat<L, D>;
    if constexpr (kBytes) unpack_bytes<Gm::WORDS, G>(pop + (size_t)slot * (Gm::N / 4), sp, gl);
    else copy_words<Gm::WORDS, G>(pop + (size_t)slot * Gm::WORDS, sp, gl);
}

// anti-parallel bonds and up spins of the replica in shared memory
// +-J model: a neighbour word seen through the couplings (bit flipped where
// J < 0), so "disagree" means an unsatisfied bond in every formula below
template <int L>
__device__ __forceinline__ void apply_bonds(const uint32_t* __restrict__ bonds, int c, int w, uint32_t& same,
                                            uint32_t& side, uint32_t& up, uint32_t& down)
{
    constexpr int WP = Geo<L>::WP;
    const uint32_t* B = bonds + c * WP + w;
    same ^= __ldg(B);
    side ^= __ldg(B + 2 * WP);
    up ^= __ldg(B + 4 * WP);
    down ^= __ldg(B + 6 * WP);
}

template <int L, int G, int D = 2>
__device__ __forceinline__ void measure_bits(const uint32_t* sp, int gl, unsigned& anti, unsigned& ups,
                                             const uint32_t* __restrict__ bonds)
{
    using Gm = Lat<L, D>;
    anti = 0;
    ups = 0;
    for (int w = gl; w < Gm::WP; w += G) {
        const uint32_t s = sp[w];
        if constexpr (D == 3) {
            uint32_t same, side, up, down, zup, zdn;
            neighbours3<L>(sp + Gm::WP, 0, w, same, side, up, down, zup, zdn);
            anti += __popc(s ^ same) + __popc(s ^ side) + __popc(s ^ up) + __popc(s ^ down) + __popc(s ^ zup) +
                    __popc(s ^ zdn);
        } else {
            uint32_t same, side, up, down;
            neighbours<L>(sp + Gm::WP, 0, w, same, side, up, down);
            if (bonds) apply_bonds<L>(bonds, 0, w, same, side, up, down);
            anti += __popc(s ^ same) + __popc(s ^ side) + __popc(s ^ up) + __popc(s ^ down);
        }
        ups += __popc(s) + __popc(sp[Gm::WP + w]);
    }
}

// ======================================================== replica groups
// G threads update one replica held in shared memory. G <= 32: 32/G groups
// per warp and the colour phases synchronise with __syncwarp. G > 32: one
// group per CTA (blockDim == G) synchronising with __syncthreads; such a
// kernel also needs 33 words of shared memory after the replica (reduction
// and broadcast).
template <int G>
struct Group {
    static constexpr bool kCta = G > 32;
    static constexpr int kPerWarp = kCta ? 1 : 32 / G;
    __device__ static __forceinline__ void sync()
    {
        if constexpr (kCta) __syncthreads();
        else __syncwarp();
    }
    // total over the group's threads, returned to every thread
    __device__ static __forceinline__ unsigned sum(unsigned v, unsigned* red)
    {
        if constexpr (kCta) {
            v = group_sum<32>(v);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
            __syncthreads();
            unsigned t = 0;
#pragma unroll
            for (int w = 0; w < G / 32; w++) t += red[w];
            return t;
        } else {
            return group_sum<G>(v);
        }
    }
    // Work items of a persistent loop: every group of the grid starts with
    // a fixed replica (first_item; static_items of them in all), and takes
    // further ones from the run's counter (grab() + static_items()), so the
    // counter is touched only by groups that finish while work remains.
    __device__ static __forceinline__ unsigned first_item()
    {
        if constexpr (kCta) return blockIdx.x;
        else return (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kPerWarp + (threadIdx.x & 31) / G;
    }
    __device__ static __forceinline__ unsigned static_items()
    {
        return kCta ? gridDim.x : gridDim.x * (blockDim.x >> 5) * kPerWarp;
    }
    // first replica index of this group's next work item (persistent loop)
    __device__ static __forceinline__ unsigned grab(unsigned* work, unsigned* bcast)
    {
        if constexpr (kCta) {
            __syncthreads();
            if (threadIdx.x == 0) *bcast = atomicAdd(work, 1u);
            __syncthreads();
            return *bcast;
        } else {
            unsigned base = 0;
            if ((threadIdx.x & 31) == 0) base = atomicAdd(work, (unsigned)kPerWarp);
            return __shfl_sync(0xffffffffu, base, 0) + (threadIdx.x & 31) / G;
        }
    }
    __device__ static __forceinline__ int thread_in_group()
    {
        return kCta ? (int)threadIdx.x : (int)(threadIdx.x & 31) % G;
    }
    // this group's replica buffer within the CTA's shared memory
    __device__ static __forceinline__ uint32_t* buffer(uint32_t* smem, int words)
    {
        if constexpr (kCta) return smem;
        else return smem + ((threadIdx.x >> 5) * kPerWarp + (threadIdx.x & 31) / G) * words;
    }
};

// One temperature step of the replica in new slot k (gather of its parent,
// theta sweeps, measurement, write-back). Every thread of the group calls
// this, active or not (inactive groups only take part in the syncs).
// Threads per replica that a bit-packed lattice supports: a power of two
// dividing the plane's words (each thread owns whole words), or, on the
// square lattice, 2..8 threads per word (G = S * words per plane <= 32)
// sharing each word's eight Philox blocks.
template <int L, int D>
__host__ __device__ constexpr bool bits_group_ok(int G)
{
    constexpr int WP = Lat<L, D>::WP;
    if (G < 1 || (G & (G - 1))) return false;
    if (WP % G == 0) return true;
    return D == 2 && G <= 32 && G % WP == 0 && G / WP <= 8;
}

// kBytes: the population is stored one byte per site (PA_SPIN_INT8) and
// packed into the same shared-memory words on load, unpacked on store.
// pf (CTA groups): the replica is already in sp (loaded by a bulk copy),
// and pf describes the next replica's bulk copy, issued after the first
// colour phase; null: load the replica here.
template <int L, int G, int D = 2, bool kBytes = false>
__device__ __forceinline__ void bits_group_step(const RunDev& r, int step, long long k, bool active,
                                                uint32_t* sp, int gl, unsigned* red, unsigned& families,
                                                const Prefetch* pf = nullptr)
{
    using Gm = Lat<L, D>;
    using Gr = Group<G>;
    static_assert(bits_group_ok<L, D>(G), "unsupported threads per replica");
    constexpr bool kSplit = G > Gm::WP;             // several lanes per word
    constexpr int S = kSplit ? G / Gm::WP : 1;      // lanes per word
    constexpr int WPT = kSplit ? 1 : Gm::WP / G;    // words per thread per plane
    const int cur = (step - 1) & 1, nxt = step & 1;
    const uint32_t t4m1 = r.thr[2 * step], t8m1 = r.thr[2 * step + 1];
    uint32_t t12m1 = 0;
    if constexpr (D == 3) t12m1 = r.thr12[step];
    const PhiloxKey key{r.key[0], r.key[1]};
    const int theta = r.theta;
    const unsigned u0 = (unsigned)(step - 1) * (unsigned)theta;
    const uint32_t* __restrict__ bonds = r.bonds;
    // read once: batched runs pass r in global memory, where a load inside
    // the update loop would be repeated for every word
    const uint32_t unit = r.unit;
    uint32_t p = 0;
    if (active) {
        p = r.parent[k];
        if (!pf) load_replica<L, G, D, kBytes>(sp, r.pop[cur], p, gl);
    }
    Gr::sync();
    for (int sw = 0; sw < theta; sw++) {
        const unsigned u = u0 + (unsigned)sw;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            if constexpr (kSplit) {
                if (active) {
                    uint32_t* P = sp + c * Gm::WP;
                    const uint32_t* O = sp + (1 - c) * Gm::WP;
                    const int w = gl / S, sub = gl - (gl / S) * S;
                    const unsigned gmask = G == 32 ? 0xffffffffu
                                                   : ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
                    uint32_t same, side, up, down;
                    neighbours<L>(O, c, w, same, side, up, down);
                    if (bonds) apply_bonds<L>(bonds, c, w, same, side, up, down);
                    const uint32_t nw = metropolis_word_split<S>(P[w], same, side, up, down, 8u * (unsigned)w, sub,
                                                                 (unsigned)k, 2u * u + (unsigned)c, t4m1, t8m1,
                                                                 unit, key, gmask);
                    if (sub == 0) P[w] = nw;
                }
            } else if (active) {
                uint32_t* P = sp + c * Gm::WP;
                const uint32_t* O = sp + (1 - c) * Gm::WP;
                const unsigned c2 = 2u * u + (unsigned)c;
#pragma unroll 2
                for (int m = 0; m < WPT; m++) {
                    const int w = gl + m * G;
                    if constexpr (D == 3) {
                        uint32_t same, side, up, down, zup, zdn;
                        neighbours3<L>(O, c, w, same, side, up, down, zup, zdn);
                        P[w] = metropolis_word3(P[w], same, side, up, down, zup, zdn, 8u * (unsigned)w,
                                                (unsigned)k, c2, t4m1, t8m1, t12m1, unit, key);
                    } else {
                        uint32_t same, side, up, down;
                        neighbours<L>(O, c, w, same, side, up, down);
                        if (bonds) apply_bonds<L>(bonds, c, w, same, side, up, down);
                        P[w] = metropolis_word(P[w], same, side, up, down, 8u * (unsigned)w, (unsigned)k, c2,
                                               t4m1, t8m1, unit, key);
                    }
                }
            }
            Gr::sync();
            if constexpr (Gr::kCta) {
                if (pf && sw == 0 && c == 0 && threadIdx.x == 0 && pf->src) bulk_load(pf->dst, pf->src, pf->bytes, pf->mbar);
            }
        }
    }
    unsigned anti = 0, ups = 0;
    if (active) measure_bits<L, G, D>(sp, gl, anti, ups, bonds);
    anti = Gr::sum(anti, red);
    ups = Gr::sum(ups, red);
    if (active) {
        store_replica<L, G, D, kBytes>(r.pop[nxt], k, sp, gl);
        if (gl == 0) {
            const uint32_t f = r.fam[cur][p];
            record_replica(r, nxt, k, anti, ups, f);
            families += (k == 0 || r.fam[cur][r.parent[k - 1]] != f) ? 1u : 0u;
        }
    }
    Gr::sync();
}

// Initial spins of replica k (INIT stream: site g = c*N/2 + b, counter
// (0, g>>2, 0, k), spin up iff x < 2^31), measured and written to pop[0].
template <int L, int G, int D = 2, bool kBytes = false>
__device__ __forceinline__ void bits_group_init(const RunDev& r, long long k, bool active, uint32_t* sp, int gl,
                                                unsigned* red)
{
    using Gm = Lat<L, D>;
    using Gr = Group<G>;
    const PhiloxKey key{r.key[0], r.key[1]};
    if (active) {
        for (int i = gl; i < Gm::WORDS; i += G) {
            const int c = i / Gm::WP, w = i - c * Gm::WP;
            const unsigned c0 = (unsigned)(c * (Gm::N / 8) + 8 * w);
            uint32_t word = 0;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint4 x = philox10(make_uint4(0u, c0 + q, kTagInit, (unsigned)k), key);
                word |= ((x.x >> 31) ^ 1u) << (4 * q) | ((x.y >> 31) ^ 1u) << (4 * q + 1) |
                        ((x.z >> 31) ^ 1u) << (4 * q + 2) | ((x.w >> 31) ^ 1u) << (4 * q + 3);
            }
            sp[i] = word;
        }
    }
    Gr::sync();
    unsigned anti = 0, ups = 0;
    if (active) measure_bits<L, G, D>(sp, gl, anti, ups, r.bonds);
    anti = Gr::sum(anti, red);
    ups = Gr::sum(ups, red);
    if (active) {
        store_replica<L, G, D, kBytes>(r.pop[0], k, sp, gl);
        if (gl == 0) record_replica(r, 0, k, anti, ups, (uint32_t)k);
    }
    Gr::sync();
}

// ======================================================== bit-packed kernels
// Persistent: each group repeatedly takes the next replica of the run's
// work counter, so the tail of a step is at most one replica's work.
template <int L, int G, int D = 2, bool kBytes = false>
__global__ void __launch_bounds__(256) k_init_bits(const __grid_constant__ RunDev r)
{
    using Gm = Lat<L, D>;
    using Gr = Group<G>;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    uint32_t* sp = Gr::buffer(smem, Gm::WORDS);
    unsigned* red = smem + Gm::WORDS;  // CTA groups only
    const int gl = Gr::thread_in_group();
    const long long R0 = r.R;
    for (unsigned first = Gr::first_item();; first = Gr::grab(r.work, red + 32) + Gr::static_items()) {
        const unsigned base = Gr::kCta ? first : first - (threadIdx.x & 31) / G;
        if (base >= R0) break;
        bits_group_init<L, G, D, kBytes>(r, (long long)first, first < R0, sp, gl, red);
    }
}

// kCover: the grid holds every replica of the population (small runs):
// each group sweeps one fixed replica and never touches the counter.
// Otherwise the groups take replicas from the run's counter.
template <int L, int G, int D = 2, bool kBytes = false, bool kCover = false>
__global__ void __launch_bounds__(256) k_sweep_bits(const __grid_constant__ RunDev r, int step)
{
    pdl_wait();
    pdl_trigger();
    using Gm = Lat<L, D>;
    using Gr = Group<G>;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    uint32_t* sp = Gr::buffer(smem, Gm::WORDS);
    unsigned* red = smem + Gm::WORDS;  // CTA groups only
    const int gl = Gr::thread_in_group();
    const long long Ri = r.rec[step].R;
    unsigned families = 0;
    if constexpr (kCover) {
        const unsigned first = Gr::first_item();
        const unsigned base = Gr::kCta ? first : first - (threadIdx.x & 31) / G;
        if (base < Ri) bits_group_step<L, G, D, kBytes>(r, step, (long long)first, first < Ri, sp, gl, red, families);
    } else if constexpr (Gr::kCta && !kBytes && Gm::WORDS <= kPrefetchMaxWords) {
        static_assert(Gm::WORDS % 4 == 0, "bulk copies move multiples of 16 bytes");
        // One replica per CTA, two replica buffers: while the CTA sweeps
        // replica `cur` in buf[b], a bulk copy brings the next one's parent
        // into buf[b ^ 1] (shared memory: buf0, buf1, then the reduction words).
        __shared__ __align__(8) unsigned long long s_mbar[2];
        uint32_t* const buf0 = smem;
        uint32_t* const buf1 = smem + Gm::WORDS;
        unsigned* red2 = smem + 2 * Gm::WORDS;
        const int cur_pop = (step - 1) & 1;
        const unsigned bytes = Gm::WORDS * 4u;
        if (threadIdx.x == 0) {
            mbar_init(&s_mbar[0]);
            mbar_init(&s_mbar[1]);
        }
        unsigned cur = Gr::grab(r.work, red2 + 32);  // (synchronises: the barriers are initialised)
        if (threadIdx.x == 0 && cur < Ri)
            bulk_load(buf0, r.pop[cur_pop] + (size_t)r.parent[cur] * Gm::WORDS, bytes, &s_mbar[0]);
        // buffer b (0/1) alternates; each barrier's phase parity flips once
        // per use of its buffer, i.e. every second replica
        unsigned b = 0, phases = 0;  // bit i: parity to wait for on barrier i
        for (;;) {
            if (cur >= Ri) break;
            const unsigned nxt = Gr::grab(r.work, red2 + 32);
            Prefetch pf{nullptr, b ? buf0 : buf1, &s_mbar[b ^ 1u], bytes};
            if (threadIdx.x == 0 && nxt < Ri) pf.src = r.pop[cur_pop] + (size_t)r.parent[nxt] * Gm::WORDS;
            const unsigned par = (phases >> b) & 1u;
            if (!mbar_wait(&s_mbar[b], par)) {
                // the copy did not land in time: report it and leave no copy
                // in flight (a second bounded wait), then stop
                if (threadIdx.x == 0) *r.status = kStatusTimeout;
                mbar_wait(&s_mbar[b], par);
                break;
            }
            phases ^= 1u << b;
            bits_group_step<L, G, D, kBytes>(r, step, (long long)cur, true, b ? buf1 : buf0, gl, red2, families,
                                              &pf);
            cur = nxt;
            b ^= 1u;
        }
    } else {
        for (;;) {
            const unsigned first = Gr::grab(r.work, red + 32);
            const unsigned base = Gr::kCta ? first : first - (threadIdx.x & 31) / G;
            if (base >= Ri) break;
            bits_group_step<L, G, D, kBytes>(r, step, (long long)first, first < Ri, sp, gl, red, families);
        }
    }
    families = group_sum<32>(families);
    if ((threadIdx.x & 31) == 0 && families) atomicAdd(&r.rec[step].fam, (unsigned long long)families);
}

// ======================================================== byte-spin kernels
// Same RNG streams and update rule with one byte per spin (any even L >= 4).

// next work item of a warp from the run's counter (lane 0 takes n items)
__device__ __forceinline__ unsigned warp_grab(unsigned* work, unsigned n)
{
    unsigned v = 0;
    if ((threadIdx.x & 31) == 0) v = atomicAdd(work, n);
    return __shfl_sync(0xffffffffu, v, 0);
}
// Thread handles the sites of one Philox block (4 consecutive b) at a time.
__device__ __forceinline__ int nb_index_side(int b, int c, int L, int half)
{
    const int y = b / half, h = b - y * half;
    const int xodd = (c + y) & 1;
    const int h2 = xodd ? (h + 1 == half ? 0 : h + 1) : (h == 0 ? half - 1 : h - 1);
    return y * half + h2;
}

// Row y = b / half of in-plane index b without a division: with
// m = ceil(2^32 / half), floor(b m / 2^32) = floor(b / half) exactly for
// half <= 512 and b < 2^22 (the rounding excess b (m half - 2^32) / 2^32
// stays below 1/half).
__device__ __forceinline__ unsigned row_magic(int half)
{
    return (unsigned)(((1ull << 32) + (unsigned long long)half - 1ull) / (unsigned long long)half);
}

// the four neighbours (same index, side, up, down) in the other plane O of
// site b of plane c, with y = b / half given by the reciprocal m
__device__ __forceinline__ void byte_neighbours(const uint8_t* __restrict__ O, int b, int c, int L, int half,
                                                unsigned m, int& n0, int& n1, int& n2, int& n3)
{
    const int y = (int)__umulhi((unsigned)b, m), h = b - y * half;
    const int h2 = ((c + y) & 1) ? (h + 1 == half ? 0 : h + 1) : (h == 0 ? half - 1 : h - 1);
    n0 = O[b];
    n1 = O[y * half + h2];
    n2 = O[(y == 0 ? L - 1 : y - 1) * half + h];
    n3 = O[(y == L - 1 ? 0 : y + 1) * half + h];
}

// bond byte (1: J < 0) of direction dir for site b of plane c, or 0
__device__ __forceinline__ int bond8(const uint8_t* __restrict__ bonds8, int dir, int c, int NP, int b)
{
    return bonds8 ? (int)__ldg(bonds8 + ((size_t)(dir * 2 + c) * NP + b)) : 0;
}

template <int G>
__device__ __forceinline__ void measure_bytes(const uint8_t* sp, int L, int gl, unsigned& anti, unsigned& ups,
                                              const uint8_t* __restrict__ bonds8)
{
    const int N = L * L, half = L / 2, NP = N / 2;
    const uint8_t* o = sp + NP;
    anti = 0;
    ups = 0;
    for (int b = gl; b < NP; b += G) {
        const int s = sp[b];
        const int y = b / half, h = b - y * half;
        const int up = ((y == 0 ? L - 1 : y - 1)) * half + h;
        const int dn = ((y == L - 1 ? 0 : y + 1)) * half + h;
        anti += (unsigned)(((o[b] ^ bond8(bonds8, 0, 0, NP, b)) != s) +
                           ((o[nb_index_side(b, 0, L, half)] ^ bond8(bonds8, 1, 0, NP, b)) != s) +
                           ((o[up] ^ bond8(bonds8, 2, 0, NP, b)) != s) + ((o[dn] ^ bond8(bonds8, 3, 0, NP, b)) != s));
        ups += (unsigned)(s + o[b]);
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_init_bytes(const __grid_constant__ RunDev r)
{
    constexpr int RPW = 32 / G;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / G, gl = lane % G;
    uint8_t* sp = reinterpret_cast<uint8_t*>(smem + (warp * RPW + g) * r.words);
    const PhiloxKey key{r.key[0], r.key[1]};
    const long long R0 = r.R;
    const int N = r.N, NP = N / 2;
    for (;;) {
        const unsigned base = warp_grab(r.work, (unsigned)RPW);
        if (base >= R0) break;
        const long long k = (long long)base + g;
        const bool active = k < R0;
        if (active) {
            for (int gq = gl; gq < (N + 3) / 4; gq += G) {
                const uint4 x = philox10(make_uint4(0u, (unsigned)gq, kTagInit, (unsigned)k), key);
                const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int l = 0; l < 4; l++) {
                    const int gi = 4 * gq + l;  // = c*N/2 + b
                    if (gi < N) sp[gi] = (uint8_t)(xs[l] < 0x80000000u);
                }
            }
        }
        (void)NP;
        __syncwarp();
        unsigned anti = 0, ups = 0;
        if (active) measure_bytes<G>(sp, r.L, gl, anti, ups, r.bonds8);
        anti = group_sum<G>(anti);
        ups = group_sum<G>(ups);
        if (active) {
            uint32_t* dst = r.pop[0] + (size_t)k * r.words;
            const uint32_t* s32 = reinterpret_cast<const uint32_t*>(sp);
            for (int i = gl; i < r.words; i += G) dst[i] = s32[i];
            if (gl == 0) record_replica(r, 0, k, anti, ups, (uint32_t)k);
        }
        __syncwarp();
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_sweep_bytes(const __grid_constant__ RunDev r, int step)
{
    pdl_wait();
    pdl_trigger();
    constexpr int RPW = 32 / G;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / G, gl = lane % G;
    uint8_t* sp = reinterpret_cast<uint8_t*>(smem + (warp * RPW + g) * r.words);
    const int cur = (step - 1) & 1, nxt = step & 1;
    const long long Ri = r.rec[step].R;
    const uint32_t t4m1 = r.thr[2 * step], t8m1 = r.thr[2 * step + 1];
    const PhiloxKey key{r.key[0], r.key[1]};
    const unsigned u0 = (unsigned)(step - 1) * (unsigned)r.theta;
    const int L = r.L, half = r.half, NP = r.N / 2, QP = (NP + 3) / 4;
    const unsigned hm = row_magic(half);
    unsigned families = 0;
    for (;;) {
        const unsigned base = warp_grab(r.work, (unsigned)RPW);
        if (base >= Ri) break;
        const long long k = (long long)base + g;
        const bool active = k < Ri;
        uint32_t p = 0;
        if (active) {
            p = r.parent[k];
            const uint32_t* src = r.pop[cur] + (size_t)p * r.words;
            uint32_t* s32 = reinterpret_cast<uint32_t*>(sp);
            for (int i = gl; i < r.words; i += G) s32[i] = src[i];
        }
        __syncwarp();
        for (int sw = 0; sw < r.theta; sw++) {
            const unsigned u = u0 + (unsigned)sw;
            for (int c = 0; c < 2; c++) {
                if (active) {
                    uint8_t* __restrict__ P = sp + c * NP;
                    const uint8_t* __restrict__ O = sp + (1 - c) * NP;
                    // independent Philox blocks: unrolled so that their chains overlap
#pragma unroll 4
                    for (int q = gl; q < QP; q += G) {
                        const uint4 x = philox10(make_uint4(2u * u + (unsigned)c, (unsigned)q, kTagSweep, (unsigned)k),
                                                 key);
                        const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int l = 0; l < 4; l++) {
                            const int b = 4 * q + l;
                            if (b < NP) {
                                const int s = P[b];
                                int nb0, nb1, nb2, nb3;
                                byte_neighbours(O, b, c, L, half, hm, nb0, nb1, nb2, nb3);
                                const uint8_t* B8 = r.bonds8;
                                const int n = ((nb0 ^ bond8(B8, 0, c, NP, b)) == s) +
                                              ((nb1 ^ bond8(B8, 1, c, NP, b)) == s) +
                                              ((nb2 ^ bond8(B8, 2, c, NP, b)) == s) +
                                              ((nb3 ^ bond8(B8, 3, c, NP, b)) == s);
                                bool flip = n <= 2;
                                if (n == 3) flip = xs[l] <= t4m1;
                                if (n == 4) flip = xs[l] <= t8m1;
                                if (flip) P[b] = (uint8_t)(s ^ 1);
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
        unsigned anti = 0, ups = 0;
        if (active) measure_bytes<G>(sp, L, gl, anti, ups, r.bonds8);
        anti = group_sum<G>(anti);
        ups = group_sum<G>(ups);
        if (active) {
            uint32_t* dst = r.pop[nxt] + (size_t)k * r.words;
            const uint32_t* s32 = reinterpret_cast<const uint32_t*>(sp);
            for (int i = gl; i < r.words; i += G) dst[i] = s32[i];
            if (gl == 0) {
                const uint32_t f = r.fam[cur][p];
                record_replica(r, nxt, k, anti, ups, f);
                families += (k == 0 || r.fam[cur][r.parent[k - 1]] != f) ? 1u : 0u;
            }
        }
        __syncwarp();
    }
    families = group_sum<32>(families);
    if (lane == 0 && families) atomicAdd(&r.rec[step].fam, (unsigned long long)families);
}



// ======================================================== q-state Potts
// Byte states 0..q-1 in the byte layout (plane 0 then plane 1); the update
// of the oracle's Potts mode: the POTTS block (2u + c, b>>1, 6, k) gives
// the proposal word out[2(b&1)] and the acceptance word out[2(b&1) + 1].
// Proposal s' = (s + 1 + floor(w0 (q-1) / 2^32)) mod q; with n(t) the
// neighbours in state t, dE = n(s) - n(s'); accepted if dE <= 0, else iff
// w1 <= T_dE - 1.
__device__ __forceinline__ int potts_state(unsigned x, int q)
{
    return (int)(((unsigned long long)x * (unsigned long long)q) >> 32);
}

// satisfied bonds (each bond once: the four neighbours of every plane-0 site)
// and the number of sites in each state
template <int G>
__device__ __forceinline__ void measure_potts(const uint8_t* sp, int L, int q, int gl, unsigned& eq,
                                              unsigned cnt[8])
{
    const int N = L * L, half = L / 2, NP = N / 2;
    const uint8_t* o = sp + NP;
    eq = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) cnt[t] = 0;
    for (int b = gl; b < NP; b += G) {
        const int s = sp[b];
        const int y = b / half, h = b - y * half;
        const int up = ((y == 0 ? L - 1 : y - 1)) * half + h;
        const int dn = ((y == L - 1 ? 0 : y + 1)) * half + h;
        eq += (unsigned)((o[b] == s) + (o[nb_index_side(b, 0, L, half)] == s) + (o[up] == s) + (o[dn] == s));
#pragma unroll
        for (int t = 0; t < 8; t++) cnt[t] += (unsigned)(s == t) + (unsigned)(o[b] == t);
    }
    (void)q;
}

// group totals of a Potts measurement, then the record (E + 2N = 2N - eq,
// majority size)
template <int G>
__device__ __forceinline__ void record_potts(const RunDev& r, int nxt, long long k, bool active, int gl,
                                             unsigned eq, unsigned cnt[8], uint32_t family)
{
    eq = group_sum<G>(eq);
    unsigned mx = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) {
        const unsigned c = group_sum<G>(cnt[t]);
        if (t < r.potts_q) mx = max(mx, c);
    }
    if (active && gl == 0) record_levels(r, nxt, k, 2 * r.N - (int)eq, (int)mx, (long long)mx, family);
}

template <int G>
__global__ void __launch_bounds__(256) k_init_potts(const __grid_constant__ RunDev r)
{
    constexpr int RPW = 32 / G;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / G, gl = lane % G;
    uint8_t* sp = reinterpret_cast<uint8_t*>(smem + (warp * RPW + g) * r.words);
    const PhiloxKey key{r.key[0], r.key[1]};
    const long long R0 = r.R;
    const int N = r.N, q = r.potts_q;
    for (;;) {
        const unsigned base = warp_grab(r.work, (unsigned)RPW);
        if (base >= R0) break;
        const long long k = (long long)base + g;
        const bool active = k < R0;
        if (active) {
            for (int gq = gl; gq < (N + 3) / 4; gq += G) {
                const uint4 x = philox10(make_uint4(0u, (unsigned)gq, kTagInit, (unsigned)k), key);
                const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int l = 0; l < 4; l++) {
                    const int gi = 4 * gq + l;  // = c*N/2 + b
                    if (gi < N) sp[gi] = (uint8_t)potts_state(xs[l], q);
                }
            }
        }
        __syncwarp();
        unsigned eq = 0, cnt[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        if (active) measure_potts<G>(sp, r.L, q, gl, eq, cnt);
        if (active) {
            uint32_t* dst = r.pop[0] + (size_t)k * r.words;
            const uint32_t* s32 = reinterpret_cast<const uint32_t*>(sp);
            for (int i = gl; i < r.words; i += G) dst[i] = s32[i];
        }
        record_potts<G>(r, 0, k, active, gl, eq, cnt, (uint32_t)k);
        __syncwarp();
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_sweep_potts(const __grid_constant__ RunDev r, int step)
{
    pdl_wait();
    pdl_trigger();
    constexpr int RPW = 32 / G;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / G, gl = lane % G;
    uint8_t* sp = reinterpret_cast<uint8_t*>(smem + (warp * RPW + g) * r.words);
    const int cur = (step - 1) & 1, nxt = step & 1;
    const long long Ri = r.rec[step].R;
    const uint32_t* T = r.thrp + 4 * step;
    const uint32_t t1 = T[0], t2 = T[1], t3 = T[2], t4 = T[3];
    const PhiloxKey key{r.key[0], r.key[1]};
    const unsigned u0 = (unsigned)(step - 1) * (unsigned)r.theta;
    const int L = r.L, half = r.half, NP = r.N / 2, QP = NP / 2, q = r.potts_q;
    const unsigned hm = row_magic(half);
    unsigned families = 0;
    for (;;) {
        const unsigned base = warp_grab(r.work, (unsigned)RPW);
        if (base >= Ri) break;
        const long long k = (long long)base + g;
        const bool active = k < Ri;
        uint32_t p = 0;
        if (active) {
            p = r.parent[k];
            const uint32_t* src = r.pop[cur] + (size_t)p * r.words;
            uint32_t* s32 = reinterpret_cast<uint32_t*>(sp);
            for (int i = gl; i < r.words; i += G) s32[i] = src[i];
        }
        __syncwarp();
        for (int sw = 0; sw < r.theta; sw++) {
            const unsigned u = u0 + (unsigned)sw;
            for (int c = 0; c < 2; c++) {
                if (active) {
                    uint8_t* __restrict__ P = sp + c * NP;
                    const uint8_t* __restrict__ O = sp + (1 - c) * NP;
                    // independent Philox blocks: unrolled so that their chains overlap
#pragma unroll 4
                    for (int pb = gl; pb < QP; pb += G) {
                        const uint4 x =
                            philox10(make_uint4(2u * u + (unsigned)c, (unsigned)pb, kTagPotts, (unsigned)k), key);
#pragma unroll
                        for (int l = 0; l < 2; l++) {
                            const int b = 2 * pb + l;
                            const unsigned w0 = l ? x.z : x.x, w1 = l ? x.w : x.y;
                            const int s = P[b];
                            int sn = s + 1 + potts_state(w0, q - 1);
                            if (sn >= q) sn -= q;
                            int nb0, nb1, nb2, nb3;
                            byte_neighbours(O, b, c, L, half, hm, nb0, nb1, nb2, nb3);
                            const int ns = (nb0 == s) + (nb1 == s) + (nb2 == s) + (nb3 == s);
                            const int nn = (nb0 == sn) + (nb1 == sn) + (nb2 == sn) + (nb3 == sn);
                            const int dE = ns - nn;
                            bool acc = dE <= 0;
                            if (dE == 1) acc = w1 <= t1;
                            if (dE == 2) acc = w1 <= t2;
                            if (dE == 3) acc = w1 <= t3;
                            if (dE == 4) acc = w1 <= t4;
                            if (acc) P[b] = (uint8_t)sn;
                        }
                    }
                }
                __syncwarp();
            }
        }
        unsigned eq = 0, cnt[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        if (active) measure_potts<G>(sp, L, q, gl, eq, cnt);
        uint32_t f = 0;
        if (active) {
            uint32_t* dst = r.pop[nxt] + (size_t)k * r.words;
            const uint32_t* s32 = reinterpret_cast<const uint32_t*>(sp);
            for (int i = gl; i < r.words; i += G) dst[i] = s32[i];
            f = r.fam[cur][p];
            if (gl == 0) families += (k == 0 || r.fam[cur][r.parent[k - 1]] != f) ? 1u : 0u;
        }
        record_potts<G>(r, nxt, k, active, gl, eq, cnt, f);
        __syncwarp();
    }
    families = group_sum<32>(families);
    if (lane == 0 && families) atomicAdd(&r.rec[step].fam, (unsigned long long)families);
}

// ======================================================== replica-parallel
// The paper's generic fallback (Sec. 3 "Spin updates"): one thread per
// replica walks its lattice site by site; byte spins stored with the replica
// index fastest (site g of replica k at byte g * cap + k, g = c*N/2 + b), so
// the threads of a warp touch consecutive bytes. Same random-number contract
// as the other single-spin formats (one Philox word per attempt).
__device__ __forceinline__ void rp_measure(const uint8_t* col, size_t cap, int L, unsigned& anti, unsigned& ups)
{
    const int half = L / 2, NP = L * L / 2;
    anti = 0;
    ups = 0;
    for (int b = 0; b < NP; b++) {
        const int s = col[(size_t)b * cap];
        const int y = b / half, h = b - y * half;
        const int up = (y == 0 ? L - 1 : y - 1) * half + h;
        const int dn = (y == L - 1 ? 0 : y + 1) * half + h;
        const uint8_t* o = col + (size_t)NP * cap;
        anti += (unsigned)((o[(size_t)b * cap] != s) + (o[(size_t)nb_index_side(b, 0, L, half) * cap] != s) +
                           (o[(size_t)up * cap] != s) + (o[(size_t)dn * cap] != s));
        ups += (unsigned)(s + o[(size_t)b * cap]);
    }
}

__global__ void __launch_bounds__(256) k_init_rp(const __grid_constant__ RunDev r)
{
    if (*r.status) return;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= r.R) return;
    const size_t cap = (size_t)r.cap;
    uint8_t* col = reinterpret_cast<uint8_t*>(r.pop[0]) + k;
    const PhiloxKey key{r.key[0], r.key[1]};
    const int N = r.N;
    for (int gq = 0; gq < (N + 3) / 4; gq++) {
        const uint4 x = philox10(make_uint4(0u, (unsigned)gq, kTagInit, (unsigned)k), key);
        const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int l = 0; l < 4; l++) {
            const int g = 4 * gq + l;
            if (g < N) col[(size_t)g * cap] = (uint8_t)(xs[l] < 0x80000000u);
        }
    }
    unsigned anti, ups;
    rp_measure(col, cap, r.L, anti, ups);
    record_replica(r, 0, k, anti, ups, (uint32_t)k);
}

__global__ void __launch_bounds__(256) k_sweep_rp(const __grid_constant__ RunDev r, int step)
{
    pdl_wait();
    pdl_trigger();
    if (*r.status) return;
    const long long Ri = r.rec[step].R;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned families = 0;
    if (k < Ri) {
        const int cur = (step - 1) & 1, nxt = step & 1;
        const size_t cap = (size_t)r.cap;
        const int L = r.L, N = r.N, half = L / 2, NP = N / 2, QP = (NP + 3) / 4;
        const uint32_t p = r.parent[k];
        const uint8_t* src = reinterpret_cast<const uint8_t*>(r.pop[cur]) + p;
        uint8_t* col = reinterpret_cast<uint8_t*>(r.pop[nxt]) + k;
        for (int g = 0; g < N; g++) col[(size_t)g * cap] = src[(size_t)g * cap];
        const uint32_t t4m1 = r.thr[2 * step], t8m1 = r.thr[2 * step + 1];
        const PhiloxKey key{r.key[0], r.key[1]};
        const unsigned u0 = (unsigned)(step - 1) * (unsigned)r.theta;
        for (int sw = 0; sw < r.theta; sw++) {
            const unsigned u = u0 + (unsigned)sw;
            for (int c = 0; c < 2; c++) {
                uint8_t* P = col + (size_t)c * NP * cap;
                const uint8_t* O = col + (size_t)(1 - c) * NP * cap;
                for (int q = 0; q < QP; q++) {
                    const uint4 x = philox10(make_uint4(2u * u + (unsigned)c, (unsigned)q, kTagSweep, (unsigned)k), key);
                    const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int l = 0; l < 4; l++) {
                        const int b = 4 * q + l;
                        if (b < NP) {
                            const int s = P[(size_t)b * cap];
                            const int y = b / half, h = b - y * half;
                            const int up = (y == 0 ? L - 1 : y - 1) * half + h;
                            const int dn = (y == L - 1 ? 0 : y + 1) * half + h;
                            const int n = (O[(size_t)b * cap] == s) + (O[(size_t)nb_index_side(b, c, L, half) * cap] == s) +
                                          (O[(size_t)up * cap] == s) + (O[(size_t)dn * cap] == s);
                            bool flip = n <= 2;
                            if (n == 3) flip = xs[l] <= t4m1;
                            if (n == 4) flip = xs[l] <= t8m1;
                            if (flip) P[(size_t)b * cap] = (uint8_t)(s ^ 1);
                        }
                    }
                }
            }
        }
        unsigned anti, ups;
        rp_measure(col, cap, L, anti, ups);
        const uint32_t f = r.fam[cur][p];
        record_replica(r, nxt, k, anti, ups, f);
        families = (k == 0 || r.fam[cur][r.parent[k - 1]] != f) ? 1u : 0u;
    }
    families = group_sum<32>(families);
    if ((threadIdx.x & 31) == 0 && families) atomicAdd(&r.rec[step].fam, (unsigned long long)families);
}

// ======================================================== multi-spin coding
// Asynchronous multi-spin coding (Sec. 4): replica k is bit k%32 of its
// group's words, one word per site (plane 0 sites then plane 1, site b of a
// plane at word b). A warp owns one group; lane j is replica 32G + j. The 32
// replicas of a site are updated together by bit-sliced neighbour counts;
// their random numbers come from the linear congruential generator
// r <- A r + C (mod 2^32), A = 1664525, C = 1013904223, seeded with the
// Philox word at counter (2u + c, b>>2, 5, G), lane b&3: replica bit j uses
// the (j+1)-th output, computed directly as a_{j+1} seed + c_{j+1}.
constexpr unsigned kLcgA = 1664525u, kLcgC = 1013904223u;
constexpr unsigned kTagMsc = 5u;

struct LcgJump {
    unsigned a[33], c[33];  // r_n = a[n] r_0 + c[n]
    constexpr LcgJump() : a(), c()
    {
        a[0] = 1u;
        c[0] = 0u;
        for (int n = 1; n <= 32; n++) {
            a[n] = kLcgA * a[n - 1];
            c[n] = kLcgA * c[n - 1] + kLcgC;
        }
    }
};
__constant__ LcgJump c_lcg = LcgJump();

template <int L>
struct MscGeo {
    static constexpr int N = L * L, HALF = L / 2, NP = N / 2, QP = (NP + 3) / 4;
};

// index of the row neighbour (other plane) of site b of plane c
template <int L>
__device__ __forceinline__ int msc_side(int b, int c)
{
    constexpr int HALF = L / 2;
    const int y = b / HALF, h = b - y * HALF;
    const int h2 = ((c + y) & 1) ? (h + 1 == HALF ? 0 : h + 1) : (h == 0 ? HALF - 1 : h - 1);
    return y * HALF + h2;
}

// anti-parallel bonds and up spins of replica bit `lane` of the group in smem
template <int L>
__device__ __forceinline__ void msc_measure(const uint32_t* sp, int lane, unsigned& anti, unsigned& ups)
{
    using G = MscGeo<L>;
    const uint32_t* o = sp + G::NP;
    anti = 0;
    ups = 0;
    for (int b = 0; b < G::NP; b++) {
        const uint32_t s = sp[b];
        const int y = b / G::HALF, h = b - y * G::HALF;
        const int up = (y == 0 ? L - 1 : y - 1) * G::HALF + h;
        const int dn = (y == L - 1 ? 0 : y + 1) * G::HALF + h;
        const uint32_t x = ((s ^ o[b]) >> lane & 1u) + ((s ^ o[msc_side<L>(b, 0)]) >> lane & 1u) +
                           ((s ^ o[up]) >> lane & 1u) + ((s ^ o[dn]) >> lane & 1u);
        anti += x;
        ups += (s >> lane & 1u) + (o[b] >> lane & 1u);
    }
}

// accept bits of replicas J .. 31 against both thresholds: LCG value j+1 of
// the site's seed
template <int J>
__device__ __forceinline__ void msc_accept(uint32_t& acc4, uint32_t& acc8, unsigned seed, uint32_t t4m1,
                                           uint32_t t8m1, uint32_t unit)
{
    if constexpr (J < 32) {
        const unsigned xj = c_lcg.a[J + 1] * seed + c_lcg.c[J + 1];
        acc4 = accept_bit<J>(acc4, xj, t4m1, unit);
        acc8 = accept_bit<J>(acc8, xj, t8m1, unit);
        msc_accept<J + 1>(acc4, acc8, seed, t4m1, t8m1, unit);
    }
}

// the 32 replicas' Metropolis update of site word s with neighbour words
__device__ __forceinline__ uint32_t msc_update(uint32_t s, uint32_t n1, uint32_t n2, uint32_t n3, uint32_t n4,
                                               unsigned seed, uint32_t t4m1, uint32_t t8m1, uint32_t unit)
{
    const uint32_t d1 = s ^ n1, d2 = s ^ n2, d3 = s ^ n3, d4 = s ^ n4;
    const uint32_t a = d1 ^ d2, bb = d1 & d2, cc = d3 ^ d4, e = d3 & d4;
    const uint32_t ge2 = bb | e | (a & cc);
    const uint32_t eq0 = ~(d1 | d2 | d3 | d4);
    uint32_t acc4 = 0, acc8 = 0;
    msc_accept<0>(acc4, acc8, seed, t4m1, t8m1, unit);
    return s ^ (ge2 | (acc4 & ~eq0) | (acc8 & eq0));
}

// Warps per 32-replica group: enough that each thread updates one to four
// Philox blocks of sites per colour phase (a group is one CTA).
template <int L>
__host__ __device__ constexpr int msc_warps()
{
    constexpr int qp = MscGeo<L>::QP;
    return qp >= 32 * 16 ? 16 : (qp >= 32 * 8 ? 8 : (qp >= 32 * 4 ? 4 : (qp >= 64 ? 2 : 1)));
}

// Persistent CTAs, one 32-replica group at a time: thread 0 takes the next
// group; warp w handles sites w, w + W, ... when gathering and measuring
// (lane j = replica bit j); all threads share the colour phases.
template <int L>
__device__ __forceinline__ unsigned msc_grab(unsigned* work, unsigned* bcast)
{
    __syncthreads();
    if (threadIdx.x == 0) *bcast = atomicAdd(work, 1u);
    __syncthreads();
    return *bcast;
}

// anti-parallel bonds and up spins of replica bit `lane` over this warp's sites,
// then summed over the CTA's warps (every lane of warp 0 gets its replica's totals)
template <int L, int W>
__device__ __forceinline__ void msc_measure_cta(const uint32_t* sp, unsigned* red, unsigned& anti, unsigned& ups)
{
    using G = MscGeo<L>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* o = sp + G::NP;
    unsigned a = 0, u = 0;
    for (int b = warp; b < G::NP; b += W) {
        const uint32_t s = sp[b];
        const int y = b / G::HALF, h = b - y * G::HALF;
        const int up = (y == 0 ? L - 1 : y - 1) * G::HALF + h;
        const int dn = (y == L - 1 ? 0 : y + 1) * G::HALF + h;
        a += ((s ^ o[b]) >> lane & 1u) + ((s ^ o[msc_side<L>(b, 0)]) >> lane & 1u) + ((s ^ o[up]) >> lane & 1u) +
             ((s ^ o[dn]) >> lane & 1u);
        u += (s >> lane & 1u) + (o[b] >> lane & 1u);
    }
    __syncthreads();
    red[warp * 32 + lane] = a;
    red[(W + warp) * 32 + lane] = u;
    __syncthreads();
    anti = 0;
    ups = 0;
    if (warp == 0) {
#pragma unroll
        for (int w = 0; w < W; w++) {
            anti += red[w * 32 + lane];
            ups += red[(W + w) * 32 + lane];
        }
    }
}

template <int L>
__global__ void __launch_bounds__(32 * msc_warps<L>()) k_init_msc(const __grid_constant__ RunDev r)
{
    using Gm = MscGeo<L>;
    constexpr int W = msc_warps<L>(), N = Gm::N;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* sp = smem;
    unsigned* red = smem + N;
    const PhiloxKey key{r.key[0], r.key[1]};
    const long long R0 = r.R, groups = (R0 + 31) / 32;
    for (;;) {
        const unsigned G = msc_grab<L>(r.work, red + 2 * W * 32);
        if ((long long)G >= groups) break;
        const long long k = 32ll * G + lane;
        const bool valid = k < R0;
        // INIT stream of replica k: site g = c*N/2 + b, counter (0, g>>2, 0, k)
        for (int gq = warp; gq < (N + 3) / 4; gq += W) {
            const uint4 x = philox10(make_uint4(0u, (unsigned)gq, kTagInit, (unsigned)k), key);
            const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int l = 0; l < 4; l++) {
                const int g = 4 * gq + l;
                const uint32_t w = __ballot_sync(0xffffffffu, valid && xs[l] < 0x80000000u);
                if (g < N && lane == (g & 31)) sp[g] = w;
            }
        }
        __syncthreads();
        unsigned anti, ups;
        msc_measure_cta<L, W>(sp, red, anti, ups);
        uint32_t* dst = r.pop[0] + (size_t)G * N;
        for (int i = threadIdx.x; i < N; i += 32 * W) dst[i] = sp[i];
        if (warp == 0 && valid) record_replica(r, 0, k, anti, ups, (uint32_t)k);
    }
}

template <int L>
__global__ void __launch_bounds__(32 * msc_warps<L>()) k_sweep_msc(const __grid_constant__ RunDev r, int step)
{
    pdl_wait();
    pdl_trigger();
    using Gm = MscGeo<L>;
    constexpr int W = msc_warps<L>(), N = Gm::N, HALF = Gm::HALF, NP = Gm::NP, QP = Gm::QP;
    extern __shared__ uint32_t smem[];
    if (*r.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* sp = smem;
    unsigned* red = smem + N;
    const int cur = (step - 1) & 1, nxt = step & 1;
    const long long Ri = r.rec[step].R, groups = (Ri + 31) / 32;
    const uint32_t t4m1 = r.thr[2 * step], t8m1 = r.thr[2 * step + 1];
    const PhiloxKey key{r.key[0], r.key[1]};
    const unsigned u0 = (unsigned)(step - 1) * (unsigned)r.theta;
    const int theta = r.theta;
    unsigned families = 0;
    for (;;) {
        const unsigned G = msc_grab<L>(r.work, red + 2 * W * 32);
        if ((long long)G >= groups) break;
        const long long k = 32ll * G + lane;
        const bool valid = k < Ri;
        // gather: bit `lane` of every site word comes from this lane's parent
        const uint32_t p = valid ? r.parent[k] : 0u;
        const uint32_t* src = r.pop[cur] + (size_t)(p >> 5) * N;
        const unsigned pb = p & 31u;
        for (int g = warp; g < N; g += W) {
            const uint32_t w = __ballot_sync(0xffffffffu, valid && ((src[g] >> pb) & 1u));
            if (lane == (g & 31)) sp[g] = w;
        }
        __syncthreads();
        for (int sw = 0; sw < theta; sw++) {
            const unsigned u = u0 + (unsigned)sw;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                uint32_t* P = sp + c * NP;
                const uint32_t* O = sp + (1 - c) * NP;
                for (int q = threadIdx.x; q < QP; q += 32 * W) {
                    const uint4 x = philox10(make_uint4(2u * u + (unsigned)c, (unsigned)q, kTagMsc, G), key);
                    const unsigned seeds[4] = {x.x, x.y, x.z, x.w};
                    if constexpr (HALF % 4 == 0) {
                        // the 4 sites of a Philox block share one row
                        const int b0 = 4 * q, y = b0 / HALF, h0 = b0 - y * HALF;
                        const int rup = (y == 0 ? L - 1 : y - 1) * HALF, rdn = (y == L - 1 ? 0 : y + 1) * HALF;
                        const bool xodd = (c + y) & 1;
#pragma unroll
                        for (int l = 0; l < 4; l++) {
                            const int h = h0 + l, b = b0 + l;
                            const int h2 = xodd ? (h + 1 == HALF ? 0 : h + 1) : (h == 0 ? HALF - 1 : h - 1);
                            P[b] = msc_update(P[b], O[b], O[y * HALF + h2], O[rup + h], O[rdn + h], seeds[l], t4m1,
                                              t8m1, r.unit);
                        }
                    } else {
#pragma unroll
                        for (int l = 0; l < 4; l++) {
                            const int b = 4 * q + l;
                            if (b < NP) {
                                const int y = b / HALF, h = b - y * HALF;
                                const int up = (y == 0 ? L - 1 : y - 1) * HALF + h;
                                const int dn = (y == L - 1 ? 0 : y + 1) * HALF + h;
                                P[b] = msc_update(P[b], O[b], O[msc_side<L>(b, c)], O[up], O[dn], seeds[l], t4m1,
                                                  t8m1, r.unit);
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
        unsigned anti, ups;
        msc_measure_cta<L, W>(sp, red, anti, ups);
        uint32_t* dst = r.pop[nxt] + (size_t)G * N;
        for (int i = threadIdx.x; i < N; i += 32 * W) dst[i] = sp[i];
        if (warp == 0 && valid) {
            const uint32_t f = r.fam[cur][p];
            record_replica(r, nxt, k, anti, ups, f);
            families += (k == 0 || r.fam[cur][r.parent[k - 1]] != f) ? 1u : 0u;
        }
    }
    families = group_sum<32>(families);
    if (lane == 0 && families) atomicAdd(&r.rec[step].fam, (unsigned long long)families);
}

template <int L>
__host__ __device__ constexpr int msc_threads()
{
    return 32 * msc_warps<L>();
}

// L values with a multi-spin-coded kernel
#define PA_MSC_SIZES(X) X(4) X(6) X(8) X(10) X(12) X(16) X(20) X(24) X(32) X(48) X(64) X(96) X(128)

// ======================================================== resampling kernels
__device__ __forceinline__ int pad_pow2(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// S = pairwise tree over T[k] = H[k] t[k - kmin] (k in [kmin, kmax], 0
// elsewhere) padded to a power of two, then the copy tables over [kmin, kmax].
// Thread t sums the aligned block [t*chunk, (t+1)*chunk) with a carry stack
// (the block's subtree), then a shared-memory tree joins neighbours.
// kmin, kmax: occupied range of population i-1 (from its record, or handed
// over in shared memory by the same CTA); sF, sU: optional shared-memory
// copies of the copy tables over [kmin, kmax] (null: global only).
__device__ __forceinline__ void tables_body(const RunDev& r, int step, int kmin, int kmax, uint32_t* sF = nullptr,
                                            unsigned long long* sU = nullptr)
{
    __shared__ double s[kOneCta];
    const int t = threadIdx.x;
    const uint32_t* H = r.H[(step - 1) & 1];
    const double* tw = r.tw;
    const int P = pad_pow2(r.nlev);
    const int nthr = P < kOneCta ? P : kOneCta;
    const int chunk = P / nthr;
    double v = 0.0;
    if (t < nthr) {
        const int lo = t * chunk, hi = lo + chunk;  // [lo, hi)
        if (hi > kmin && lo <= kmax) {
            double stk[24];
            int top = 0;
            for (int e = 0; e < chunk; e++) {
                const int kk = lo + e;
                double x = (kk >= kmin && kk <= kmax) ? __dmul_rn((double)H[kk], tw[kk - kmin]) : 0.0;
                for (int m = e; m & 1; m >>= 1) x = __dadd_rn(stk[--top], x);
                stk[top++] = x;
            }
            v = stk[0];
        }
    }
    // The same pairwise tree over the nthr leaves, level by level: within a
    // warp the lane holding the left subtree adds its right neighbour's
    // (offsets 1, 2, 4, 8, 16), then warp 0 joins the warps' subtrees the
    // same way. Each sum is (left subtree) + (right subtree), as above.
    const int lane = t & 31, warp = t >> 5;
    const int wl = nthr < 32 ? nthr : 32;  // leaves per warp
    for (int off = 1; off < wl; off <<= 1) {
        const double y = __shfl_down_sync(0xffffffffu, v, off);
        if ((lane & (2 * off - 1)) == 0) v = __dadd_rn(v, y);
    }
    if (lane == 0 && t < nthr) s[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = nthr / wl;  // warp subtrees (power of two <= 32)
        double x = lane < nw ? s[lane] : 0.0;
        for (int off = 1; off < nw; off <<= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, off);
            if ((lane & (2 * off - 1)) == 0) x = __dadd_rn(x, y);
        }
        if (lane == 0) s[0] = x;
    }
    __syncthreads();
    const double S = s[0];
    const double Rd = (double)r.R;
    for (int kk = kmin + t; kk <= kmax; kk += kOneCta) {
        const double tau = __ddiv_rn(__dmul_rn(Rd, tw[kk - kmin]), S);
        const double F = floor(tau);
        const double frac = __dsub_rn(tau, F);
        const uint32_t f32 = (uint32_t)F;
        const unsigned long long u64 = (unsigned long long)ceil(__dmul_rn(frac, 4294967296.0));
        if (sF) {
            sF[kk - kmin] = f32;
            sU[kk - kmin] = u64;
        } else {
            r.F[kk] = f32;
            r.U[kk] = u64;
        }
    }
    uint32_t* Hn = r.H[step & 1];
    for (int i = t; i < 2 * r.nlev; i += kOneCta) Hn[i] = 0u;
    if (t == 0) {
        r.rec[step].S = S;
        r.rec[step].kmin_prev = kmin;
        r.rec[step].fam = 0ull;
        *r.work = 0u;
    }
}

__global__ void __launch_bounds__(kOneCta) k_tables(const __grid_constant__ RunDev r, int step)
{
    if (*r.status) return;
    tables_body(r, step, r.rec[step - 1].kmin, r.rec[step - 1].kmax);
}

__global__ void __launch_bounds__(kOneCta) k_tables_batch(const __grid_constant__ BatchDev b, int step)
{
    const RunDev& r = b.runs[blockIdx.x];
    if (*r.status || step > r.nsteps) return;
    tables_body(r, step, r.rec[step - 1].kmin, r.rec[step - 1].kmax);
}

// Copy numbers of the old population (Eq. resampling-factors): one Philox
// block serves 4 consecutive old slots j (RESAMPLE stream (i, j>>2, 2, 0)).
__device__ __forceinline__ long long n_old_of(const ResampleArgs& a)
{
    return a.n_old_dev ? *a.n_old_dev : a.n_old;
}

// The copy numbers, their tile prefix and the tile total are summed in 64
// bits: the tables may come from a caller (pa_resample), and 1024 slots with
// F near 2^32 would wrap a 32-bit total to a small R_i. A tile whose total
// exceeds the capacity sets the capacity status here, so the scan and the
// parent scatter (later launches, which return when the status is set) never
// see a wrapped total; the stored 32-bit values are exact whenever the
// status stays clear (every total <= cap < 2^31).
__device__ __forceinline__ void counts_body(const ResampleArgs& a, int tile)
{
    __shared__ unsigned long long wsum[kTileThreads / 32];
    const long long Rp = n_old_of(a);
    const long long tile0 = (long long)tile * kTile;
    if (tile0 >= Rp) return;
    const long long j0 = tile0 + 4 * threadIdx.x;
    unsigned long long c[4] = {0ull, 0ull, 0ull, 0ull};
    if (j0 < Rp) {
        const uint4 x = philox10(make_uint4(a.step, (unsigned)(j0 >> 2), kTagResample, 0u),
                                 PhiloxKey{a.key[0], a.key[1]});
        const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int l = 0; l < 4; l++) {
            const long long j = j0 + l;
            if (j < Rp) {
                const int lv = a.lev[j];
                c[l] = (unsigned long long)a.F[lv] + (((unsigned long long)xs[l] < a.U[lv]) ? 1ull : 0ull);
            }
        }
    }
    const unsigned long long tsum = c[0] + c[1] + c[2] + c[3];
    // block exclusive scan of tsum
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = tsum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned long long wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kTileThreads / 32; w++) {
        if (w < warp) wbase += wsum[w];
        tot += wsum[w];
    }
    if (tot > (unsigned long long)a.cap) {
        // R_i > cap for certain: leave cnt/loc/tile_sum alone (never read)
        if (threadIdx.x == 0) *a.status = kStatusCapacity;
        return;
    }
    unsigned long long run = wbase + incl - tsum;
#pragma unroll
    for (int l = 0; l < 4; l++) {
        const long long j = j0 + l;
        if (j < Rp) {
            a.cnt[j] = (uint32_t)c[l];
            a.loc[j] = (uint32_t)run;
        }
        run += c[l];
    }
    if (threadIdx.x == 0) a.tile_sum[tile] = (uint32_t)tot;
}

__global__ void __launch_bounds__(kTileThreads) k_counts(const __grid_constant__ ResampleArgs a)
{
    if (*a.status) return;
    counts_body(a, blockIdx.x);
}

// Exclusive scan of the tile totals; R_i and the capacity check.
__device__ __forceinline__ void scan_body(const ResampleArgs& a)
{
    __shared__ unsigned long long part[kOneCta];
    const int t = threadIdx.x;
    const long long Rp = n_old_of(a);
    const int ntiles = (int)((Rp + kTile - 1) / kTile);
    const int per = (ntiles + kOneCta - 1) / kOneCta;
    const int lo = t * per, hi = min(lo + per, ntiles);
    unsigned long long sum = 0;
    for (int i = lo; i < hi; i++) sum += a.tile_sum[i];
    part[t] = sum;
    __syncthreads();
    // inclusive Hillis-Steele scan over the 1024 partial sums
    for (int off = 1; off < kOneCta; off <<= 1) {
        const unsigned long long y = t >= off ? part[t - off] : 0ull;
        __syncthreads();
        part[t] += y;
        __syncthreads();
    }
    unsigned long long run = part[t] - sum;
    for (int i = lo; i < hi; i++) {
        a.tile_off[i] = (uint32_t)run;
        run += a.tile_sum[i];
    }
    if (t == 0) {
        const unsigned long long Ri = part[kOneCta - 1];
        *a.n_new = (long long)Ri;
        if (a.n_prev_out) *a.n_prev_out = Rp;
        if ((long long)Ri > a.cap) *a.status = kStatusCapacity;
        else if (Ri == 0) *a.status = kStatusExtinct;
        if (a.work) *a.work = 0u;
    }
}

__global__ void __launch_bounds__(kOneCta) k_scan(const __grid_constant__ ResampleArgs a)
{
    if (*a.status) return;
    scan_body(a);
}

// parent[o_j + c] = j for c < r_j: new slots keep the order of old slots.
__device__ __forceinline__ void parent_body(const ResampleArgs& a, int tile)
{
    const long long Rp = n_old_of(a);
    const long long j = (long long)tile * kTile + threadIdx.x;
    if (j >= Rp) return;
    const uint32_t n = a.cnt[j];
    const uint32_t o = a.tile_off[tile] + a.loc[j];
    for (uint32_t c = 0; c < n; c++) a.parent[o + c] = (uint32_t)j;
}

__global__ void __launch_bounds__(kTile) k_parent(const __grid_constant__ ResampleArgs a)
{
    if (*a.status) return;
    parent_body(a, blockIdx.x);
}

// Resampling arguments of step `step` of a run (its records hold R_{i-1}).
__host__ __device__ __forceinline__ ResampleArgs resample_args(const RunDev& h, int step)
{
    ResampleArgs a{};
    a.n_old_dev = &h.rec[step - 1].R;
    a.n_old = 0;
    a.lev = h.elev[(step - 1) & 1];
    a.F = h.F;
    a.U = h.U;
    a.key = h.key;
    a.step = (unsigned)step;
    a.cnt = h.cnt;
    a.loc = h.loc;
    a.tile_sum = h.tile_sum;
    a.tile_off = h.tile_off;
    a.parent = h.parent;
    a.cap = h.cap;
    a.n_new = &h.rec[step].R;
    a.n_prev_out = &h.rec[step].R_prev;
    a.status = h.status;
    a.work = h.work;
    return a;
}

__global__ void __launch_bounds__(kTileThreads) k_counts_batch(const __grid_constant__ BatchDev b, int step)
{
    const int run = b.tile_run[blockIdx.x];
    const RunDev& r = b.runs[run];
    if (*r.status || step > r.nsteps) return;
    counts_body(resample_args(r, step), blockIdx.x - b.tile_first[run]);
}

__global__ void __launch_bounds__(kOneCta) k_scan_batch(const __grid_constant__ BatchDev b, int step)
{
    const RunDev& r = b.runs[blockIdx.x];
    if (*r.status || step > r.nsteps) return;
    scan_body(resample_args(r, step));
}

__global__ void __launch_bounds__(kTile) k_parent_batch(const __grid_constant__ BatchDev b, int step)
{
    const int run = b.tile_run[blockIdx.x];
    const RunDev& r = b.runs[run];
    if (*r.status || step > r.nsteps) return;
    parent_body(resample_args(r, step), blockIdx.x - b.tile_first[run]);
}

// ======================================================== statistics
struct I128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ I128 to_i128(__int128 v)
{
    return I128{(unsigned long long)v, (unsigned long long)((unsigned __int128)v >> 64)};
}
__device__ __forceinline__ __int128 from_i128(I128 v)
{
    return (__int128)(((unsigned __int128)v.hi << 64) | v.lo);
}
__device__ __forceinline__ __int128 warp_sum128(__int128 v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        I128 a = to_i128(v);
        I128 b{__shfl_xor_sync(0xffffffffu, a.lo, off), __shfl_xor_sync(0xffffffffu, a.hi, off)};
        v += from_i128(b);
    }
    return v;
}

// Integer moments of population i from its histograms (exact: every sum is
// an integer, so no order matters), occupied range, running sum for MHR.
// range (optional): shared-memory pair that receives (kmin, kmax) for the
// rest of the CTA (valid after the next __syncthreads)
__device__ __forceinline__ void stats_body(const RunDev& r, int step, int* range = nullptr)
{
    __shared__ __int128 ws[5][kOneCta / 32];
    __shared__ int wmin[kOneCta / 32], wmax[kOneCta / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int N = r.N, NL = r.nlev;
    const uint32_t* HE = r.H[step & 1];
    const uint32_t* HM = HE + NL;
    __int128 sE = 0, sE2 = 0, sAM = 0, sM2 = 0, sM4 = 0;
    int kmin = 0x7fffffff, kmax = -1;
    uint32_t* rec_hist = nullptr;
    if (r.record_hist && r.hist_rec && step < r.hist_steps) rec_hist = r.hist_rec + (size_t)step * 2 * NL;
    for (int k = t; k < NL; k += kOneCta) {
        const uint32_t h = HE[k];
        const uint32_t hm = HM[k];
        if (h) {
            kmin = min(kmin, k);
            kmax = max(kmax, k);
            const long long E = (long long)r.estep * k - r.eoff;
            sE += (__int128)h * E;
            sE2 += (__int128)h * (E * E);
            r.Hsum[k] += h;
        }
        if (hm) {
            const long long M = r.potts_q ? (long long)k : 2ll * k - N;  // Potts: the majority state's size
            const long long aM = M < 0 ? -M : M;
            const long long M2 = M * M;
            sAM += (__int128)hm * aM;
            sM2 += (__int128)hm * M2;
            sM4 += (__int128)hm * ((__int128)M2 * M2);
        }
        if (rec_hist) {
            rec_hist[k] = h;
            rec_hist[NL + k] = hm;
        }
    }
    sE = warp_sum128(sE);
    sE2 = warp_sum128(sE2);
    sAM = warp_sum128(sAM);
    sM2 = warp_sum128(sM2);
    sM4 = warp_sum128(sM4);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, off));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
    }
    if (lane == 0) {
        ws[0][warp] = sE;
        ws[1][warp] = sE2;
        ws[2][warp] = sAM;
        ws[3][warp] = sM2;
        ws[4][warp] = sM4;
        wmin[warp] = kmin;
        wmax[warp] = kmax;
    }
    __syncthreads();
    // warps 0..4 each total one moment over the 32 warp partials (exact
    // integer sums); warp 5 the occupied range
    StepDev& rec = r.rec[step];
    if (warp < 5) {
        const I128 p = to_i128(warp_sum128(ws[warp][lane]));
        if (lane == 0) {
            rec.sums[2 * warp] = p.lo;
            rec.sums[2 * warp + 1] = p.hi;
        }
    } else if (warp == 5) {
        int mn = wmin[lane], mx = wmax[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        }
        if (lane == 0) {
            rec.kmin = mn;
            rec.kmax = mx;
            if (range) {
                range[0] = mn;
                range[1] = mx;
            }
        }
    }
    if (t == 0) {
        if (step == 0) {
            rec.R = r.R;
            rec.R_prev = r.R;
            rec.fam = (unsigned long long)r.R;
        }
    }
}

__global__ void __launch_bounds__(kOneCta) k_stats(const __grid_constant__ RunDev r, int step)
{
    if (*r.status) return;
    stats_body(r, step);
}

__global__ void __launch_bounds__(kOneCta) k_stats_batch(const __grid_constant__ BatchDev b, int step)
{
    const RunDev& r = b.runs[blockIdx.x];
    if (*r.status || step > r.nsteps) return;
    stats_body(r, step);
}

// ======================================================== one-CTA resampling
// For populations of at most kSmallCap slots, the per-step bookkeeping of a
// run is one launch of one 1024-thread CTA instead of five: optionally the
// statistics of population i-1 (deferred from the previous step when the
// whole schedule is enqueued at once), then S and the copy tables (as
// k_tables), then the copy numbers, their running offsets and the parent
// list (as k_counts + k_scan + k_parent). The slots are walked in chunks of
// 4096 (one Philox block of 4 slots per thread, RESAMPLE stream (i, j>>2, 2,
// 0) as in k_counts); each chunk's exclusive scan is added to the total of
// the chunks before it, so parent[] gets exactly the same old-slot order.
// A chunk that would take R_i past the capacity sets the capacity status
// before any of its parents is written.
// Rp: R_{i-1}; lv0: this thread's first four old-slot levels (loaded by
// the caller before the tables, -1 beyond Rp); sF, sU: the copy tables in
// shared memory over [kmin, ...] (null: read the global tables).
__device__ __forceinline__ void resample_small_body(const RunDev& r, int step, long long Rp, const int lv0[4],
                                                    const uint32_t* sF, const unsigned long long* sU, int kmin)
{
    __shared__ unsigned long long s_wsum[kOneCta / 32];
    __shared__ unsigned long long s_chunk;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int32_t* __restrict__ lev = r.elev[(step - 1) & 1];
    const PhiloxKey key{r.key[0], r.key[1]};
    const unsigned long long cap = (unsigned long long)r.cap;
    unsigned long long base = 0;  // copies of the chunks before this one (same in every thread)
    bool over = false;
    for (long long c0 = 0; c0 < Rp; c0 += 4 * kOneCta) {
        const long long j0 = c0 + 4 * t;
        unsigned long long cnt[4] = {0ull, 0ull, 0ull, 0ull};
        if (j0 < Rp) {
            const uint4 x = philox10(make_uint4((unsigned)step, (unsigned)(j0 >> 2), kTagResample, 0u), key);
            const unsigned xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int l = 0; l < 4; l++) {
                const long long j = j0 + l;
                if (j < Rp) {
                    const int lv = c0 == 0 ? lv0[l] : lev[j];
                    const uint32_t F = sF ? sF[lv - kmin] : r.F[lv];
                    const unsigned long long U = sF ? sU[lv - kmin] : r.U[lv];
                    cnt[l] = (unsigned long long)F + (((unsigned long long)xs[l] < U) ? 1ull : 0ull);
                }
            }
        }
        const unsigned long long tsum = cnt[0] + cnt[1] + cnt[2] + cnt[3];
        unsigned long long incl = tsum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of the 32 warp totals, and the chunk total
            const unsigned long long v = s_wsum[lane];
            unsigned long long w = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            s_wsum[lane] = w - v;
            if (lane == 31) s_chunk = w;
        }
        __syncthreads();
        const unsigned long long chunk = s_chunk;
        if (base + chunk > cap) {  // same decision in every thread
            over = true;
            break;
        }
        unsigned long long o = base + s_wsum[warp] + incl - tsum;
#pragma unroll
        for (int l = 0; l < 4; l++) {
            const long long j = j0 + l;
            for (unsigned long long c = 0; c < cnt[l]; c++) r.parent[o + c] = (uint32_t)j;
            o += cnt[l];
        }
        base += chunk;
        __syncthreads();  // s_wsum and s_chunk are rewritten by the next chunk
    }
    if (t == 0) {
        StepDev& rec = r.rec[step];
        rec.R = over ? 0ll : (long long)base;
        rec.R_prev = Rp;
        if (over) *r.status = kStatusCapacity;
        else if (base == 0) *r.status = kStatusExtinct;
        *r.work = 0u;
    }
}

constexpr int kSmallLevels = 2048;  // copy tables kept in shared memory up to this range

// The whole one-CTA step of run r (shared memory from the calling kernel)
template <bool kStats>
__device__ __forceinline__ void resample_small_step(const RunDev& r, int step, int* s_range, uint32_t* s_F,
                                                    unsigned long long* s_U)
{
    // loads that depend on nothing computed here, issued first: R_{i-1} and
    // this thread's first four old-slot levels (written by the previous step)
    const long long Rp = r.rec[step - 1].R;
    const int32_t* __restrict__ lev = r.elev[(step - 1) & 1];
    int lv0[4];
#pragma unroll
    for (int l = 0; l < 4; l++) lv0[l] = 4ll * threadIdx.x + l < Rp ? lev[4 * threadIdx.x + l] : -1;
    int kmin, kmax;
    if constexpr (kStats) {
        stats_body(r, step - 1, s_range);  // population i-1, deferred from its own step
        __syncthreads();
        kmin = s_range[0];
        kmax = s_range[1];
    } else {
        kmin = r.rec[step - 1].kmin;
        kmax = r.rec[step - 1].kmax;
    }
    const bool in_smem = kmax - kmin + 1 <= kSmallLevels;
    tables_body(r, step, kmin, kmax, in_smem ? s_F : nullptr, in_smem ? s_U : nullptr);
    __syncthreads();  // the copy tables and rec[step] are read by the whole CTA below
    resample_small_body(r, step, Rp, lv0, in_smem ? s_F : nullptr, in_smem ? s_U : nullptr, kmin);
}

template <bool kStats>
__global__ void __launch_bounds__(kOneCta) k_resample_small(const __grid_constant__ RunDev r, int step)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int s_range[2];
    __shared__ uint32_t s_F[kSmallLevels];
    __shared__ unsigned long long s_U[kSmallLevels];
    if (*r.status) return;
    resample_small_step<kStats>(r, step, s_range, s_F, s_U);
}

// The same for every run of a batch whose runs all have capacity <=
// kSmallCap: one CTA per run (blockIdx.x = run index). A run past its last
// step only does the statistics of that step (deferred to the step after
// it), then idles; the batch's last step is followed by k_stats_batch.
template <bool kStats>
__global__ void __launch_bounds__(kOneCta) k_resample_small_batch(const __grid_constant__ BatchDev b, int step)
{
    __shared__ int s_range[2];
    __shared__ uint32_t s_F[kSmallLevels];
    __shared__ unsigned long long s_U[kSmallLevels];
    const RunDev& r = b.runs[blockIdx.x];
    if (*r.status) return;
    if (step > r.nsteps) {
        if (kStats && step == r.nsteps + 1) stats_body(r, step - 1);
        return;
    }
    resample_small_step<kStats>(r, step, s_range, s_F, s_U);
}

// ======================================================== batched sweep
// Work items of step `step`, laid out in queue order: ceil(R_i / (replicas
// per warp)) per warp-group run (one per replica for CTA-wide groups, whose
// runs are swept by their own kernels and never read theirs). The runs that
// do not fill the device alone are cut into segments that share (L, threads
// per replica); each segment is swept by its own instance of the kernel
// below (compiled for that shape alone), on parallel branches of the
// captured graph, each with its own counter work[seg].
__global__ void k_plan(const __grid_constant__ BatchDev b, int step)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long acc = 0;
    for (int q = 0; q < b.nruns; q++) {
        b.item_off[q] = acc;
        const RunDev& r = b.runs[b.order[q]];
        if (*r.status == 0 && step <= r.nsteps) {
            const int per = r.gt > 32 ? 1 : 32 / r.gt;
            acc += (r.rec[step].R + per - 1) / per;
        }
    }
    b.item_off[b.nruns] = acc;
    for (int s = 0; s < b.nseg; s++) b.work[s] = 0u;
}

// (L, G) pairs a batched sweep can run: warp groups dividing the plane (a
// segment kernel, or the run's own sweep kernel when it fills the device), and
// one replica per 256-thread CTA for L >= 128 (always the run's own kernel)
#define PA_BATCH_SHAPES(X) X(8, 1) X(16, 2) X(16, 4) X(32, 8) X(32, 16) X(64, 16) X(64, 32) X(128, 32) X(256, 32)
#define PA_BATCH_CTA_SIZES(X) X(128) X(256) X(512)

// largest q in [0, n) with off[q] <= it
__device__ __forceinline__ int batch_run_of(const long long* off, int n, long long it)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Persistent sweep of the segment q0..q1-1 of the queue (warp-group runs of
// one shape): each warp takes (run, replica batch) items from the segment's
// counter work[seg]. (Runs of one replica per CTA are swept by their own
// sweep kernel, launched beside the segments.)
template <int L, int G>
__global__ void __launch_bounds__(256) k_sweep_batch_seg(const __grid_constant__ BatchDev b, int step, int q0, int q1,
                                                         int seg)
{
    static_assert(G <= 32, "warp groups only");
    using Gm = Geo<L>;
    using Gr = Group<G>;
    extern __shared__ uint32_t smem[];
    __shared__ long long s_off[kMaxBatchRuns + 1];
    const int nq = q1 - q0;
    for (int i = threadIdx.x; i <= nq; i += blockDim.x) s_off[i] = b.item_off[q0 + i];
    __syncthreads();
    const long long first = s_off[0], end = s_off[nq];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane / G;
    uint32_t* wsm = smem + warp * (Gr::kPerWarp * Gm::WORDS);
    for (;;) {
        const long long it = first + (long long)warp_grab(b.work + seg, 1u);
        if (it >= end) break;
        const int q = batch_run_of(s_off, nq, it);
        const RunDev& r = b.runs[b.order[q0 + q]];
        const long long k = (it - s_off[q]) * Gr::kPerWarp + g;
        unsigned fam = 0;
        bits_group_step<L, G>(r, step, k, k < r.rec[step].R, wsm + g * Gm::WORDS, lane % G, nullptr, fam);
        fam = group_sum<32>(fam);
        if (lane == 0 && fam) atomicAdd(&r.rec[step].fam, (unsigned long long)fam);
    }
}

// ======================================================== bounded-wait self-test
// One CTA of 32 threads runs the sweep's bulk-copy path on `bytes` bytes of
// src: thread 0 arms the barrier for them and, if `copy`, issues the copy;
// every thread waits at most `tries` polls. out[0] = 0 when the bytes landed
// and equal src, kStatusTimeout when the wait ran out (the barrier armed
// without a copy: nothing is in flight when the CTA exits), 1 when the
// bytes landed but differ.
__global__ void __launch_bounds__(32) k_bulk_selftest(const uint32_t* __restrict__ src, int bytes, int copy, int tries,
                                                     int* out)
{
    __shared__ __align__(16) uint32_t buf[1024];
    __shared__ __align__(8) unsigned long long mbar;
    if (threadIdx.x == 0) mbar_init(&mbar);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (copy) {
            bulk_load(buf, src, (unsigned)bytes, &mbar);
        } else {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar)),
                         "r"((unsigned)bytes)
                         : "memory");
        }
    }
    const bool landed = mbar_wait(&mbar, 0u, tries);
    unsigned diff = 0;
    if (landed)
        for (int i = threadIdx.x; i < bytes / 4; i += 32) diff |= buf[i] ^ src[i];
    diff = __reduce_or_sync(0xffffffffu, diff);
    if (threadIdx.x == 0) out[0] = !landed ? kStatusTimeout : (diff ? 1 : 0);
}

cudaError_t launch_bulk_selftest(const uint32_t* src, int bytes, bool copy, int tries, int* out, cudaStream_t s)
{
    if (bytes < 16 || bytes > 4096 || bytes % 16 || ((uintptr_t)src & 15) || tries < 1) return cudaErrorInvalidValue;
    k_bulk_selftest<<<1, 32, 0, s>>>(src, bytes, copy ? 1 : 0, tries, out);
    return cudaGetLastError();
}

// ======================================================== standalone gather
// The replica copy of the resampling step (the paper's resampleKer) on its
// own: new slot o receives the words of old slot parent[o]. The engine fuses
// this copy into the sweep's shared-memory load; this kernel measures the
// copy against HBM bandwidth. LPR lanes copy one replica in 16-byte vectors
// with streaming (evict-first) loads and stores; a parent outside the source
// is skipped and counted in *bad.
template <int LPR>
__global__ void __launch_bounds__(256) k_gather(const uint4* __restrict__ src, const uint32_t* __restrict__ parent,
                                                long long n_new, long long n_src, int w4, uint4* __restrict__ dst,
                                                unsigned* bad)
{
    constexpr int RPW = 32 / LPR;  // replicas per warp at a time
    const int lane = threadIdx.x & 31, sub = lane / LPR, l = lane % LPR;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long o = warp * RPW + sub; o < n_new; o += warps * RPW) {
        const uint32_t p = parent[o];
        if ((long long)p >= n_src) {
            if (l == 0) atomicAdd(bad, 1u);
            continue;
        }
        const uint4* s = src + (size_t)p * (size_t)w4;
        uint4* d = dst + (size_t)o * (size_t)w4;
        int i = l;
        for (; i + 3 * LPR < w4; i += 4 * LPR) {  // four loads in flight per lane
            const uint4 a = __ldcs(s + i), b = __ldcs(s + i + LPR), c = __ldcs(s + i + 2 * LPR),
                        e = __ldcs(s + i + 3 * LPR);
            __stcs(d + i, a);
            __stcs(d + i + LPR, b);
            __stcs(d + i + 2 * LPR, c);
            __stcs(d + i + 3 * LPR, e);
        }
        for (; i < w4; i += LPR) __stcs(d + i, __ldcs(s + i));
    }
}

cudaError_t launch_gather(const uint32_t* src, const uint32_t* parent, long long n_new, long long n_src, int words,
                          uint32_t* dst, unsigned* bad, int grid, cudaStream_t s)
{
    if (words < 4 || words % 4 || grid < 1) return cudaErrorInvalidValue;
    const int w4 = words / 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    if (w4 >= 32) k_gather<32><<<grid, 256, 0, s>>>(s4, parent, n_new, n_src, w4, d4, bad);
    else if (w4 >= 16) k_gather<16><<<grid, 256, 0, s>>>(s4, parent, n_new, n_src, w4, d4, bad);
    else if (w4 >= 8) k_gather<8><<<grid, 256, 0, s>>>(s4, parent, n_new, n_src, w4, d4, bad);
    else if (w4 >= 4) k_gather<4><<<grid, 256, 0, s>>>(s4, parent, n_new, n_src, w4, d4, bad);
    else if (w4 >= 2) k_gather<2><<<grid, 256, 0, s>>>(s4, parent, n_new, n_src, w4, d4, bad);
    else k_gather<1><<<grid, 256, 0, s>>>(s4, parent, n_new, n_src, w4, d4, bad);
    return cudaGetLastError();
}

// ======================================================== Philox test kernel
__global__ void k_philox(const uint32_t* __restrict__ ctr, long long n, PhiloxKey key, uint32_t* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = reinterpret_cast<const uint4*>(ctr)[i];
    reinterpret_cast<uint4*>(out)[i] = philox10(c, key);
}

// ======================================================== RNG ceiling
// Philox alone, with the counter layout of the sweep (only word 1 varies
// across lanes): the words are XOR-folded so none is dead code.
__global__ void __launch_bounds__(256) k_rng_peak(long long blocks, PhiloxKey key, uint32_t* __restrict__ sink)
{
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (long long q = 0; q < blocks; q += 8) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint4 x = philox10(make_uint4(12345u, (unsigned)(q + j) + 64u * tid, kTagSweep, 77u), key);
            acc ^= x.x ^ x.y ^ x.z ^ x.w;
        }
    }
    sink[tid] = acc;
}

// ======================================================== launch wrappers
namespace {

template <int L, int G, int D = 2, bool kBytes = false>
const void* bits_ptr(bool init)
{
    return init ? (const void*)k_init_bits<L, G, D, kBytes> : (const void*)k_sweep_bits<L, G, D, kBytes>;
}

// simple cubic lattice: the warp groups and CTA groups the default choice
// uses (power-of-two words per plane: 8, 64, 512, 4096 for L = 8 .. 64)
template <int L>
const void* bits3_ptr_L(int gt, bool init)
{
    constexpr int WP = Lat<L, 3>::WP;
    switch (gt) {
    case 8: if constexpr (WP % 8 == 0 && WP <= 64) return bits_ptr<L, 8, 3>(init); break;
    case 16: if constexpr (WP % 16 == 0 && WP <= 512) return bits_ptr<L, 16, 3>(init); break;
    case 32: if constexpr (WP % 32 == 0 && WP <= 512) return bits_ptr<L, 32, 3>(init); break;
    case 256: if constexpr (WP % 256 == 0) return bits_ptr<L, 256, 3>(init); break;
    default: break;
    }
    return nullptr;
}

template <int L, bool kBytes = false>
const void* bits_ptr_L(int gt, bool init)
{
    constexpr int WP = L * L / 64;
    switch (gt) {
    case 1: return bits_ptr<L, 1, 2, kBytes>(init);
    case 2: if constexpr (bits_group_ok<L, 2>(2)) return bits_ptr<L, 2, 2, kBytes>(init); break;
    case 4: if constexpr (bits_group_ok<L, 2>(4)) return bits_ptr<L, 4, 2, kBytes>(init); break;
    case 8: if constexpr (bits_group_ok<L, 2>(8)) return bits_ptr<L, 8, 2, kBytes>(init); break;
    case 16: if constexpr (bits_group_ok<L, 2>(16)) return bits_ptr<L, 16, 2, kBytes>(init); break;
    case 32: if constexpr (bits_group_ok<L, 2>(32)) return bits_ptr<L, 32, 2, kBytes>(init); break;
    case 256: if constexpr (WP % 256 == 0) return bits_ptr<L, 256, 2, kBytes>(init); break;
    default: break;
    }
    return nullptr;
}

template <int G>
const void* bytes_ptr(bool init)
{
    return init ? (const void*)k_init_bytes<G> : (const void*)k_sweep_bytes<G>;
}

template <int G>
const void* potts_ptr(bool init)
{
    return init ? (const void*)k_init_potts<G> : (const void*)k_sweep_potts<G>;
}

}  // namespace

// Square-lattice shapes with a sweep instance for grids that hold the whole
// population (the default shapes of small runs: several threads per word)
#define PA_COVER_SHAPES(X) X(8, 8) X(16, 32) X(32, 32)

namespace {
const void* cover_kernel(const RunDev& h)
{
    if (h.dim == 3 || !(h.fmt == 1 || (h.fmt == 0 && h.packed))) return nullptr;
    const bool bytes = h.fmt == 0;
    switch (h.L * 64 + h.gt) {
#define PA_COVER_PTR(LL, GG)                                                                  \
    case LL * 64 + GG:                                                                        \
        return bytes ? (const void*)k_sweep_bits<LL, GG, 2, true, true>                     \
                     : (const void*)k_sweep_bits<LL, GG, 2, false, true>;
        PA_COVER_SHAPES(PA_COVER_PTR)
#undef PA_COVER_PTR
    default: return nullptr;
    }
}
}  // namespace

// The init / sweep kernel of a run's (format, L, threads per replica).
const void* sweep_kernel(const RunDev& h, bool init)
{
    if (h.fmt == 3) return init ? (const void*)k_init_rp : (const void*)k_sweep_rp;
    if (h.fmt == 2) {
        switch (h.L) {
#define PA_MSC_PTR(LL) \
    case LL: return init ? (const void*)k_init_msc<LL> : (const void*)k_sweep_msc<LL>;
            PA_MSC_SIZES(PA_MSC_PTR)
#undef PA_MSC_PTR
        default: return nullptr;
        }
    }
    if (h.fmt == 1 && h.dim == 3) {
        switch (h.L) {
        case 8: return bits3_ptr_L<8>(h.gt, init);
        case 16: return bits3_ptr_L<16>(h.gt, init);
        case 32: return bits3_ptr_L<32>(h.gt, init);
        case 64: return bits3_ptr_L<64>(h.gt, init);
        default: return nullptr;
        }
    }
    if (h.fmt == 0 && h.packed) {
        // byte-stored spins swept in the bit-packed kernel (packed on load)
        switch (h.L) {
        case 8: return bits_ptr_L<8, true>(h.gt, init);
        case 16: return bits_ptr_L<16, true>(h.gt, init);
        case 32: return bits_ptr_L<32, true>(h.gt, init);
        case 64: return bits_ptr_L<64, true>(h.gt, init);
        case 128: return bits_ptr_L<128, true>(h.gt, init);
        case 256: return bits_ptr_L<256, true>(h.gt, init);
        case 512: return bits_ptr_L<512, true>(h.gt, init);
        default: return nullptr;
        }
    }
    if (h.fmt == 1) {
        switch (h.L) {
        case 8: return bits_ptr_L<8>(h.gt, init);
        case 16: return bits_ptr_L<16>(h.gt, init);
        case 32: return bits_ptr_L<32>(h.gt, init);
        case 64: return bits_ptr_L<64>(h.gt, init);
        case 128: return bits_ptr_L<128>(h.gt, init);
        case 256: return bits_ptr_L<256>(h.gt, init);
        case 512: return bits_ptr_L<512>(h.gt, init);
        default: return nullptr;
        }
    }
    if (h.potts_q) {
        switch (h.gt) {
        case 1: return potts_ptr<1>(init);
        case 2: return potts_ptr<2>(init);
        case 4: return potts_ptr<4>(init);
        case 8: return potts_ptr<8>(init);
        case 16: return potts_ptr<16>(init);
        case 32: return potts_ptr<32>(init);
        default: return nullptr;
        }
    }
    switch (h.gt) {
    case 1: return bytes_ptr<1>(init);
    case 2: return bytes_ptr<2>(init);
    case 4: return bytes_ptr<4>(init);
    case 8: return bytes_ptr<8>(init);
    case 16: return bytes_ptr<16>(init);
    case 32: return bytes_ptr<32>(init);
    default: return nullptr;
    }
}

static int msc_threads_of(int L)
{
    switch (L) {
#define PA_MSC_THR(LL) \
    case LL: return msc_threads<LL>();
        PA_MSC_SIZES(PA_MSC_THR)
#undef PA_MSC_THR
    default: return 0;
    }
}

cudaError_t plan_sweep(const RunDev& h, Launch* ln)
{
    int dev = 0, sms = 0, max_optin = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    const void* kin = sweep_kernel(h, true);
    const void* ksw = sweep_kernel(h, false);
    if (!kin || !ksw) return cudaErrorInvalidConfiguration;
    size_t smem;
    int threads;
    if (h.fmt == 3) {
        // one thread per replica over the whole capacity, no shared memory
        ln->sweep_threads = 256;
        ln->sweep_smem = 0;
        ln->sweep_blocks = (int)((h.cap + 255) / 256);
        ln->sweep_full = false;
        ln->count_blocks = h.ntiles;
        return cudaSuccess;
    }
    if (h.fmt == 2) {
        // one 32-replica group per CTA: its N site words and the reductions
        threads = msc_threads_of(h.L);
        if (threads <= 0) return cudaErrorInvalidConfiguration;
        smem = ((size_t)h.N + 2 * (size_t)threads + 1) * 4u;
    } else if (h.gt > 32) {
        // one replica per CTA of gt threads, plus reduction/broadcast words;
        // bit-packed sweeps keep a second replica buffer for the bulk prefetch
        threads = h.gt;
        const size_t rep = h.packed ? (size_t)h.N / 32 : (size_t)h.words;
        smem = ((h.fmt == 1 && rep <= (size_t)kPrefetchMaxWords ? 2 : 1) * rep + 33) * 4u;
    } else {
        // CTA of up to 8 warps; fewer when one warp's replicas need much shared memory
        const size_t rep_words = h.packed ? (size_t)h.N / 32 : (size_t)h.words;  // packed image of a byte replica
        const size_t per_warp = (size_t)(32 / h.gt) * rep_words * 4u;
        int warps = h.bw > 0 && h.bw <= 8 ? h.bw : 8;
        while (warps > 1 && per_warp * warps > (size_t)max_optin) warps >>= 1;
        smem = per_warp * warps;
        threads = 32 * warps;
    }
    if (smem > (size_t)max_optin) return cudaErrorInvalidConfiguration;
    for (const void* k : {kin, ksw}) {
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
    }
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ksw, threads, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // persistent grid: enough CTAs to hold every replica of a full population
    // at once, at most what the device keeps resident
    long long units;  // work items of a full population, and their number per CTA
    long long per_cta;
    if (h.fmt == 2) {
        units = (h.cap + 31) / 32;
        per_cta = 1;
    } else if (h.gt > 32) {
        units = h.cap;
        per_cta = 1;
    } else {
        units = h.cap;
        per_cta = (long long)(threads / 32) * (32 / h.gt);
    }
    const long long need = (units + per_cta - 1) / per_cta;
    ln->sweep_threads = threads;
    ln->sweep_smem = smem;
    ln->sweep_blocks = (int)std::max(1ll, std::min((long long)sms * per_sm, need));
    ln->sweep_full = need >= (long long)sms * per_sm;
    // a grid that holds the whole capacity can sweep with one fixed replica
    // per group (no counter), where that instance exists
    ln->sweep_cover = nullptr;
    if (need <= (long long)sms * per_sm) {
        const void* kc = cover_kernel(h);
        int per_sm_c = 0;
        if (kc && cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, kc, threads, smem) == cudaSuccess &&
            per_sm_c >= 1 && (long long)sms * per_sm_c >= need)
            ln->sweep_cover = kc;
        cudaGetLastError();
    }
    ln->count_blocks = h.ntiles;
    return cudaSuccess;
}

cudaError_t launch_init(const RunDev* /*d_run*/, const RunDev& h, const Launch& ln, cudaStream_t s)
{
    const void* k = sweep_kernel(h, true);
    if (!k) return cudaErrorInvalidConfiguration;
    RunDev arg = h;
    void* args[] = {&arg};
    return cudaLaunchKernel(k, dim3(ln.sweep_blocks), dim3(ln.sweep_threads), args, ln.sweep_smem, s);
}

// A launch of kernel k that may overlap the previous kernel of stream s
// (programmatic serialization; the kernel starts with pdl_wait)
static cudaError_t launch_pdl(const void* k, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k, args);
}

cudaError_t launch_sweep(const RunDev* /*d_run*/, const RunDev& h, const Launch& ln, int step, cudaStream_t s,
                         bool pdl)
{
    const void* k = ln.sweep_cover ? ln.sweep_cover : sweep_kernel(h, false);
    if (!k) return cudaErrorInvalidConfiguration;
    RunDev arg = h;
    int st = step;
    void* args[] = {&arg, &st};
    if (pdl) return launch_pdl(k, dim3(ln.sweep_blocks), dim3(ln.sweep_threads), args, ln.sweep_smem, s);
    return cudaLaunchKernel(k, dim3(ln.sweep_blocks), dim3(ln.sweep_threads), args, ln.sweep_smem, s);
}

cudaError_t launch_tables(const RunDev* /*d_run*/, const RunDev& h, int step, cudaStream_t s)
{
    k_tables<<<1, kOneCta, 0, s>>>(h, step);
    return cudaGetLastError();
}

cudaError_t launch_counts(const RunDev* /*d_run*/, const RunDev& h, const Launch& ln, int step, cudaStream_t s)
{
    k_counts<<<ln.count_blocks, kTileThreads, 0, s>>>(resample_args(h, step));
    return cudaGetLastError();
}

cudaError_t launch_scan(const RunDev* /*d_run*/, const RunDev& h, int step, cudaStream_t s)
{
    k_scan<<<1, kOneCta, 0, s>>>(resample_args(h, step));
    return cudaGetLastError();
}

cudaError_t launch_parent(const RunDev* /*d_run*/, const RunDev& h, const Launch& ln, int step, cudaStream_t s)
{
    k_parent<<<ln.count_blocks, kTile, 0, s>>>(resample_args(h, step));
    return cudaGetLastError();
}

cudaError_t launch_resample(const ResampleArgs& a, int tiles, cudaStream_t s)
{
    if (tiles < 1) return cudaErrorInvalidValue;
    k_counts<<<tiles, kTileThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan<<<1, kOneCta, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_parent<<<tiles, kTile, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resample_small(const RunDev& h, int step, bool with_stats, cudaStream_t s, bool pdl)
{
    if (h.cap > kSmallCap) return cudaErrorInvalidValue;
    if (pdl) {
        RunDev arg = h;
        int st = step;
        void* args[] = {&arg, &st};
        const void* k = with_stats ? (const void*)k_resample_small<true> : (const void*)k_resample_small<false>;
        return launch_pdl(k, dim3(1), dim3(kOneCta), args, 0, s);
    }
    if (with_stats) k_resample_small<true><<<1, kOneCta, 0, s>>>(h, step);
    else k_resample_small<false><<<1, kOneCta, 0, s>>>(h, step);
    return cudaGetLastError();
}

cudaError_t launch_stats(const RunDev* /*d_run*/, const RunDev& h, int step, cudaStream_t s)
{
    k_stats<<<1, kOneCta, 0, s>>>(h, step);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, long long n, PhiloxKey key, uint32_t* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (n + threads - 1) / threads;
    k_philox<<<(unsigned)blocks, threads, 0, s>>>(ctr, n, key, out);
    return cudaGetLastError();
}

bool batch_supports(int L, int gt)
{
    if (gt == 256) {
        switch (L) {
#define PA_BATCH_CTA_OK(LL) case LL:
            PA_BATCH_CTA_SIZES(PA_BATCH_CTA_OK)
#undef PA_BATCH_CTA_OK
            return true;
        default: return false;
        }
    }
    switch (L * 64 + gt) {
#define PA_BATCH_OK(LL, GG) case LL * 64 + GG:
        PA_BATCH_SHAPES(PA_BATCH_OK)
#undef PA_BATCH_OK
        return true;
    default: return false;
    }
}

namespace {
// the segment kernel of shape (L, G), or null
const void* batch_seg_kernel(int L, int G)
{
    if (G > 32) return nullptr;  // CTA groups: swept by each run's own kernel
    switch (L * 64 + G) {
#define PA_BATCH_PTR(LL, GG) \
    case LL * 64 + GG: return (const void*)k_sweep_batch_seg<LL, GG>;
        PA_BATCH_SHAPES(PA_BATCH_PTR)
#undef PA_BATCH_PTR
    default: return nullptr;
    }
}
}  // namespace

// Grid and shared memory of a segment's kernel: enough persistent CTAs for
// `units` replicas (the capacities of its runs), at most the resident ones.
cudaError_t plan_batch_segment(BatchSeg* sg, long long units)
{
    int dev = 0, sms = 0, max_optin = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    const void* k = batch_seg_kernel(sg->L, sg->G);
    if (!k) return cudaErrorInvalidConfiguration;
    const size_t words = (size_t)sg->L * sg->L / 32;
    const size_t smem = (size_t)8 * (32 / sg->G) * words * 4;  // 8 warps of 32/G replicas
    const size_t fixed = (kMaxBatchRuns + 1) * 8 + 64;  // static shared memory of the kernel
    if (smem + fixed > (size_t)max_optin) return cudaErrorInvalidConfiguration;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long per_cta = 8ll * (32 / sg->G);
    const long long need = std::max(1ll, (units + per_cta - 1) / per_cta);
    sg->blocks = (int)std::min((long long)sms * per_sm, need);
    sg->smem = smem;
    return cudaSuccess;
}

// Whether phase `phase` of step `step` launches anything: batches of small
// runs do phases 0-3 (and the statistics, deferred) in one launch, and
// their statistics phase only after the last step.
bool batch_phase_launches(const BatchLaunch& ln, int step, int phase)
{
    if (!ln.small) return true;
    if (phase >= 1 && phase <= 3) return false;
    return phase != 5 || step == ln.last;
}

// One phase of a batched step: 0 tables, 1 counts, 2 scan, 3 parent, 4 plan +
// sweep, 5 stats (the phase numbers of pa_phase_times); in batches of small
// runs, phase 0 is the one-CTA resampling (with the previous step's
// statistics) and phase 5 only follows the last step.
cudaError_t launch_batch_step(const BatchDev& b, const BatchLaunch& ln, int step, cudaStream_t s, int phase,
                              int* /*unused*/)
{
    if (!batch_phase_launches(ln, step, phase)) return cudaSuccess;
    switch (phase) {
    case 0:
        if (!ln.small) k_tables_batch<<<b.nruns, kOneCta, 0, s>>>(b, step);
        else if (step > 1) k_resample_small_batch<true><<<b.nruns, kOneCta, 0, s>>>(b, step);
        else k_resample_small_batch<false><<<b.nruns, kOneCta, 0, s>>>(b, step);
        break;
    case 1: k_counts_batch<<<ln.tiles, kTileThreads, 0, s>>>(b, step); break;
    case 2: k_scan_batch<<<b.nruns, kOneCta, 0, s>>>(b, step); break;
    case 3: k_parent_batch<<<ln.tiles, kTile, 0, s>>>(b, step); break;
    case 4: {
        k_plan<<<1, 32, 0, s>>>(b, step);
        cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) return e;
        // every segment on its own branch, the own-kernel runs in turn on
        // kBatchOwnStreams more: the kernels overlap at their tails
        int live = 0;  // own-kernel runs still stepping
        for (int j = 0; j < ln.nown; j++) live += step <= ln.own_last[j];
        const int ncs = std::min(live, kBatchOwnStreams);
        const bool fork = ln.nseg + ncs > 1;
        if (fork && (e = cudaEventRecord(ln.fork, s)) != cudaSuccess) return e;
        for (int i = 0; i < ln.nseg; i++) {
            const BatchSeg& sg = ln.seg[i];
            cudaStream_t t = fork ? ln.side[i] : s;
            if (fork && (e = cudaStreamWaitEvent(t, ln.fork, 0)) != cudaSuccess) return e;
            BatchDev arg = b;
            int st = step, q0 = sg.q0, q1 = sg.q1, si = i;
            void* args[] = {&arg, &st, &q0, &q1, &si};
            if ((e = cudaLaunchKernel(batch_seg_kernel(sg.L, sg.G), dim3(sg.blocks), dim3(256), args, sg.smem, t)) !=
                cudaSuccess)
                return e;
            if (fork) {
                if ((e = cudaEventRecord(ln.join[i], t)) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(s, ln.join[i], 0)) != cudaSuccess) return e;
            }
        }
        for (int i = 0; i < ncs; i++)
            if (fork && (e = cudaStreamWaitEvent(ln.own_side[i], ln.fork, 0)) != cudaSuccess) return e;
        for (int j = 0, n = 0; j < ln.nown; j++) {
            if (step > ln.own_last[j]) continue;
            cudaStream_t t = fork ? ln.own_side[n++ % kBatchOwnStreams] : s;
            if ((e = launch_sweep(nullptr, ln.own_h[j], ln.own_ln[j], step, t)) != cudaSuccess) return e;
        }
        for (int i = 0; fork && i < ncs; i++) {
            if ((e = cudaEventRecord(ln.own_join[i], ln.own_side[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, ln.own_join[i], 0)) != cudaSuccess) return e;
        }
        break;
    }
    case 5: k_stats_batch<<<b.nruns, kOneCta, 0, s>>>(b, step); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rng_peak(long long blocks, uint32_t* sink, int grid, int threads, cudaStream_t s)
{
    k_rng_peak<<<grid, threads, 0, s>>>(blocks, PhiloxKey{0x1234u, 0x5678u}, sink);
    return cudaGetLastError();
}

}  // namespace pa
