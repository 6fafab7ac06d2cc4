/*
 * Population-annealing ORACLE, C part: the per-site Monte Carlo loops.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain CPU statement of what
 * the GPU engine computes. Only the tests, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load it. It shares no code, header, table
 * or constant generator with the CUDA engine under paper_1703_03676_gb300/.
 *
 * Model (Sec. 3, Eq. hamiltonian): H = -sum_<ij> s_i s_j on a periodic L x L
 * lattice, J = 1. Spins are stored in the natural layout s[y*L + x] as int8
 * +1/-1, one replica after the other.
 *
 * Random numbers (Sec. 3, "Spin updates"): the paper draws one uniform per
 * spin-flip attempt from the counter-based Philox4x32-10 generator of Salmon,
 * Moraes, Dror and Shaw (SC'11). Philox is written here from that
 * publication's definition: ten rounds of two 32x32->64 multiplications with
 * M0 = 0xD2511F53 and M1 = 0xCD9E8D57, the high halves XORed with the other
 * counter words and the round key, and a Weyl key schedule with increments
 * 0x9E3779B9 and 0xBB67AE85.
 *
 * Counter layout ("stream map"). The paper seeds per thread from grid and
 * block indices, which would tie the result to the launch shape; here the
 * counter is a function of logical indices only, so any implementation that
 * visits the same (replica, site, sweep) gets the same number. The index
 * that differs between neighbouring sites (or slots) sits in counter word 1
 * and the stream tag in word 2:
 *   key = (seed & 0xffffffff, seed >> 32)
 *   INIT     (tag 0): g = c*N/2 + b,  ctr = (0, g>>2, 0, k),        x = out[g&3]
 *   SWEEP    (tag 1): ctr = (2u + c, b>>2, 1, k),                   x = out[b&3]
 *   RESAMPLE (tag 2): ctr = (i, j>>2, 2, 0),                        x = out[j&3]
 *   MSC seed (tag 5): ctr = (2u + c, b>>2, 5, k/32),               x = out[b&3]
 *   POTTS    (tag 6): ctr = (2u + c, b>>1, 6, k), proposal word out[2(b&1)],
 *                     acceptance word out[2(b&1) + 1]
 * where c = (x+y)&1 is the checkerboard colour of site (x, y),
 * b = y*(L/2) + (x>>1) its index within the colour, k the replica slot,
 * u the global sweep number, i the temperature step and j the old slot.
 *
 * The three-dimensional model (the simple cubic L x L x L torus, one of the
 * other models the paper's conclusion names for the method) uses the same
 * streams with c = (x+y+z)&1 and b = (z*L + y)*(L/2) + (x>>1), spins stored
 * as s[(z*L + y)*L + x].
 */
#include <stdint.h>
#include <stddef.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

/* Philox4x32-10 bijection of a 128-bit counter under a 64-bit key. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One 32-bit word of a tagged stream: lane l of Philox(ctr = (c0, c1, tag, c3)). */
static uint32_t stream_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t tag,
                            uint32_t c3, unsigned lane)
{
    uint32_t ctr[4] = {c0, c1, tag, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[lane & 3u];
}

/*
 * Initial configurations at beta0 = 0 (Sec. 2.1, step 1): independent spins,
 * +1 with probability 1/2. Spin = +1 iff the INIT word is < 2^31.
 * slot[r] is the replica index k of the r-th replica in `s`.
 */
void oracle_init(int L, int64_t n, const int64_t *slot, uint64_t seed, int8_t *s)
{
    const int N = L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int y = 0; y < L; y++)
            for (int x = 0; x < L; x++) {
                uint32_t c = (uint32_t)((x + y) & 1);
                uint32_t b = (uint32_t)(y * half + (x >> 1));
                uint32_t g = c * (uint32_t)(N / 2) + b;
                uint32_t w = stream_word(seed, 0u, g >> 2, 0u, k, g & 3u);
                S[y * L + x] = (w < 0x80000000u) ? 1 : -1;
            }
    }
}

/*
 * theta Metropolis sweeps at one inverse temperature (Sec. 2.1 step 3,
 * Sec. 3 "Spin updates"). Each sweep updates colour 0 first, then colour 1
 * (checkerboard decomposition, Fig. 1): all sites of one colour are
 * independent, so visiting them in raster order is one valid order.
 *
 * A flip changes the energy by dE = 2 s_i sum_nb s_j = 4 n - 8, where n is
 * the number of the four neighbours aligned with s_i. Metropolis accepts with
 * probability min(1, exp(-beta dE)): always for n <= 2, exp(-4 beta) for
 * n = 3, exp(-8 beta) for n = 4. With x the SWEEP word, a flip with n = 3 is
 * accepted iff x < T4, with n = 4 iff x < T8, where T = ceil(p * 2^32)
 * (computed by the caller) makes Pr[x < T] = p up to 2^-32.
 * Sweep number u runs from u0 to u0 + theta - 1.
 */
/* Couplings of the +-J model (Sec. 1: the method is for disordered systems
 * too): Jr[y*L+x] couples (x,y) to (x+1,y), Jd[y*L+x] couples it to
 * (x,y+1); NULL means the ferromagnet (all +1). A neighbour is "aligned"
 * when J s_i s_j = +1, so dE = 4 n - 8 as before. */
static int jr(const int8_t *Jr, int L, int x, int y) { return Jr ? Jr[y * L + x] : 1; }
static int jd(const int8_t *Jd, int L, int x, int y) { return Jd ? Jd[y * L + x] : 1; }

static int aligned_j(const int8_t *S, const int8_t *Jr, const int8_t *Jd, int L, int x, int y)
{
    int si = S[y * L + x];
    int xr = (x + 1) % L, xl = (x + L - 1) % L, yd = (y + 1) % L, yu = (y + L - 1) % L;
    return (jr(Jr, L, x, y) * si * S[y * L + xr] == 1) + (jr(Jr, L, xl, y) * si * S[y * L + xl] == 1) +
           (jd(Jd, L, x, y) * si * S[yd * L + x] == 1) + (jd(Jd, L, x, yu) * si * S[yu * L + x] == 1);
}

void oracle_sweep_j(int L, int64_t n, const int64_t *slot, uint64_t seed, int64_t u0, int theta,
                    uint64_t T4, uint64_t T8, const int8_t *Jr, const int8_t *Jd, int8_t *s)
{
    const int N = L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int sw = 0; sw < theta; sw++) {
            uint32_t u = (uint32_t)(u0 + sw);
            for (int c = 0; c < 2; c++) {
                for (int y = 0; y < L; y++)
                    for (int x = 0; x < L; x++) {
                        if (((x + y) & 1) != c)
                            continue;
                        int aligned = aligned_j(S, Jr, Jd, L, x, y);
                        int flip = 1;
                        if (aligned > 2) {
                            uint32_t b = (uint32_t)(y * half + (x >> 1));
                            uint32_t w = stream_word(seed, 2u * u + (uint32_t)c, b >> 2, 1u, k, b & 3u);
                            flip = ((uint64_t)w < ((aligned == 3) ? T4 : T8));
                        }
                        if (flip)
                            S[y * L + x] = (int8_t)(-S[y * L + x]);
                    }
            }
        }
    }
}

void oracle_measure_j(int L, int64_t n, const int8_t *s, const int8_t *Jr, const int8_t *Jd,
                      int64_t *E, int64_t *M)
{
    const int N = L * L;
    for (int64_t r = 0; r < n; r++) {
        const int8_t *S = s + (size_t)r * N;
        int64_t e = 0, m = 0;
        for (int y = 0; y < L; y++)
            for (int x = 0; x < L; x++) {
                int si = S[y * L + x];
                e -= si * (jr(Jr, L, x, y) * S[y * L + (x + 1) % L] + jd(Jd, L, x, y) * S[((y + 1) % L) * L + x]);
                m += si;
            }
        E[r] = e;
        M[r] = m;
    }
}

void oracle_sweep(int L, int64_t n, const int64_t *slot, uint64_t seed, int64_t u0,
                  int theta, uint64_t T4, uint64_t T8, int8_t *s)
{
    const int N = L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int sw = 0; sw < theta; sw++) {
            uint32_t u = (uint32_t)(u0 + sw);
            for (int c = 0; c < 2; c++) {
                for (int y = 0; y < L; y++)
                    for (int x = 0; x < L; x++) {
                        if (((x + y) & 1) != c)
                            continue;
                        int si = S[y * L + x];
                        int aligned = (S[y * L + (x + 1) % L] == si) +
                                      (S[y * L + (x + L - 1) % L] == si) +
                                      (S[((y + 1) % L) * L + x] == si) +
                                      (S[((y + L - 1) % L) * L + x] == si);
                        int flip;
                        if (aligned <= 2) {
                            flip = 1;  /* dE <= 0 */
                        } else {
                            uint32_t b = (uint32_t)(y * half + (x >> 1));
                            uint32_t w = stream_word(seed, 2u * u + (uint32_t)c, b >> 2, 1u, k, b & 3u);
                            uint64_t T = (aligned == 3) ? T4 : T8;
                            flip = ((uint64_t)w < T);
                        }
                        if (flip)
                            S[y * L + x] = (int8_t)(-si);
                    }
            }
        }
    }
}

/*
 * Multi-spin-coded variant (Sec. 4): replicas are grouped 32 per machine
 * word (replica k is bit k%32 of group k/32) and, as in the paper's LCG
 * variant, one Philox word per (group, site, sweep, colour) seeds a linear
 * congruential generator r_{n+1} = A r_n + C mod 2^32 with A = 1664525 and
 * C = 1013904223 that supplies the 32 replicas' random numbers: replica bit
 * j uses r_{j+1}, r_0 being the seed. The seed is the MSC stream word
 * (tag 5): ctr = (2u + c, b>>2, 5, k/32), x = out[b&3]. Everything else
 * (acceptance rule, thresholds, colour order) is as in oracle_sweep.
 */
#define LCG_A 1664525u
#define LCG_C 1013904223u

static uint32_t msc_word(uint64_t seed, uint32_t u, uint32_t c, uint32_t b, uint32_t k)
{
    uint32_t r = stream_word(seed, 2u * u + c, b >> 2, 5u, k >> 5, b & 3u);
    for (uint32_t j = 0; j <= (k & 31u); j++)
        r = LCG_A * r + LCG_C;
    return r;
}

/* The random word of replica k at site b of colour c in sweep u (for tests). */
uint32_t oracle_msc_word(uint64_t seed, uint32_t u, uint32_t c, uint32_t b, uint32_t k)
{
    return msc_word(seed, u, c, b, k);
}

void oracle_sweep_msc(int L, int64_t n, const int64_t *slot, uint64_t seed, int64_t u0,
                      int theta, uint64_t T4, uint64_t T8, int8_t *s)
{
    const int N = L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int sw = 0; sw < theta; sw++) {
            uint32_t u = (uint32_t)(u0 + sw);
            for (int c = 0; c < 2; c++) {
                for (int y = 0; y < L; y++)
                    for (int x = 0; x < L; x++) {
                        if (((x + y) & 1) != c)
                            continue;
                        int si = S[y * L + x];
                        int aligned = (S[y * L + (x + 1) % L] == si) +
                                      (S[y * L + (x + L - 1) % L] == si) +
                                      (S[((y + 1) % L) * L + x] == si) +
                                      (S[((y + L - 1) % L) * L + x] == si);
                        int flip;
                        if (aligned <= 2) {
                            flip = 1;
                        } else {
                            uint32_t b = (uint32_t)(y * half + (x >> 1));
                            uint32_t w = msc_word(seed, u, (uint32_t)c, b, k);
                            uint64_t T = (aligned == 3) ? T4 : T8;
                            flip = ((uint64_t)w < T);
                        }
                        if (flip)
                            S[y * L + x] = (int8_t)(-si);
                    }
            }
        }
    }
}

/* Configurational energy E = -sum over bonds s_i s_j and magnetisation M. */
void oracle_measure(int L, int64_t n, const int8_t *s, int64_t *E, int64_t *M)
{
    const int N = L * L;
    for (int64_t r = 0; r < n; r++) {
        const int8_t *S = s + (size_t)r * N;
        int64_t e = 0, m = 0;
        for (int y = 0; y < L; y++)
            for (int x = 0; x < L; x++) {
                int si = S[y * L + x];
                e -= si * (S[y * L + (x + 1) % L] + S[((y + 1) % L) * L + x]);
                m += si;
            }
        E[r] = e;
        M[r] = m;
    }
}

/* The resampling uniform word of each old slot j = 0..n-1 at step i. */
void oracle_resample_words(uint64_t seed, int64_t step, int64_t n, uint32_t *out)
{
    for (int64_t j = 0; j < n; j++)
        out[j] = stream_word(seed, (uint32_t)step, (uint32_t)(j >> 2), 2u, 0u, (unsigned)(j & 3));
}

/* Raw Philox block for tests: out[4*r .. 4*r+3] = Philox(ctr[4*r..], key). */
void oracle_philox_many(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int64_t r = 0; r < n; r++)
        oracle_philox4x32_10(ctr + 4 * r, key, out + 4 * r);
}

/* ------------------------------------------------------------------ 3D
 * Simple cubic L x L x L torus, H = -sum over the 3N bonds (each site's +x,
 * +y and +z neighbour). A flip changes the energy by dE = 2 s_i sum_nb s_j =
 * 4 n - 12 with n the number of the six neighbours aligned with s_i:
 * always accepted for n <= 3, with probability exp(-4 beta), exp(-8 beta),
 * exp(-12 beta) for n = 4, 5, 6, i.e. iff the SWEEP word is < T4, T8, T12.
 * L = 2 is allowed here: the +x and -x neighbours are then the same site,
 * counted twice, consistently in the energy and in dE.
 */
static int site3(int L, int x, int y, int z)
{
    return (z * L + y) * L + x;
}

void oracle_init3(int L, int64_t n, const int64_t *slot, uint64_t seed, int8_t *s)
{
    const int N = L * L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int z = 0; z < L; z++)
            for (int y = 0; y < L; y++)
                for (int x = 0; x < L; x++) {
                    uint32_t c = (uint32_t)((x + y + z) & 1);
                    uint32_t b = (uint32_t)((z * L + y) * half + (x >> 1));
                    uint32_t g = c * (uint32_t)(N / 2) + b;
                    uint32_t w = stream_word(seed, 0u, g >> 2, 0u, k, g & 3u);
                    S[site3(L, x, y, z)] = (w < 0x80000000u) ? 1 : -1;
                }
    }
}

void oracle_sweep3(int L, int64_t n, const int64_t *slot, uint64_t seed, int64_t u0, int theta, uint64_t T4,
                   uint64_t T8, uint64_t T12, int8_t *s)
{
    const int N = L * L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int sw = 0; sw < theta; sw++) {
            uint32_t u = (uint32_t)(u0 + sw);
            for (int c = 0; c < 2; c++) {
                for (int z = 0; z < L; z++)
                    for (int y = 0; y < L; y++)
                        for (int x = 0; x < L; x++) {
                            if (((x + y + z) & 1) != c)
                                continue;
                            int si = S[site3(L, x, y, z)];
                            int aligned = (S[site3(L, (x + 1) % L, y, z)] == si) +
                                          (S[site3(L, (x + L - 1) % L, y, z)] == si) +
                                          (S[site3(L, x, (y + 1) % L, z)] == si) +
                                          (S[site3(L, x, (y + L - 1) % L, z)] == si) +
                                          (S[site3(L, x, y, (z + 1) % L)] == si) +
                                          (S[site3(L, x, y, (z + L - 1) % L)] == si);
                            int flip;
                            if (aligned <= 3) {
                                flip = 1;  /* dE <= 0 */
                            } else {
                                uint32_t b = (uint32_t)((z * L + y) * half + (x >> 1));
                                uint32_t w = stream_word(seed, 2u * u + (uint32_t)c, b >> 2, 1u, k, b & 3u);
                                uint64_t T = (aligned == 4) ? T4 : (aligned == 5) ? T8 : T12;
                                flip = ((uint64_t)w < T);
                            }
                            if (flip)
                                S[site3(L, x, y, z)] = (int8_t)(-si);
                        }
            }
        }
    }
}

void oracle_measure3(int L, int64_t n, const int8_t *s, int64_t *E, int64_t *M)
{
    const int N = L * L * L;
    for (int64_t r = 0; r < n; r++) {
        const int8_t *S = s + (size_t)r * N;
        int64_t e = 0, m = 0;
        for (int z = 0; z < L; z++)
            for (int y = 0; y < L; y++)
                for (int x = 0; x < L; x++) {
                    int si = S[site3(L, x, y, z)];
                    e -= si * (S[site3(L, (x + 1) % L, y, z)] + S[site3(L, x, (y + 1) % L, z)] +
                               S[site3(L, x, y, (z + 1) % L)]);
                    m += si;
                }
        E[r] = e;
        M[r] = m;
    }
}

/* ------------------------------------------------------------------ Potts
 * q-state Potts model on the periodic L x L lattice (one of the further
 * models the paper's conclusion names): H = -sum over the 2N bonds of
 * delta(s_i, s_j), s in {0, .., q-1}. Readings:
 *  - initial states: s = floor(x q / 2^32) with x the INIT word of the site;
 *  - Metropolis update of a site in state s: the POTTS words (w0, w1) of the
 *    site propose s' = (s + 1 + floor(w0 (q-1) / 2^32)) mod q, uniform over
 *    the q-1 other states; with n(t) the number of the four neighbours in
 *    state t, dE = n(s) - n(s'); accepted if dE <= 0, else iff w1 < T[dE-1],
 *    T[d-1] = ceil(exp(-d beta) 2^32) (computed by the caller), d = 1 .. 4;
 *  - "magnetisation" M = the number of sites in the most populated state.
 */
static uint32_t potts_state(uint64_t x, int q)
{
    return (uint32_t)((x * (uint64_t)q) >> 32);
}

void oracle_init_potts(int L, int q, int64_t n, const int64_t *slot, uint64_t seed, int8_t *s)
{
    const int N = L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int y = 0; y < L; y++)
            for (int x = 0; x < L; x++) {
                uint32_t c = (uint32_t)((x + y) & 1);
                uint32_t b = (uint32_t)(y * half + (x >> 1));
                uint32_t g = c * (uint32_t)(N / 2) + b;
                uint32_t w = stream_word(seed, 0u, g >> 2, 0u, k, g & 3u);
                S[y * L + x] = (int8_t)potts_state(w, q);
            }
    }
}

void oracle_sweep_potts(int L, int q, int64_t n, const int64_t *slot, uint64_t seed, int64_t u0, int theta,
                        const uint64_t *T, int8_t *s)
{
    const int N = L * L, half = L / 2;
    for (int64_t r = 0; r < n; r++) {
        int8_t *S = s + (size_t)r * N;
        uint32_t k = (uint32_t)slot[r];
        for (int sw = 0; sw < theta; sw++) {
            uint32_t u = (uint32_t)(u0 + sw);
            for (int c = 0; c < 2; c++) {
                for (int y = 0; y < L; y++)
                    for (int x = 0; x < L; x++) {
                        if (((x + y) & 1) != c)
                            continue;
                        uint32_t b = (uint32_t)(y * half + (x >> 1));
                        uint32_t ctr[4] = {2u * u + (uint32_t)c, b >> 1, 6u, k};
                        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
                        uint32_t out[4];
                        oracle_philox4x32_10(ctr, key, out);
                        uint32_t w0 = out[2 * (b & 1u)], w1 = out[2 * (b & 1u) + 1];
                        int si = S[y * L + x];
                        int sp = (int)((si + 1 + (int)potts_state(w0, q - 1)) % q);
                        int nb[4] = {S[y * L + (x + 1) % L], S[y * L + (x + L - 1) % L],
                                     S[((y + 1) % L) * L + x], S[((y + L - 1) % L) * L + x]};
                        int ns = 0, np = 0;
                        for (int j = 0; j < 4; j++) {
                            ns += nb[j] == si;
                            np += nb[j] == sp;
                        }
                        int dE = ns - np;
                        int accept = dE <= 0 || (uint64_t)w1 < T[dE - 1];
                        if (accept)
                            S[y * L + x] = (int8_t)sp;
                    }
            }
        }
    }
}

void oracle_measure_potts(int L, int q, int64_t n, const int8_t *s, int64_t *E, int64_t *M)
{
    const int N = L * L;
    for (int64_t r = 0; r < n; r++) {
        const int8_t *S = s + (size_t)r * N;
        int64_t e = 0;
        int64_t cnt[256] = {0};
        for (int y = 0; y < L; y++)
            for (int x = 0; x < L; x++) {
                int si = S[y * L + x];
                e -= (S[y * L + (x + 1) % L] == si) + (S[((y + 1) % L) * L + x] == si);
                cnt[si]++;
            }
        int64_t mx = 0;
        for (int t = 0; t < q; t++)
            if (cnt[t] > mx)
                mx = cnt[t];
        E[r] = e;
        M[r] = mx;
    }
}
