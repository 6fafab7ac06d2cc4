// Integer-pipe measurement kernels: the issue rates behind the roofline of
// the Metropolis sweep (Philox4x32-10 products and XORs, Sec. 3; the
// accept-bit insert and the LCG of Sec. 4). Not on the simulation path.
#include "pa_internal.cuh"

namespace pa {

// ======================================================== integer pipe peaks
// Eight independent dependency chains per thread of one instruction class,
// operands from kernel arguments so nothing folds at compile time:
//   0: 32x32->64 product by a constant with its halves XORed, as in a Philox
//      round (one wide multiply and one logic op per step);
//   1: three-input logic (lop3) with non-linear tables (xor, majority,
//      select), so no chain collapses to a shorter one;
//   2: 32-bit multiply-add (mad.lo.u32), the accept-bit insert and the LCG.
// The chains are folded into one store per thread.
__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t lop3_maj(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t lop3_sel(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xCA;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <int P>
__global__ void __launch_bounds__(256) k_pipe_peak(long long iters, uint32_t m, uint32_t c, uint32_t* __restrict__ sink)
{
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    if constexpr (P == 0) {
        uint32_t x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = tid * 8u + (unsigned)j + c;
#pragma unroll 4
        for (long long i = 0; i < iters; i++) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                // as in a Philox round: a product by a constant, halves XORed
                const unsigned long long d = (unsigned long long)0xD2511F53u * x[j];
                x[j] = (uint32_t)d ^ (uint32_t)(d >> 32) ^ m;
            }
        }
#pragma unroll
        for (int j = 0; j < 8; j++) acc ^= x[j];
    } else if constexpr (P == 1) {
        uint32_t a[8], b[8], e[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            a[j] = tid + (unsigned)j;
            b[j] = m ^ (unsigned)j;
            e[j] = c + 3u * (unsigned)j;
        }
#pragma unroll 4
        for (long long i = 0; i < iters; i++) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                a[j] = lop3_xor(a[j], b[j], e[j]);
                b[j] = lop3_maj(b[j], e[j], a[j]);
                e[j] = lop3_sel(a[j], b[j], e[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; j++) acc ^= a[j] ^ b[j] ^ e[j];
    } else {
        uint32_t x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = tid * 8u + (unsigned)j;
#pragma unroll 4
        for (long long i = 0; i < iters; i++) {
#pragma unroll
            for (int j = 0; j < 8; j++) asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(m), "r"(c));
        }
#pragma unroll
        for (int j = 0; j < 8; j++) acc ^= x[j];
    }
    sink[tid] = acc;
}

cudaError_t launch_pipe_peak(int pipe, long long iters, uint32_t* sink, int grid, int threads, cudaStream_t s)
{
    const uint32_t m = 0xD2511F53u, c = 0x9E3779B9u;
    switch (pipe) {
    case 0: k_pipe_peak<0><<<grid, threads, 0, s>>>(iters, m, c, sink); break;
    case 1: k_pipe_peak<1><<<grid, threads, 0, s>>>(iters, m, c, sink); break;
    case 2: k_pipe_peak<2><<<grid, threads, 0, s>>>(iters, m, c, sink); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pa
