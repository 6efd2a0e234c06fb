// S = X^T X / n with SIMT fused multiply-adds (Alg. 2 step 2): the FP64 mode and
// the "plain FP32" mode that the tensor-core modes are measured against.
//
// X is n x p row-major, so a K-slab X[k0:k0+BK, i0:i0+BM] is BK contiguous row
// segments: both operands of the tile S[I, J] are loaded coalesced from the same
// matrix.  Only tiles with I <= J run; each writes its tile and the mirror
// S[J, I], so S is bitwise symmetric (the product x_ki x_kj is commutative and
// every entry is one FMA chain over k in the same order).
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.cuh"

namespace hpc {
namespace {

template <typename TX, typename T>
__device__ __forceinline__ T load_as(const TX* p) { return (T)(*p); }
template <>
__device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <>
__device__ __forceinline__ double load_as<__nv_bfloat16, double>(const __nv_bfloat16* p) {
    return (double)__bfloat162float(*p);
}

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }

// 256 threads as 16 x 16; each thread owns a TM x TM micro-tile at rows ty + 16a,
// columns tx + 16b of the BM x BM tile (BM = 16 TM).
template <typename TX, typename T, int TM>
__global__ void __launch_bounds__(256)
k_gram_simt(const TX* __restrict__ X, int64_t n, int64_t p, T* __restrict__ S, int64_t lds, int nb) {
    constexpr int BM = 16 * TM;
    constexpr int BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BM + 1];
    // map the linear block index to an upper-triangular tile (bi <= bj)
    int t = blockIdx.x, bi = 0;
    while (t >= nb - bi) { t -= nb - bi; ++bi; }
    const int bj = bi + t;
    const int64_t i0 = (int64_t)bi * BM, j0 = (int64_t)bj * BM;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);

    for (int64_t k0 = 0; k0 < n; k0 += BK) {
        for (int idx = threadIdx.x; idx < BK * BM; idx += 256) {
            const int kk = idx / BM, ii = idx % BM;
            const int64_t k = k0 + kk;
            const int64_t ia = i0 + ii, ja = j0 + ii;
            As[kk][ii] = (k < n && ia < p) ? load_as<TX, T>(X + k * p + ia) : T(0);
            Bs[kk][ii] = (k < n && ja < p) ? load_as<TX, T>(X + k * p + ja) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TM];
#pragma unroll
            for (int q = 0; q < TM; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
            for (int q = 0; q < TM; ++q)
#pragma unroll
                for (int r = 0; r < TM; ++r) acc[q][r] = fmaT(a[q], b[r], acc[q][r]);
        }
        __syncthreads();
    }
    const T dn = (T)n;
#pragma unroll
    for (int q = 0; q < TM; ++q) {
        const int64_t i = i0 + ty + 16 * q;
        if (i >= p) continue;
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            const int64_t j = j0 + tx + 16 * r;
            if (j >= p) continue;
            const T v = acc[q][r] / dn;
            S[i * lds + j] = v;
            if (bi != bj) S[j * lds + i] = v;
        }
    }
}

// FP32 form for rows of X that start on 16-byte boundaries (p a multiple of 4 and X
// aligned; S likewise for its rows): 128 x 128 tiles, 256 threads as 16 x 16, each
// thread owning an 8 x 8 micro-tile made of rows {4 ty .. 4 ty + 3, 64 + 4 ty .. + 3}
// and the same split of columns around tx, so that the 16-byte operand reads of
// eight consecutive lanes fall on 32 different banks.  K-slabs of 8 rows are
// double-buffered in shared memory: the next slab is loaded into registers (one
// 4-element vector of each operand per thread) while the current one is multiplied,
// one barrier per slab; 4 vector reads per 64 FMAs.  Every entry is still one FMA
// chain over k in ascending order, so S is bitwise symmetric and equals the scalar
// kernel's values.
template <typename TX>
__device__ __forceinline__ float4 load4(const TX* p);
template <>
__device__ __forceinline__ float4 load4<float>(const float* p) { return *reinterpret_cast<const float4*>(p); }
template <>
__device__ __forceinline__ float4 load4<__nv_bfloat16>(const __nv_bfloat16* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
}

template <typename TX>
__global__ void __launch_bounds__(256)
k_gram_simt_v4(const TX* __restrict__ X, int64_t n, int64_t p, float* __restrict__ S, int64_t lds, int nb) {
    constexpr int BM = 128, BK = 8;
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BM];
    int t = blockIdx.x, bi = 0;
    while (t >= nb - bi) { t -= nb - bi; ++bi; }
    const int bj = bi + t;
    const int64_t i0 = (int64_t)bi * BM, j0 = (int64_t)bj * BM;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // slab loader: thread -> (row kk = tid / 32, columns 4 (tid % 32) .. + 3) of each operand
    const int lk = threadIdx.x >> 5, lc = 4 * (threadIdx.x & 31);
    const bool ai = i0 + lc < p, bj_ok = j0 + lc < p;          // p % 4 == 0: a vector is all in or all out
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ra = z4, rb = z4;
    if (lk < n) {
        if (ai) ra = load4<TX>(X + (int64_t)lk * p + i0 + lc);
        if (bj_ok) rb = load4<TX>(X + (int64_t)lk * p + j0 + lc);
    }
    *reinterpret_cast<float4*>(&As[0][lk][lc]) = ra;
    *reinterpret_cast<float4*>(&Bs[0][lk][lc]) = rb;
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = 0; k0 < n; k0 += BK) {
        const int64_t kn = k0 + BK + lk;
        const bool more = k0 + BK < n;
        ra = z4;
        rb = z4;
        if (more && kn < n) {
            if (ai) ra = load4<TX>(X + kn * p + i0 + lc);
            if (bj_ok) rb = load4<TX>(X + kn * p + j0 + lc);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + 4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int r = 0; r < 8; ++r) acc[q][r] = __fmaf_rn(a[q], b[r], acc[q][r]);
        }
        if (more) {
            *reinterpret_cast<float4*>(&As[buf ^ 1][lk][lc]) = ra;
            *reinterpret_cast<float4*>(&Bs[buf ^ 1][lk][lc]) = rb;
        }
        __syncthreads();
        buf ^= 1;
    }
    const float dn = (float)n;
    // rows (columns) q < 4 at 4 ty + q, q >= 4 at 64 + 4 ty + q - 4; p % 4 == 0, so each
    // group of four is all inside or all outside
    const int64_t ia[2] = {i0 + 4 * ty, i0 + 64 + 4 * ty};
    const int64_t ja[2] = {j0 + 4 * tx, j0 + 64 + 4 * tx};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t i = ia[q >> 2] + (q & 3);
        if (i >= p) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (ja[h] < p)
                *reinterpret_cast<float4*>(S + i * lds + ja[h]) =
                    make_float4(acc[q][4 * h] / dn, acc[q][4 * h + 1] / dn, acc[q][4 * h + 2] / dn,
                                acc[q][4 * h + 3] / dn);
        }
    }
    if (bi != bj) {
        // the mirror S[j, i] = S[i, j]: row j of the lower tile gets this thread's column r
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int64_t j = ja[r >> 2] + (r & 3);
            if (j >= p) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (ia[h] < p)
                    *reinterpret_cast<float4*>(S + j * lds + ia[h]) =
                        make_float4(acc[4 * h][r] / dn, acc[4 * h + 1][r] / dn, acc[4 * h + 2][r] / dn,
                                    acc[4 * h + 3][r] / dn);
            }
        }
    }
}

template <typename TX>
cudaError_t run_v4(const void* X, int64_t n, int64_t p, void* S, int64_t lds, cudaStream_t s) {
    const int nb = (int)((p + 127) / 128);
    const long long tiles = (long long)nb * (nb + 1) / 2;
    k_gram_simt_v4<TX><<<(unsigned)tiles, 256, 0, s>>>(static_cast<const TX*>(X), n, p, static_cast<float*>(S), lds,
                                                        nb);
    return cudaGetLastError();
}

template <typename TX, typename T, int TM>
cudaError_t run(const void* X, int64_t n, int64_t p, void* S, int64_t lds, cudaStream_t s) {
    constexpr int BM = 16 * TM;
    const int nb = (int)((p + BM - 1) / BM);
    const long long tiles = (long long)nb * (nb + 1) / 2;
    k_gram_simt<TX, T, TM><<<(unsigned)tiles, 256, 0, s>>>(static_cast<const TX*>(X), n, p, static_cast<T*>(S),
                                                           lds, nb);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gram_simt(const void* X, int xdt, int64_t n, int64_t p, void* S, int sdt, int64_t lds,
                      cudaStream_t s, int* launches) {
    if (launches) *launches += 1;
    if (sdt == HPC_F64) {
        if (xdt == HPC_F64) return run<double, double, 4>(X, n, p, S, lds, s);
        if (xdt == HPC_F32) return run<float, double, 4>(X, n, p, S, lds, s);
        return run<__nv_bfloat16, double, 4>(X, n, p, S, lds, s);
    }
    if (xdt == HPC_F64) return run<double, float, 8>(X, n, p, S, lds, s);
    // the vector form needs 16-byte (8-byte for BF16) aligned rows of X and S
    const bool vec = p % 4 == 0 && lds % 4 == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(X) & (xdt == HPC_F32 ? 15 : 7)) == 0;
    if (xdt == HPC_F32) return vec ? run_v4<float>(X, n, p, S, lds, s) : run<float, float, 8>(X, n, p, S, lds, s);
    return vec ? run_v4<__nv_bfloat16>(X, n, p, S, lds, s) : run<__nv_bfloat16, float, 8>(X, n, p, S, lds, s);
}

}  // namespace hpc
