// S = X^T X / n with SIMT fused multiply-adds (Alg. 2 step 2): the FP64 mode and
// the "plain FP32" mode that the tensor-core modes are measured against.
//
// X is n x p row-major, so a K-slab X[k0:k0+BK, i0:i0+BM] is BK contiguous row
// segments: both operands of the tile S[I, J] are loaded coalesced from the same
// matrix.  Only tiles with I <= J run; each writes its tile and the mirror
// S[J, I], so S is bitwise symmetric (the product x_ki x_kj is commutative and
// every entry is one FMA chain over k in the same order).
#include <cuda_bf16.h>

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
    if (xdt == HPC_F32) return run<float, float, 8>(X, n, p, S, lds, s);
    return run<__nv_bfloat16, float, 8>(X, n, p, S, lds, s);
}

}  // namespace hpc
