// Differentiation of the solver's outputs.
//
//  * Gradients of the smooth loss L(Omega, X) = -sum log w_ii + tr(Omega S Omega)/2
//    + lambda2/2 ||Omega||_F^2, S = X^T X / n, at the (symmetric) iterate:
//      dL/dOmega = -diag(1/w_ii) + (Omega S + S Omega)/2 + lambda2 Omega   (Alg. 1 step 4's G, dense)
//      dL/dX     = X Omega^2 / n = Y Omega / n,  Y = X Omega.
//    Dense W = Omega S comes from a row-split SpMM in the screening pass's
//    canonical FMA order (so G agrees bitwise with the solver's G on its
//    candidates), then an in-place tile-pair symmetrisation and the support
//    terms.  X Omega^2 / n is two row-split SpMMs on X^T.
//  * The implicit lambda-gradient of a held-out loss on the support A: the
//    support-restricted products (E S)_ij by gathers, the Hessian-vector product
//      H[E]_ij = ((E S)_ij + (E S)_ji)/2 + lambda2 E_ij + [i=j] E_ii / w_ii^2,
//    and conjugate gradients in FP64 with fixed-order reductions (the vectors
//    live on the nnz entries of A, so FP64 costs little there).
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace hpc {
namespace {

constexpr int kW = 8;   // warps per block

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mulT(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulT(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

template <typename TI>
__device__ __forceinline__ float to_f(TI v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// C[i, c] = sum_k w_ik B[k, c], canonical order: w_ii B[i, c] first, then the
// off-diagonal k ascending.  Warp per row, lanes over 32 * 4 consecutive columns.
template <typename T>
__global__ void __launch_bounds__(256)
k_spmm_dense(int p, Csr<T> om, const int4* __restrict__ rinfo, const T* __restrict__ rdv, const T* __restrict__ B,
             int64_t ldb, int64_t m, T* __restrict__ C, int64_t ldc) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kW + (threadIdx.x >> 5);
    if (i >= p) return;
    const int64_t c0 = (int64_t)blockIdx.y * 128;
    const int4 info = rinfo[i];
    const T dv = rdv[i];
    T acc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int64_t c = c0 + lane + 32 * v;
        acc[v] = c < m ? mulT(dv, B[(int64_t)i * ldb + c]) : T(0);
    }
    for (int q = info.x; q < info.y; ++q) {
        if (q == info.z) continue;
        const int k = om.ci[q];
        const T w = om.cv[q];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t c = c0 + lane + 32 * v;
            if (c < m) acc[v] = fmaT(w, B[(int64_t)k * ldb + c], acc[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int64_t c = c0 + lane + 32 * v;
        if (c < m) C[(int64_t)i * ldc + c] = acc[v];
    }
}

// In place, per pair of 32 x 32 tiles (I <= J): A_ij <- (A_ij + A_ji) / 2 on both sides.
template <typename T>
__global__ void __launch_bounds__(256) k_symmetrize(T* __restrict__ A, int64_t lda, int p, int nt) {
    __shared__ T a[32][33];
    __shared__ T b[32][33];
    int t = blockIdx.x, bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    const int bj = bi + t;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int y = ty; y < 32; y += 8) {
        const int i = bi * 32 + y, j = bj * 32 + tx;
        a[y][tx] = (i < p && j < p) ? A[(int64_t)i * lda + j] : T(0);
        const int i2 = bj * 32 + y, j2 = bi * 32 + tx;
        b[y][tx] = (i2 < p && j2 < p) ? A[(int64_t)i2 * lda + j2] : T(0);
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int i = bi * 32 + y, j = bj * 32 + tx;
        if (i < p && j < p) A[(int64_t)i * lda + j] = T(0.5) * (a[y][tx] + b[tx][y]);
        const int i2 = bj * 32 + y, j2 = bi * 32 + tx;
        if (i2 < p && j2 < p) A[(int64_t)i2 * lda + j2] = T(0.5) * (b[y][tx] + a[tx][y]);
    }
}

// Support terms of G: A_ij <- fma(lambda2, w_ij, A_ij) - [i=j] / w_ii (the solver's rounding sequence).
template <typename T>
__global__ void k_support_terms(int p, Csr<T> om, T* __restrict__ A, int64_t lda, T lam2) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kW + (threadIdx.x >> 5);
    if (i >= p) return;
    for (int q = om.rp[i] + lane; q < om.rp[i + 1]; q += 32) {
        const int j = om.ci[q];
        const T w = om.cv[q];
        T g = fmaT(lam2, w, A[(int64_t)i * lda + j]);
        if (j == i) g -= T(1) / w;
        A[(int64_t)i * lda + j] = g;
    }
}

template <typename T>
__global__ void k_scale(T* __restrict__ A, int64_t rows, int64_t cols, int64_t lda, T s) {
    const int64_t n = rows * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, c = t % cols;
        A[r * lda + c] *= s;
    }
}

// out[c][r] = in[r][c] * scale, 32 x 32 shared-memory tiles.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256)
k_transpose(const TI* __restrict__ in, int64_t rows, int64_t cols, int64_t ldi, TO* __restrict__ out, int64_t ldo,
            float scale) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int y = ty; y < 32; y += 8) {
        const int64_t r = r0 + y, c = c0 + tx;
        tile[y][tx] = (r < rows && c < cols) ? to_f<TI>(in[r * ldi + c]) : 0.f;
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int64_t c = c0 + y, r = r0 + tx;
        if (c < cols && r < rows) out[c * ldo + r] = (TO)(tile[tx][y] * scale);
    }
}

// tr[e] = position of entry (j, i) for entry e = (i, j) of a symmetric CSR (-1 if absent).
template <typename T>
__global__ void k_transpose_index(int p, Csr<T> om, int* __restrict__ tr) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kW + (threadIdx.x >> 5);
    if (i >= p) return;
    for (int e = om.rp[i] + lane; e < om.rp[i + 1]; e += 32) {
        const int j = om.ci[e];
        int lo = om.rp[j], hi = om.rp[j + 1] - 1, pos = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int c = om.ci[mid];
            if (c == i) { pos = mid; break; }
            if (c < i) lo = mid + 1; else hi = mid - 1;
        }
        tr[e] = pos;
    }
}

// T_e = sum_{q in row i} v_q S[ci[q], j_e] for every support entry e = (i, j_e), FP64,
// diagonal term first then off-diagonals ascending.
template <typename T>
__global__ void k_support_product(int p, Csr<T> om, const int4* __restrict__ rinfo, const double* __restrict__ v,
                                  const T* __restrict__ S, int64_t lds, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kW + (threadIdx.x >> 5);
    if (i >= p) return;
    const int4 info = rinfo[i];
    for (int e = info.x + lane; e < info.y; e += 32) {
        const int j = om.ci[e];
        double acc = info.z >= 0 ? v[info.z] * (double)S[(int64_t)i * lds + j] : 0.0;
        for (int q = info.x; q < info.y; ++q)
            if (q != info.z) acc = fma(v[q], (double)S[(int64_t)om.ci[q] * lds + j], acc);
        out[e] = acc;
    }
}

// Hessian-vector product on the support and the held-out gradient:
//   mode 0 (HVP):      out_e = (T_e + T_tr(e))/2 + lambda2 v_e + [diag] v_e / w_ii^2
//   mode 1 (gradient): out_e = (T_e + T_tr(e))/2 - [diag] / w_ii
template <typename T>
__global__ void k_support_combine(int p, Csr<T> om, const int* __restrict__ tr, const double* __restrict__ Tv,
                                  const double* __restrict__ v, double lam2, int mode, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kW + (threadIdx.x >> 5);
    if (i >= p) return;
    for (int e = om.rp[i] + lane; e < om.rp[i + 1]; e += 32) {
        const int j = om.ci[e];
        const double w = (double)om.cv[e];
        const int te = tr[e] >= 0 ? tr[e] : e;     // a symmetric pattern always has (j, i)
        double o = 0.5 * (Tv[e] + Tv[te]);
        if (mode == 0) {
            o += lam2 * v[e];
            if (j == i) o += v[e] / (w * w);
        } else if (j == i) {
            o -= 1.0 / w;
        }
        out[e] = o;
    }
}

// ---------------------------------------------------------------- CG (FP64, on the nnz entries)
struct CgState {
    double rr, rr0, pap, alpha, beta;
    int done;
    int pad;
};

// block partials of <a, b> (fixed grid-stride order)
__global__ void __launch_bounds__(256) k_dot_part(int64_t n, const double* a, const double* b, double* part) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[t], b[t], s);
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < 8; ++w) r += red[w];
        part[blockIdx.x] = r;
    }
}

__device__ double reduce_parts(const double* part, int nb) {
    __shared__ double red[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
    return r;
}

// stage 0: rr = rr0 = <r, r> (initial); stage 1: alpha = rr / <p, Ap>; stage 2: beta = rr_new / rr, done test
__global__ void __launch_bounds__(256) k_cg_scalar(const double* part, int nb, int stage, double tol2, CgState* cg) {
    const double v = reduce_parts(part, nb);
    if (threadIdx.x != 0) return;
    if (stage == 0) {
        cg->rr = v;
        cg->rr0 = v;
        cg->done = (v == 0.0) ? 1 : 0;
    } else if (stage == 1) {
        cg->pap = v;
        cg->alpha = (v > 0.0) ? cg->rr / v : 0.0;
        if (!(v > 0.0)) cg->done = 2;      // H not positive definite along p: stop
    } else {
        cg->beta = (cg->rr > 0.0) ? v / cg->rr : 0.0;
        cg->rr = v;
        if (v <= tol2 * cg->rr0) cg->done = 1;
    }
}

// x += alpha p; r -= alpha Ap
__global__ void k_cg_xr(int64_t n, const CgState* cg, const double* p, const double* Ap, double* x, double* r) {
    if (cg->done) return;
    const double a = cg->alpha;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        x[t] = fma(a, p[t], x[t]);
        r[t] = fma(-a, Ap[t], r[t]);
    }
}

// p = r + beta p
__global__ void k_cg_p(int64_t n, const CgState* cg, const double* r, double* p) {
    if (cg->done) return;
    const double b = cg->beta;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        p[t] = fma(b, p[t], r[t]);
}

// FP64 copy of the support values.
template <typename T>
__global__ void k_support_values(int64_t nnz, const T* __restrict__ cv, double* __restrict__ omega_d) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        omega_d[e] = (double)cv[e];
}

// sign(w_ij) off the diagonal, 0 on it.
template <typename T>
__global__ void k_sign_off(int p, Csr<T> om, double* sign_off) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kW + (threadIdx.x >> 5);
    if (i >= p) return;
    for (int e = om.rp[i] + lane; e < om.rp[i + 1]; e += 32) {
        const double w = (double)om.cv[e];
        sign_off[e] = (om.ci[e] == i) ? 0.0 : (w > 0.0 ? 1.0 : (w < 0.0 ? -1.0 : 0.0));
    }
}

// Partials of the smooth part at the iterate: [0] sum_e w_e T_e (= tr(Omega S Omega) with
// T = (Omega S) on the support), [1] ||Omega||_F^2, [2] sum_i log w_ii.
template <typename T>
__global__ void __launch_bounds__(256) k_smooth_parts(int p, Csr<T> om, const double* __restrict__ Tv, double* part) {
    __shared__ double red[8][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = blockIdx.x * kW + warp; i < p; i += gridDim.x * kW) {
        for (int e = om.rp[i] + lane; e < om.rp[i + 1]; e += 32) {
            const double w = (double)om.cv[e];
            a = fma(w, Tv[e], a);
            b = fma(w, w, b);
            if (om.ci[e] == i) c += log(w);
        }
    }
    a = warp_sum_d(a); b = warp_sum_d(b); c = warp_sum_d(c);
    if (lane == 0) { red[warp][0] = a; red[warp][1] = b; red[warp][2] = c; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double r = 0.0;
        for (int w = 0; w < 8; ++w) r += red[w][threadIdx.x];
        part[blockIdx.x * 3 + threadIdx.x] = r;
    }
}

// out[k] = sum_b part[b * stride + k] for k < stride, in a fixed order.
__global__ void __launch_bounds__(256) k_reduce_strided(const double* part, int nb, int stride, double* out) {
    for (int k = 0; k < stride; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)b * stride + k];
        s = warp_sum_d(s);
        __shared__ double red[8];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
            for (int w = 0; w < 8; ++w) r += red[w];
            out[k] = r;
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
int launch_smooth_parts(int p, Csr<T> om, const double* Tv, double* part, double* out3, cudaStream_t s) {
    const int nb = std::min((p + kW - 1) / kW, 1024);
    k_smooth_parts<T><<<nb, 256, 0, s>>>(p, om, Tv, part);
    k_reduce_strided<<<1, 256, 0, s>>>(part, nb, 3, out3);
    return nb;
}

void launch_reduce_parts(const double* part, int nb, double* out, cudaStream_t s) {
    k_reduce_strided<<<1, 256, 0, s>>>(part, nb, 1, out);
}

template <typename T>
void launch_dense_grad(int p, Csr<T> om, const int4* rinfo, const T* rdv, const T* S, int64_t lds, T* G,
                       int64_t ldg, T lam2, T scale, cudaStream_t s) {
    dim3 g1((p + kW - 1) / kW, (unsigned)((p + 127) / 128));
    k_spmm_dense<T><<<g1, 256, 0, s>>>(p, om, rinfo, rdv, S, lds, p, G, ldg);
    const int nt = (p + 31) / 32;
    k_symmetrize<T><<<(unsigned)((int64_t)nt * (nt + 1) / 2), 256, 0, s>>>(G, ldg, p, nt);
    k_support_terms<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, G, ldg, lam2);
    if (scale != T(1)) k_scale<T><<<1024, 256, 0, s>>>(G, p, p, ldg, scale);
}

template <typename T>
void launch_spmm_dense(int p, Csr<T> om, const int4* rinfo, const T* rdv, const T* B, int64_t ldb, int64_t m,
                       T* C, int64_t ldc, cudaStream_t s) {
    dim3 g((p + kW - 1) / kW, (unsigned)((m + 127) / 128));
    k_spmm_dense<T><<<g, 256, 0, s>>>(p, om, rinfo, rdv, B, ldb, m, C, ldc);
}

void launch_transpose(const void* in, int in_dt, int64_t rows, int64_t cols, int64_t ldi, void* out, int out_dt,
                      int64_t ldo, float scale, cudaStream_t s) {
    dim3 g((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    if (in_dt == HPC_BF16) {
        k_transpose<__nv_bfloat16, float><<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(in), rows, cols, ldi,
                                                             static_cast<float*>(out), ldo, scale);
    } else if (in_dt == HPC_F64 && out_dt == HPC_F64) {
        k_transpose<double, double><<<g, 256, 0, s>>>(static_cast<const double*>(in), rows, cols, ldi,
                                                       static_cast<double*>(out), ldo, scale);
    } else if (in_dt == HPC_F64) {
        k_transpose<double, float><<<g, 256, 0, s>>>(static_cast<const double*>(in), rows, cols, ldi,
                                                      static_cast<float*>(out), ldo, scale);
    } else if (out_dt == HPC_F64) {
        k_transpose<float, double><<<g, 256, 0, s>>>(static_cast<const float*>(in), rows, cols, ldi,
                                                      static_cast<double*>(out), ldo, scale);
    } else {
        k_transpose<float, float><<<g, 256, 0, s>>>(static_cast<const float*>(in), rows, cols, ldi,
                                                     static_cast<float*>(out), ldo, scale);
    }
}

template <typename T>
void launch_transpose_index(int p, Csr<T> om, int* tr, cudaStream_t s) {
    k_transpose_index<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, tr);
}

template <typename T>
void launch_support_product(int p, Csr<T> om, const int4* rinfo, const double* v, const T* S, int64_t lds,
                            double* out, cudaStream_t s) {
    k_support_product<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, rinfo, v, S, lds, out);
}

template <typename T>
void launch_support_combine(int p, Csr<T> om, const int* tr, const double* Tv, const double* v, double lam2,
                            int mode, double* out, cudaStream_t s) {
    k_support_combine<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, tr, Tv, v, lam2, mode, out);
}

template <typename T>
void launch_support_vectors(int p, int64_t nnz, Csr<T> om, double* omega_d, double* sign_off, cudaStream_t s) {
    k_support_values<T><<<256, 256, 0, s>>>(nnz, om.cv, omega_d);
    k_sign_off<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, sign_off);
}

int cg_part_blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 1024); }

void launch_dot_part(int64_t n, const double* a, const double* b, double* part, cudaStream_t s) {
    k_dot_part<<<cg_part_blocks(n), 256, 0, s>>>(n, a, b, part);
}

void launch_cg_scalar(const double* part, int nb, int stage, double tol2, void* cg, cudaStream_t s) {
    k_cg_scalar<<<1, 256, 0, s>>>(part, nb, stage, tol2, static_cast<CgState*>(cg));
}

void launch_cg_xr(int64_t n, const void* cg, const double* p, const double* Ap, double* x, double* r,
                  cudaStream_t s) {
    k_cg_xr<<<cg_part_blocks(n), 256, 0, s>>>(n, static_cast<const CgState*>(cg), p, Ap, x, r);
}

void launch_cg_p(int64_t n, const void* cg, const double* r, double* p, cudaStream_t s) {
    k_cg_p<<<cg_part_blocks(n), 256, 0, s>>>(n, static_cast<const CgState*>(cg), r, p);
}

size_t cg_state_bytes() { return sizeof(CgState); }

#define HPC_ADJ_INSTANTIATE(T)                                                                                  \
    template void launch_dense_grad<T>(int, Csr<T>, const int4*, const T*, const T*, int64_t, T*, int64_t, T, T, \
                                       cudaStream_t);                                                           \
    template void launch_spmm_dense<T>(int, Csr<T>, const int4*, const T*, const T*, int64_t, int64_t, T*,      \
                                       int64_t, cudaStream_t);                                                  \
    template void launch_transpose_index<T>(int, Csr<T>, int*, cudaStream_t);                                   \
    template void launch_support_product<T>(int, Csr<T>, const int4*, const double*, const T*, int64_t, double*, \
                                            cudaStream_t);                                                      \
    template void launch_support_combine<T>(int, Csr<T>, const int*, const double*, const double*, double, int, \
                                            double*, cudaStream_t);                                             \
    template void launch_support_vectors<T>(int, int64_t, Csr<T>, double*, double*, cudaStream_t);          \
    template int launch_smooth_parts<T>(int, Csr<T>, const double*, double*, double*, cudaStream_t);

HPC_ADJ_INSTANTIATE(float)
HPC_ADJ_INSTANTIATE(double)

}  // namespace hpc
