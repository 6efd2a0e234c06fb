// Differentiation of the solver's outputs.
//
//  * Gradients of the smooth loss L(Omega, X) = -sum log w_ii + tr(Omega S Omega)/2
//    + lambda2/2 ||Omega||_F^2, S = X^T X / n, at the (symmetric) iterate:
//      dL/dOmega = -diag(1/w_ii) + (Omega S + S Omega)/2 + lambda2 Omega   (Alg. 1 step 4's G, dense)
//      dL/dX     = X Omega^2 / n = Y Omega / n,  Y = X Omega.
//    dL/dOmega is one kernel over pairs of tiles (I <= J): W[I, J] and W[J, I] in
//    the screening pass's canonical FMA order (so G agrees bitwise with the solver's
//    G on its candidates), symmetrised, with the support terms, written once.
//    X Omega^2 / n is two row-split SpMMs on X^T, the second writing its result
//    transposed.
//  * The implicit lambda-gradient of a held-out loss on the support A: the
//    support-restricted products (E S)_ij by gathers, the Hessian-vector product
//      H[E]_ij = ((E S)_ij + (E S)_ji)/2 + lambda2 E_ij + [i=j] E_ii / w_ii^2,
//    and conjugate gradients in FP64 with fixed-order reductions (the vectors
//    live on the nnz entries of A, so FP64 costs little there).  The held-out
//    loss's gradient needs (Omega S_val)_ij on A only: a row-split SpMM
//    Y^T = Omega X_val^T and one dot product of rows of Y^T and X_val^T per entry,
//    so S_val (p x p) is never formed.
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

template <typename TO, typename TI>
__device__ __forceinline__ TO to_t(TI v) { return (TO)v; }
template <>
__device__ __forceinline__ float to_t<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ double to_t<double, __nv_bfloat16>(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
}

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

// C^T scaled: C = Omega B as in k_spmm_dense (same order per element), for a tile of 32
// rows i x 128 columns c staged in shared memory, then written as Ct[c, i] = scale C[i, c]
// (Ct m x p, row pitch ldt), so a transpose never re-reads C.
template <typename T>
__global__ void __launch_bounds__(256)
k_spmm_dense_t(int p, Csr<T> om, const int4* __restrict__ rinfo, const T* __restrict__ rdv, const T* __restrict__ B,
               int64_t ldb, int64_t m, T* __restrict__ Ct, int64_t ldt, T scale) {
    __shared__ T tile[32][129];
    const int lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * 32;
    const int64_t c0 = (int64_t)blockIdx.y * 128;
    for (int y = threadIdx.x >> 5; y < 32; y += kW) {
        const int i = i0 + y;
        T acc[4] = {T(0), T(0), T(0), T(0)};
        if (i < p) {
            const int4 info = rinfo[i];
            const T dv = rdv[i];
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
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) tile[y][lane + 32 * v] = acc[v];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * 128; idx += 256) {
        const int cl = idx >> 5, il = idx & 31;
        const int64_t c = c0 + cl;
        if (c < m && i0 + il < p) Ct[c * ldt + i0 + il] = tile[il][cl] * scale;
    }
}

// The off-diagonal terms of row i of W = Omega S on the columns c0 .. c0 + TL - 1, added to
// w (which holds w_ii S_ic) in k_spmm_dense's order: k ascending, the diagonal skipped.
// One warp; the row's (k, w_ik) come in 32 at a time, one per lane, broadcast by
// shuffles; S[k, c] is gathered from global memory.
template <typename T, int TL>
__device__ __forceinline__ void offdiag_row(int p, const Csr<T>& om, int4 info, const T* __restrict__ S, int64_t lds,
                                            int c0, T* w) {
    constexpr int V = TL / 32;
    const int lane = threadIdx.x & 31;
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = w[lane + 32 * v];
    for (int q0 = info.x; q0 < info.y; q0 += 32) {
        const int ql = q0 + lane;
        const int kl = ql < info.y ? om.ci[ql] : 0;
        const T wl = ql < info.y ? om.cv[ql] : T(0);
        const int cnt = min(32, info.y - q0);
#pragma unroll 4
        for (int t = 0; t < cnt; ++t) {
            const int k = __shfl_sync(kFull, kl, t);
            const T wk = __shfl_sync(kFull, wl, t);
            if (q0 + t == info.z) continue;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int c = c0 + lane + 32 * v;
                if (c < p) acc[v] = fmaT(wk, S[(int64_t)k * lds + c], acc[v]);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) w[lane + 32 * v] = acc[v];
}

// The support terms of G in row i on the columns c0 .. c0 + TL - 1 (one warp):
// g_ij <- fma(lambda2, w_ij, g_ij) - [i=j] / w_ii.
template <typename T, int TL>
__device__ __forceinline__ void support_terms_row(const Csr<T>& om, int i, int c0, T lam2, T* g) {
    const int lane = threadIdx.x & 31;
    for (int q = om.rp[i] + lane; q < om.rp[i + 1]; q += 32) {
        const int j = om.ci[q];
        if (j < c0 || j >= c0 + TL) continue;
        const T wv = om.cv[q];
        T v = fmaT(lam2, wv, g[j - c0]);
        if (j == i) v -= T(1) / wv;
        g[j - c0] = v;
    }
}

// 16 bytes of T for one vector store
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static __device__ __forceinline__ float4 make(const float* v) { return make_float4(v[0], v[1], v[2], v[3]); }
    static __device__ __forceinline__ void unpack(const float4& u, float* v) {
        v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
    }
};
template <> struct Vec16<double> {
    using type = double2;
    static __device__ __forceinline__ double2 make(const double* v) { return make_double2(v[0], v[1]); }
    static __device__ __forceinline__ void unpack(const double2& u, double* v) { v[0] = u.x; v[1] = u.y; }
};

// Row and column block (bi <= bj) of the t-th tile pair, pairs numbered row by row
// (row bi holds nt - bi pairs): bi from the quadratic's root in FP32, then corrected
// by exact integer steps.
__device__ __forceinline__ void pair_of(long long t, int nt, int& bi, int& bj) {
    const float b2 = 2.0f * (float)nt + 1.0f;
    int r = (int)((b2 - sqrtf(fmaxf(b2 * b2 - 8.0f * (float)t, 0.0f))) * 0.5f);
    r = max(0, min(r, nt - 1));
    auto start = [&](long long q) { return q * nt - q * (q - 1) / 2; };
    while (r > 0 && start(r) > t) --r;
    while (r + 1 < nt && start(r + 1) <= t) ++r;
    bi = r;
    bj = r + (int)(t - start(r));
}

// dL/dOmega = scale ((W + W^T)/2 + lambda2 Omega - diag(1/w_ii)), W = Omega S, on one pair
// of TL x TL tiles (I <= J) per CTA, so G is written once and never re-read:
//  1. the tile S[I, J] is read once; it gives the diagonal terms of both W[I, J]
//     (w_ii S_ij) and W[J, I] (w_jj S_ji = w_jj S_ij: S is bitwise symmetric);
//  2. only the rows with off-diagonal entries (few: the iterate is sparse) add their
//     gathered terms, one warp per row;
//  3. G[I, J] = (W[I, J] + W[J, I]^T)/2, G[J, I] its transpose, then the support
//     terms of the same rows, the scale, and 16-byte stores.
// The rounding sequence per element is the solver's (W in the canonical order,
// 0.5 (W_ij + W_ji), the support terms, the scale).
template <typename T, int TL>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 3)
k_dense_grad_pair(int p, Csr<T> om, const int4* __restrict__ rinfo, const T* __restrict__ rdv,
                  const T* __restrict__ S, int64_t lds, T* __restrict__ G, int64_t ldg, T lam2, T scale, int nt,
                  int vec /* bit 0: 16-byte G stores; bit 1: 16-byte S loads */) {
    __shared__ T a[TL][TL + 1];      // W[I, J], then G[I, J]
    __shared__ T b[TL][TL + 1];      // W[J, I], then G[J, I]
    __shared__ T dvs[2][TL];         // w_ii of the rows of I and of J
    __shared__ int imp[2][TL];       // rows of I and of J with off-diagonal entries
    __shared__ int nimp[2];
    constexpr int E = TL * TL / 256;
    int bi, bj;
    pair_of(blockIdx.x, nt, bi, bj);
    const int I0 = bi * TL, J0 = bj * TL;
    const bool dtile = bi == bj;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 2) nimp[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x < 2 * TL) {
        const int side = threadIdx.x / TL, yl = threadIdx.x % TL;
        const int i = (side ? J0 : I0) + yl;
        T dv = T(0);
        bool impure = false;
        if (i < p) {
            dv = rdv[i];
            impure = rinfo[i].w == 0;
        }
        dvs[side][yl] = dv;
        if (impure) imp[side][atomicAdd(&nimp[side], 1)] = yl;
    }
    __syncthreads();
    // 1. diagonal terms of both tiles from one read of S[I, J]
    constexpr int VW = 16 / (int)sizeof(T), PR = TL / VW, EV = TL * PR / 256;   // 16-byte vectors
    using V16 = Vec16<T>;
    const bool full = I0 + TL <= p && J0 + TL <= p;
    if ((vec & 2) && full) {
        typename V16::type u[EV];
#pragma unroll
        for (int e = 0; e < EV; ++e) {           // all the tile's loads in flight before any use
            const int idx = threadIdx.x + 256 * e, y = idx / PR, x = (idx % PR) * VW;
            u[e] = *reinterpret_cast<const typename V16::type*>(S + (int64_t)(I0 + y) * lds + J0 + x);
        }
#pragma unroll
        for (int e = 0; e < EV; ++e) {
            const int idx = threadIdx.x + 256 * e, y = idx / PR, x = (idx % PR) * VW;
            T sv[VW];
            V16::unpack(u[e], sv);
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                a[y][x + k] = mulT(dvs[0][y], sv[k]);
                b[x + k][y] = mulT(dvs[1][x + k], sv[k]);
            }
        }
    } else {
#pragma unroll 4
        for (int e = 0; e < E; ++e) {
            const int idx = threadIdx.x + 256 * e, y = idx / TL, x = idx % TL;
            const T sv = (I0 + y < p && J0 + x < p) ? S[(int64_t)(I0 + y) * lds + J0 + x] : T(0);
            a[y][x] = mulT(dvs[0][y], sv);
            b[x][y] = mulT(dvs[1][x], sv);
        }
    }
    __syncthreads();
    // 2. off-diagonal terms of the rows that have them
    const int n0 = nimp[0], n1 = nimp[1];
    for (int r = warp; r < n0 + n1; r += kW) {
        const int side = r < n0 ? 0 : 1;
        const int yl = side ? imp[1][r - n0] : imp[0][r];
        const int i = (side ? J0 : I0) + yl;
        offdiag_row<T, TL>(p, om, rinfo[i], S, lds, side ? I0 : J0, side ? &b[yl][0] : &a[yl][0]);
    }
    __syncthreads();
    // 3. symmetrise: G[I, J] in place; G[J, I] is its transpose (a + b = b + a)
#pragma unroll 4
    for (int e = 0; e < E; ++e) {
        const int idx = threadIdx.x + 256 * e, y = idx / TL, x = idx % TL;
        a[y][x] = T(0.5) * (a[y][x] + b[x][y]);
    }
    __syncthreads();
    if (!dtile) {
#pragma unroll 4
        for (int e = 0; e < E; ++e) {
            const int idx = threadIdx.x + 256 * e, y = idx / TL, x = idx % TL;
            b[y][x] = a[x][y];
        }
        __syncthreads();
        for (int r = warp; r < n0 + n1; r += kW) {
            const int side = r < n0 ? 0 : 1;
            const int yl = side ? imp[1][r - n0] : imp[0][r];
            support_terms_row<T, TL>(om, (side ? J0 : I0) + yl, side ? I0 : J0, lam2, side ? &b[yl][0] : &a[yl][0]);
        }
    } else {
        // the diagonal tile: every row has its diagonal entry here
        for (int y = warp; y < TL && I0 + y < p; y += kW) support_terms_row<T, TL>(om, I0 + y, I0, lam2, &a[y][0]);
    }
    __syncthreads();
    const bool scaled = scale != T(1);
    if ((vec & 1) && full) {
        for (int idx = threadIdx.x; idx < TL * PR; idx += 256) {
            const int y = idx / PR, x = (idx % PR) * VW;
            T va[VW], vb[VW];
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                va[k] = scaled ? a[y][x + k] * scale : a[y][x + k];
                vb[k] = scaled ? b[y][x + k] * scale : b[y][x + k];
            }
            *reinterpret_cast<typename V16::type*>(G + (int64_t)(I0 + y) * ldg + J0 + x) = V16::make(va);
            if (!dtile) *reinterpret_cast<typename V16::type*>(G + (int64_t)(J0 + y) * ldg + I0 + x) = V16::make(vb);
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = threadIdx.x + 256 * e, y = idx / TL, x = idx % TL;
            if (I0 + y < p && J0 + x < p) {
                const T v = a[y][x];
                G[(int64_t)(I0 + y) * ldg + J0 + x] = scaled ? v * scale : v;
            }
            if (!dtile && J0 + y < p && I0 + x < p) {
                const T v = b[y][x];
                G[(int64_t)(J0 + y) * ldg + I0 + x] = scaled ? v * scale : v;
            }
        }
    }
}

// out[c][r] = in[r][c] * scale, 32 x 32 shared-memory tiles held in the output type
// (an FP64 transpose stays FP64).
template <typename TI, typename TO>
__global__ void __launch_bounds__(256)
k_transpose(const TI* __restrict__ in, int64_t rows, int64_t cols, int64_t ldi, TO* __restrict__ out, int64_t ldo,
            double scale) {
    __shared__ TO tile[32][33];
    const TO sc = (TO)scale;
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int y = ty; y < 32; y += 8) {
        const int64_t r = r0 + y, c = c0 + tx;
        tile[y][tx] = (r < rows && c < cols) ? to_t<TO>(in[r * ldi + c]) : TO(0);
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int64_t c = c0 + y, r = r0 + tx;
        if (c < cols && r < rows) out[c * ldo + r] = tile[tx][y] * sc;
    }
}

// tr[e] = position of entry (j, i) for entry e = (i, j) of a symmetric CSR (-1 if absent),
// and row[e] = i.
template <typename T>
__global__ void k_transpose_index(int p, Csr<T> om, int* __restrict__ tr, int* __restrict__ row) {
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
        row[e] = i;
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

// T_e = (1/n) sum_m Y^T[i, m] X^T[j_e, m] for every support entry e = (i, j_e), where
// Y^T = Omega X^T: the support-restricted (Omega S)_ij with S = X^T X / n, without S.
// Warp per row of the support; lanes stride m (coalesced rows of X^T and Y^T), four
// independent partials per lane in T, combined and summed across lanes in FP64.
template <typename T>
__global__ void __launch_bounds__(256)
k_support_sddmm(int p, Csr<T> om, const T* __restrict__ yt, const T* __restrict__ xt, int64_t ld, int64_t n,
                double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kW + (threadIdx.x >> 5);
    if (i >= p) return;
    const T* yi = yt + (int64_t)i * ld;
    const int e1 = om.rp[i + 1];
    for (int e = om.rp[i]; e < e1; ++e) {
        const T* xj = xt + (int64_t)om.ci[e] * ld;
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int64_t m = lane;
        for (; m + 96 < n; m += 128) {
            a0 = fmaT(yi[m], xj[m], a0);
            a1 = fmaT(yi[m + 32], xj[m + 32], a1);
            a2 = fmaT(yi[m + 64], xj[m + 64], a2);
            a3 = fmaT(yi[m + 96], xj[m + 96], a3);
        }
        for (; m < n; m += 32) a0 = fmaT(yi[m], xj[m], a0);
        const double v = warp_sum_d(((double)a0 + (double)a1) + ((double)a2 + (double)a3));
        if (lane == 0) out[e] = v / (double)n;
    }
}

// ---------------------------------------------------------------- CG (FP64, on the nnz entries)
struct CgState {
    double rr, rr0, pap, alpha, beta;
    int done;
    unsigned ticket;      // blocks of the running fused reduction that have stored their partial
};

// stage 0: rr = rr0 = <r, r> (initial); stage 1: alpha = rr / <p, Ap>; stage 2: beta = rr_new / rr, done test.
// The stop flag is set once: iterations that run on after a stop (up to the host's next
// check) leave x and r alone and must not turn "converged" into "non-positive
// curvature" (b = 0 gives p = 0) or the reverse.
__device__ void cg_update(int stage, double v, double tol2, CgState* cg) {
    if (stage == 0) {
        cg->rr = v;
        cg->rr0 = v;
        cg->beta = 0.0;                    // the first direction is r itself
        cg->done = (v == 0.0) ? 1 : 0;
    } else if (stage == 1) {
        cg->pap = v;
        cg->alpha = (v > 0.0) ? cg->rr / v : 0.0;
        if (!(v > 0.0) && cg->done == 0) cg->done = 2;      // H not positive definite along p: stop
    } else {
        cg->beta = (cg->rr > 0.0) ? v / cg->rr : 0.0;
        cg->rr = v;
        if (cg->done == 0 && v <= tol2 * cg->rr0) cg->done = 1;
    }
}

// sum_b part[b] in a fixed order (per thread strided over b, then the warp, then the warps)
__device__ double reduce_parts(const double* part, int nb) {
    __shared__ double red[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(part + b);
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
    return r;
}

// This block's partial s (256 threads) into part[blockIdx.x]; the last block of the grid
// to store its partial reduces them all and applies CG stage `stage`.  No block waits:
// the ticket counts the stores, and the block that draws the last ticket does the rest.
__device__ void partial_then_scalar(double s, double* part, int stage, double tol2, CgState* cg) {
    __shared__ double red[8];
    __shared__ int last;
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < 8; ++w) r += red[w];
        part[blockIdx.x] = r;
        __threadfence();
        last = atomicAdd(&cg->ticket, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double v = reduce_parts(part, (int)gridDim.x);
    if (threadIdx.x == 0) {
        cg_update(stage, v, tol2, cg);
        cg->ticket = 0u;
    }
}

// The CG direction and its S gathers, one thread per support entry e = (i, j):
//   p_q = r_q + beta p_old_q (p_old_q once CG has stopped) for the entries q of row i,
//   formed by each thread that needs them; entry e's thread stores p_e;
//   T_e = sum_{q in row i} p_q S[ci[q], j], the diagonal term first, then the
//   off-diagonal q ascending (k_support_product's order).
template <typename T>
__global__ void __launch_bounds__(256)
k_support_product_p(int64_t nnz, const int* __restrict__ row, Csr<T> om, const int4* __restrict__ rinfo,
                    const double* __restrict__ r, const double* __restrict__ p_old, double* __restrict__ p_new,
                    const CgState* cg, const T* __restrict__ S, int64_t lds, double* __restrict__ out) {
    const bool live = cg->done == 0;
    const double beta = cg->beta;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = row[e], j = om.ci[e];
        const int4 info = rinfo[i];
        double acc = 0.0;
        if (info.z >= 0) {
            const double pz = live ? fma(beta, p_old[info.z], r[info.z]) : p_old[info.z];
            acc = pz * (double)S[(int64_t)i * lds + j];
        }
        for (int q = info.x; q < info.y; ++q) {
            if (q == info.z) continue;
            const double pq = live ? fma(beta, p_old[q], r[q]) : p_old[q];
            acc = fma(pq, (double)S[(int64_t)om.ci[q] * lds + j], acc);
        }
        out[e] = acc;
        p_new[e] = live ? fma(beta, p_old[e], r[e]) : p_old[e];
    }
}

// Hessian-vector product on the support and the held-out gradient, one thread per entry
// e = (i, j):
//   mode 0 (HVP):      out_e = (T_e + T_tr(e))/2 + lambda2 v_e + [i=j] v_e / w_ii^2,
//                      then CG stage 1 on <v, out> (when part is given);
//   mode 1 (gradient): out_e = (T_e + T_tr(e))/2 - [i=j] / w_ii.
template <typename T>
__global__ void __launch_bounds__(256)
k_support_combine(int64_t nnz, const int* __restrict__ row, const int* __restrict__ ci, const T* __restrict__ cv,
                  const int* __restrict__ tr, const double* __restrict__ Tv, const double* __restrict__ v, double lam2,
                  int mode, double* __restrict__ out, double* part, double tol2, CgState* cg) {
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int te = tr[e] >= 0 ? tr[e] : (int)e;     // a symmetric pattern always has (j, i)
        const double w = (double)cv[e];
        const bool dg = ci[e] == row[e];
        double o = 0.5 * (Tv[e] + Tv[te]);
        if (mode == 0) {
            o += lam2 * v[e];
            if (dg) o += v[e] / (w * w);
        } else if (dg) {
            o -= 1.0 / w;
        }
        out[e] = o;
        s = fma(v[e], o, s);
    }
    if (part) partial_then_scalar(s, part, 1, tol2, cg);
}

// dL/dOmega on the support, one thread per entry e = (i, j):
//   out_e = scale ((T_e + T_tr(e))/2 + lambda2 w_e - [i = j] / w_ii),  T = Omega S on the
// support (Alg. 1 step 4's G restricted to the entries of the iterate).
template <typename T>
__global__ void __launch_bounds__(256)
k_support_grad(int64_t nnz, const int* __restrict__ row, const int* __restrict__ ci, const T* __restrict__ cv,
               const int* __restrict__ tr, const double* __restrict__ Tv, double lam2, double scale,
               double* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int te = tr[e] >= 0 ? tr[e] : (int)e;
        const double w = (double)cv[e];
        double o = 0.5 * (Tv[e] + Tv[te]) + lam2 * w;
        if (ci[e] == row[e]) o -= 1.0 / w;
        out[e] = scale * o;
    }
}

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

// one block of 256 threads: CG stage `stage` on the reduced partials
__global__ void __launch_bounds__(256) k_cg_scalar(const double* part, int nb, int stage, double tol2, CgState* cg) {
    const double v = reduce_parts(part, nb);
    if (threadIdx.x == 0) cg_update(stage, v, tol2, cg);
}

// x += alpha p; r -= alpha Ap (unless CG has stopped), then CG stage 2 on <r, r>.  Every
// block reads done and alpha before the last one updates them.
__global__ void __launch_bounds__(256)
k_cg_xr(int64_t n, CgState* cg, const double* p, const double* Ap, double* x, double* r, double* part, double tol2) {
    const bool live = cg->done == 0;
    const double a = cg->alpha;
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double rt = r[t];
        if (live) {
            x[t] = fma(a, p[t], x[t]);
            rt = fma(-a, Ap[t], rt);
            r[t] = rt;
        }
        s = fma(rt, rt, s);
    }
    partial_then_scalar(s, part, 2, tol2, cg);
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
    constexpr int TL = sizeof(T) == 4 ? 64 : 32;      // two tiles: 33 KB (FP32) / 17 KB (FP64) of shared memory
    const int nt = (p + TL - 1) / TL;
    // bit 0: 16-byte stores of G; bit 1: 16-byte loads of S
    const int vec = (((uintptr_t)G % 16 == 0 && (ldg * (int64_t)sizeof(T)) % 16 == 0) ? 1 : 0) |
                    (((uintptr_t)S % 16 == 0 && (lds * (int64_t)sizeof(T)) % 16 == 0) ? 2 : 0);
    k_dense_grad_pair<T, TL><<<(unsigned)((int64_t)nt * (nt + 1) / 2), 256, 0, s>>>(p, om, rinfo, rdv, S, lds, G,
                                                                                   ldg, lam2, scale, nt, vec);
}

template <typename T>
void launch_spmm_dense(int p, Csr<T> om, const int4* rinfo, const T* rdv, const T* B, int64_t ldb, int64_t m,
                       T* C, int64_t ldc, cudaStream_t s) {
    dim3 g((p + kW - 1) / kW, (unsigned)((m + 127) / 128));
    k_spmm_dense<T><<<g, 256, 0, s>>>(p, om, rinfo, rdv, B, ldb, m, C, ldc);
}

template <typename T>
void launch_spmm_dense_t(int p, Csr<T> om, const int4* rinfo, const T* rdv, const T* B, int64_t ldb, int64_t m,
                         T* Ct, int64_t ldt, T scale, cudaStream_t s) {
    dim3 g((unsigned)((p + 31) / 32), (unsigned)((m + 127) / 128));
    k_spmm_dense_t<T><<<g, 256, 0, s>>>(p, om, rinfo, rdv, B, ldb, m, Ct, ldt, scale);
}

void launch_transpose(const void* in, int in_dt, int64_t rows, int64_t cols, int64_t ldi, void* out, int out_dt,
                      int64_t ldo, double scale, cudaStream_t s) {
    dim3 g((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    const bool o64 = out_dt == HPC_F64;
    if (in_dt == HPC_BF16 && o64) {
        k_transpose<__nv_bfloat16, double><<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(in), rows, cols, ldi,
                                                              static_cast<double*>(out), ldo, scale);
    } else if (in_dt == HPC_BF16) {
        k_transpose<__nv_bfloat16, float><<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(in), rows, cols, ldi,
                                                             static_cast<float*>(out), ldo, scale);
    } else if (in_dt == HPC_F64 && o64) {
        k_transpose<double, double><<<g, 256, 0, s>>>(static_cast<const double*>(in), rows, cols, ldi,
                                                       static_cast<double*>(out), ldo, scale);
    } else if (in_dt == HPC_F64) {
        k_transpose<double, float><<<g, 256, 0, s>>>(static_cast<const double*>(in), rows, cols, ldi,
                                                      static_cast<float*>(out), ldo, scale);
    } else if (o64) {
        k_transpose<float, double><<<g, 256, 0, s>>>(static_cast<const float*>(in), rows, cols, ldi,
                                                      static_cast<double*>(out), ldo, scale);
    } else {
        k_transpose<float, float><<<g, 256, 0, s>>>(static_cast<const float*>(in), rows, cols, ldi,
                                                     static_cast<float*>(out), ldo, scale);
    }
}

template <typename T>
void launch_transpose_index(int p, Csr<T> om, int* tr, int* row, cudaStream_t s) {
    k_transpose_index<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, tr, row);
}

template <typename T>
void launch_support_product(int p, Csr<T> om, const int4* rinfo, const double* v, const T* S, int64_t lds,
                            double* out, cudaStream_t s) {
    k_support_product<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, rinfo, v, S, lds, out);
}

template <typename T>
void launch_support_sddmm(int p, Csr<T> om, const T* yt, const T* xt, int64_t ld, int64_t n, double* out,
                          cudaStream_t s) {
    k_support_sddmm<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, yt, xt, ld, n, out);
}

template <typename T>
void launch_support_combine(int64_t nnz, const int* row, Csr<T> om, const int* tr, const double* Tv, const double* v,
                            double lam2, int mode, double* out, double* part, double tol2, void* cg, cudaStream_t s) {
    k_support_combine<T><<<cg_part_blocks(nnz), 256, 0, s>>>(nnz, row, om.ci, om.cv, tr, Tv, v, lam2, mode, out, part,
                                                              tol2, static_cast<CgState*>(cg));
}

template <typename T>
void launch_support_grad(int64_t nnz, const int* row, Csr<T> om, const int* tr, const double* Tv, double lam2,
                         double scale, double* out, cudaStream_t s) {
    k_support_grad<T><<<cg_part_blocks(nnz), 256, 0, s>>>(nnz, row, om.ci, om.cv, tr, Tv, lam2, scale, out);
}

template <typename T>
void launch_support_vectors(int p, int64_t nnz, Csr<T> om, double* omega_d, double* sign_off, cudaStream_t s) {
    k_support_values<T><<<256, 256, 0, s>>>(nnz, om.cv, omega_d);
    k_sign_off<T><<<(p + kW - 1) / kW, 256, 0, s>>>(p, om, sign_off);
}

int cg_part_blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 1024); }

template <typename T>
void launch_support_product_p(int64_t nnz, const int* row, Csr<T> om, const int4* rinfo, const double* r,
                              const double* p_old, double* p_new, const void* cg, const T* S, int64_t lds,
                              double* out, cudaStream_t s) {
    k_support_product_p<T><<<cg_part_blocks(nnz), 256, 0, s>>>(nnz, row, om, rinfo, r, p_old, p_new,
                                                                static_cast<const CgState*>(cg), S, lds, out);
}

void launch_dot_part(int64_t n, const double* a, const double* b, double* part, cudaStream_t s) {
    k_dot_part<<<cg_part_blocks(n), 256, 0, s>>>(n, a, b, part);
}

void launch_cg_scalar(const double* part, int nb, int stage, double tol2, void* cg, cudaStream_t s) {
    k_cg_scalar<<<1, 256, 0, s>>>(part, nb, stage, tol2, static_cast<CgState*>(cg));
}

void launch_cg_xr(int64_t n, void* cg, const double* p, const double* Ap, double* x, double* r, double* part,
                  double tol2, cudaStream_t s) {
    k_cg_xr<<<cg_part_blocks(n), 256, 0, s>>>(n, static_cast<CgState*>(cg), p, Ap, x, r, part, tol2);
}

size_t cg_state_bytes() { return sizeof(CgState); }

#define HPC_ADJ_INSTANTIATE(T)                                                                                  \
    template void launch_dense_grad<T>(int, Csr<T>, const int4*, const T*, const T*, int64_t, T*, int64_t, T, T, \
                                       cudaStream_t);                                                           \
    template void launch_spmm_dense<T>(int, Csr<T>, const int4*, const T*, const T*, int64_t, int64_t, T*,      \
                                       int64_t, cudaStream_t);                                                  \
    template void launch_spmm_dense_t<T>(int, Csr<T>, const int4*, const T*, const T*, int64_t, int64_t, T*,    \
                                         int64_t, T, cudaStream_t);                                             \
    template void launch_transpose_index<T>(int, Csr<T>, int*, int*, cudaStream_t);                             \
    template void launch_support_product<T>(int, Csr<T>, const int4*, const double*, const T*, int64_t, double*, \
                                            cudaStream_t);                                                      \
    template void launch_support_sddmm<T>(int, Csr<T>, const T*, const T*, int64_t, int64_t, double*,         \
                                          cudaStream_t);                                                        \
    template void launch_support_combine<T>(int64_t, const int*, Csr<T>, const int*, const double*,             \
                                            const double*, double, int, double*, double*, double, void*,        \
                                            cudaStream_t);                                                      \
    template void launch_support_product_p<T>(int64_t, const int*, Csr<T>, const int4*, const double*,         \
                                              const double*, double*, const void*, const T*, int64_t, double*,   \
                                              cudaStream_t);                                                     \
    template void launch_support_vectors<T>(int, int64_t, Csr<T>, double*, double*, cudaStream_t);          \
    template void launch_support_grad<T>(int64_t, const int*, Csr<T>, const int*, const double*, double,      \
                                         double, double*, cudaStream_t);                                        \
    template int launch_smooth_parts<T>(int, Csr<T>, const double*, double*, double*, cudaStream_t);

HPC_ADJ_INSTANTIATE(float)
HPC_ADJ_INSTANTIATE(double)

}  // namespace hpc
