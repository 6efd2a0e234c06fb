// One outer iteration of the proximal-gradient method (Alg. 1 / Alg. 2 steps 5-12)
// as a chain of device kernels; no host round trip inside a step except the two
// control-block reads the driver does.
//
//  1. k_grad_screen   W = Omega S column block by column block (row-split CSR SpMM,
//                     Alg. 2 step 3/10).  Instead of storing W it emits the
//                     entries (i, j) that any prox step can touch: the support of
//                     Omega, the diagonal, and every |W_ij| > lambda1 (if both
//                     |W_ij| and |W_ji| are <= lambda1 then |G_ij| <= lambda1 and
//                     eq. (2) maps the entry to 0 for every tau).
//  2. candidates      symmetric per-row candidate lists: count, scan, scatter,
//                     sort + de-dup, fill W for partner entries by gathers (same
//                     FMA order as step 1, so bitwise equal), then
//                     G_ij = (W_ij + W_ji)/2 + lambda2 w_ij - [i=j]/w_ii
//                     (Alg. 2 steps 5-6; the transpose is a lookup, so G is
//                     bitwise symmetric) and the objective partials of Omega^k.
//  3. line search     for a window of tau = 2^-h values at once: the prox of eq. (2)
//                     on the candidates and the sufficient-decrease test of
//                     Alg. 1 step 9, evaluated in the algebraically identical form
//                        (D S D)/2 + lambda2/2 ||D||^2 + sum_i phi(D_ii / w_ii) <= ||D||^2 / (2 tau),
//                        D = Omega+ - Omega, phi(x) = x - log(1 + x),
//                     (g(O+) - g(O) - <D, G> expanded: the W terms cancel), with
//                     gathers of S on the candidate pattern and FP64 sums.
//  4. accept          compaction of the accepted Omega+ into CSR (ballot/popc row
//                     counts, scan, ordered write) and the stopping rule.
//
// Steps 2-4 are device functions over a grid of blocks.  They run either as a
// chain of kernels of their own or, all of them, as one cooperative kernel
// (k_iter_tail, section 5) with grid-wide barriers between them; both forms give
// the same entries and decisions.
#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <vector>

#include "internal.cuh"
#include "ptx.cuh"

namespace hpc {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ void vload(float (&a)[4], const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}
__device__ __forceinline__ void vload(double (&a)[2], const double* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    a[0] = v.x; a[1] = v.y;
}

__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Compensated FP32 accumulator for sums that would otherwise need FP64, whose
// rate on this GPU is a small fraction of FP32: every addition is Knuth's
// TwoSum, the rounding errors collect in lo, and the pair carries ~44 bits.
// FP64 appears only in the final cross-block reductions.
struct F2 {
    float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void acc_add(F2& a, float b) {
    const float s = __fadd_rn(a.hi, b);
    const float bp = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, err);
}
__device__ __forceinline__ void acc_add(double& a, double b) { a += b; }
__device__ __forceinline__ double acc_value(const F2& a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ F2 warp_sum(F2 a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(kFull, a.hi, o);
        const float l = __shfl_xor_sync(kFull, a.lo, o);
        acc_add(a, h);
        a.lo = __fadd_rn(a.lo, l);
    }
    return a;
}
template <typename T> struct AccOf { using type = F2; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float mulT(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulT(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float logT(float a) { return logf(a); }
__device__ __forceinline__ double logT(double a) { return log(a); }

// phi(x) = x - log(1 + x) for x > -1.  FP32: for |x| < 1/8 the Taylor series
// sum_{k>=0} (-1)^k x^(k+2) / (k+2), truncated after x^10 (relative error
// < 2e-9), avoids the cancellation of x - log1p(x); otherwise x - log1pf(x).
__device__ __forceinline__ float phiT(float x) {
    if (fabsf(x) < 0.125f) {
        float r = 1.0f / 10.0f;
        r = fmaf(x, r, -1.0f / 9.0f);
        r = fmaf(x, r, 1.0f / 8.0f);
        r = fmaf(x, r, -1.0f / 7.0f);
        r = fmaf(x, r, 1.0f / 6.0f);
        r = fmaf(x, r, -1.0f / 5.0f);
        r = fmaf(x, r, 1.0f / 4.0f);
        r = fmaf(x, r, -1.0f / 3.0f);
        r = fmaf(x, r, 1.0f / 2.0f);
        return x * x * r;
    }
    return x - log1pf(x);
}
__device__ __forceinline__ double phiT(double x) { return x - log1p(x); }

// Prox of eq. (2) for one candidate entry at step tau (tau and tau*lambda1 are
// exact: tau is a power of two).  The diagonal is not thresholded.
template <typename T>
__device__ __forceinline__ T prox_entry(T om, T g, T tau, T tl1, bool diag) {
    const T z = om - tau * g;
    if (diag) return z;
    if (z > tl1) return z - tl1;
    if (z < -tl1) return z + tl1;
    return T(0);
}

// ------------------------------------------------------------------ 0. reset
template <typename T>
__global__ void k_iter_begin(Buckets<T> bk, int p, Ctrl* ctrl, int use_cond, cudaGraphConditionalHandle ls_cond,
                             unsigned* bar) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = tid; i < p; i += gridDim.x * blockDim.x) {
        bk.cnt[i] = 0;
        bk.cur[i] = 0;
    }
    if (bar && tid == 0) *bar = 0u;   // arrival counter of the fused tail's grid barriers
    if (tid == 0) {
        ctrl->em_count = 0;
        ctrl->obs_next = 0;
        ctrl->n_offrows = 0;
        ctrl->n_mirror = 0;
        ctrl->n_pairs = 0;
        ctrl->n_row_items = 0;
        ctrl->bucket_total = 0;
        ctrl->flags = 0;
        ctrl->ls_accept = -1;
        ctrl->ls_base = 0;
        ctrl->nnz_next = 0;
        ctrl->converged = 0;
        ctrl->tau = 0.0;
        ctrl->delta2 = 0.0;
        ctrl->iter_attempts += 1;
        // device loop: the line-search loop of this iteration runs at least once
        if (use_cond) cudaGraphSetConditional(ls_cond, 1u);
    }
}

// Device-loop timing: globaltimer stamps around the screening pass.
__global__ void k_stamp(Ctrl* ctrl, int end) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (end) ctrl->screen_ns += (long long)t - ctrl->t_stamp;
    else ctrl->t_stamp = (long long)t;
}

// Device loop: copy the accepted iterate into the buffers the next iteration's
// kernels read, and decide whether the loop goes on (an accepted step, below the
// iteration limit, stopping rule not met or not in use, no flag raised).
template <typename T>
__global__ void k_csr_commit(Csr<T> nx, Csr<T> cu, int p, Ctrl* ctrl, int use_cond, cudaGraphConditionalHandle cond) {
    const bool ok = ctrl->flags == 0 && ctrl->ls_accept >= 0;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = gridDim.x * blockDim.x;
    if (ok) {
        const int nnz = nx.rp[p];
        for (int i = tid; i <= p; i += nt) cu.rp[i] = nx.rp[i];
        for (int q = tid; q < nnz; q += nt) {
            cu.ci[q] = nx.ci[q];
            cu.cv[q] = nx.cv[q];
        }
    }
    if (tid == 0) {
        if (ok) ctrl->nnz_cur = nx.rp[p];
        const bool more = ok && ctrl->iter < ctrl->iter_limit && !(ctrl->use_stop && ctrl->converged);
        if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
    }
}

// ------------------------------------------------------------------ 1. screening SpMM
// W = Omega S is split as W = diag(w) S + O S, O the off-diagonal part of Omega.
// Every entry is accumulated in one canonical order -- the diagonal term first,
// W_ij = w_ii * S_ij, then fma(w_ik, S_kj, .) over the off-diagonal k of row i
// in ascending column order -- which the gather fill of partner entries
// repeats, so both produce the same bits.
//
// The diagonal term streams S itself, so the pass is staged like a copy: one
// persistent CTA per SM, a producer thread loading 64-row x BJ-column tiles of S
// (32 KB, BJ = 32*V) with TMA into a kScreenStages-deep mbarrier ring, and eight
// consumer warps, each screening eight rows of every tile (lane l holds columns
// l*V .. l*V+V-1, one 16-byte shared-memory read per row).  This kernel takes the
// pure-diagonal rows, whose W row is w_ii S_i,: and needs no other row of S.
// S is symmetric (bitwise: the Gram writes one triangle and mirrors it), so for
// i < j the element S_ij gives both W_ij = w_ii S_ij (row i pure) and
// W_ji = w_jj S_ij (row j pure): only the tiles on or above the diagonal are
// streamed -- half of S -- and an entry of a pair of pure rows is emitted from
// both sides at once, flagged as paired (no partner gather downstream).  When
// only one of the two rows is pure, its side is emitted alone and the other row
// is screened by k_grad_screen_rows.  Row set-up (CSR bounds, diagonal position
// and value, the pure-diagonal flag) comes from k_row_info, cached in shared
// memory; the column side reads the diagonal values and the purity bitmask.
//
// Work order: the upper-triangle tiles of row chunk c are the column blocks
// jb >= jbmin(c) = floor(64 c / BJ); chunks are taken in the folded order
// 0, nc-1, 1, nc-2, ... so that consecutive chunks pair a long tile row with a
// short one, and CTA g owns a contiguous, equal share of that sequence (the
// host precomputes its prefix, seqoff).
constexpr int kScreenTileRows = 64;
constexpr int kScreenStages = 5;
constexpr int kScreenMaxChunks = 32;              // row chunks per CTA (shared-memory row cache)
constexpr int kScreenThreads = kThreads + 32;     // 8 consumer warps + 1 producer warp
constexpr long long kScreenWaitLimit = 1ll << 22;     // polls of at most 1 us each

// Column side of a tile, loaded with it: the BJ diagonal values and 16 bytes of the
// purity bitmask around the block.
template <typename T>
constexpr int screen_col_bytes() { return 32 * (16 / (int)sizeof(T)) * (int)sizeof(T) + 16; }

template <typename T>
constexpr int screen_smem_bytes() {
    return kScreenStages * kScreenTileRows * 32 * (16 / (int)sizeof(T)) * (int)sizeof(T)  // tiles
           + kScreenStages * screen_col_bytes<T>()                                        // column side
           + kScreenMaxChunks * kScreenTileRows * (16 + (int)sizeof(T))                   // row cache
           + 2 * kScreenStages * 8 + 16                                                   // barriers + flag
           + 1024;                                                                        // alignment
}

__host__ __device__ __forceinline__ int screen_seq_chunk(int s, int nc) { return (s & 1) ? nc - 1 - (s >> 1) : (s >> 1); }

// NaN-propagating maximum of two non-negative values.
template <typename T>
__device__ __forceinline__ T max_nan(T a, T b) { return (a != a || b != b) ? T(NAN) : (a > b ? a : b); }

// Per row of the iterate: CSR bounds, position of the diagonal (-1 if absent,
// found by binary search: columns ascend), its value, and the pure-diagonal bit
// (pmask, one word per 32 rows); rows with off-diagonal entries (or no
// diagonal) are appended to offlist (any order: the screening output is
// re-sorted per row downstream).  With colmax (the bound screening), also
// colmax[jb] = max |w_jj| over the pure rows j of column block jb (NaN if one is
// NaN): the launch gives every thread one row, so the BJ rows of a block are in
// one CTA (256 is a multiple of BJ) and are reduced in shared memory.
template <typename T>
__global__ void __launch_bounds__(256)
k_row_info(int p, Csr<T> om, int4* __restrict__ rinfo, T* __restrict__ rdv, unsigned* __restrict__ pmask,
           int* __restrict__ offlist, Ctrl* __restrict__ ctrl, T* __restrict__ colmax, int nbm) {
    constexpr int BJ = 32 * (16 / (int)sizeof(T));
    __shared__ T s_cm[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (lane == 0) s_cm[warp] = T(0);
    for (int base = gw * 32; base < p; base += nw * 32) {
        const int i = base + lane;
        bool pure = false;
        T dv = T(0);
        if (i < p) {
            const int rb = om.rp[i], re = om.rp[i + 1];
            int lo = rb, hi = re;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (om.ci[mid] < i) lo = mid + 1; else hi = mid;
            }
            const int pd = (lo < re && om.ci[lo] == i) ? lo : -1;
            dv = pd >= 0 ? om.cv[pd] : T(0);
            pure = (re - rb == 1) && pd >= 0;
            rinfo[i] = make_int4(rb, re, pd, pure ? 1 : 0);
            rdv[i] = dv;
            if (!pure && offlist) offlist[atomicAdd(&ctrl->n_offrows, 1)] = i;
        }
        const unsigned word = __ballot_sync(kFull, pure);
        if (pmask && lane == 0) pmask[base >> 5] = word;
        if (colmax) {
            T a = pure ? (T)fabs(dv) : T(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a = max_nan(a, __shfl_xor_sync(kFull, a, o));
            if (lane == 0) s_cm[warp] = a;
        }
    }
    if (colmax) {
        __syncthreads();
        constexpr int kPerBlock = 256 / BJ, kWarpsPerCol = BJ / 32;
        if (threadIdx.x < kPerBlock) {
            const int jb = blockIdx.x * kPerBlock + threadIdx.x;
            if (jb < nbm) {
                T m = T(0);
#pragma unroll
                for (int w = 0; w < kWarpsPerCol; ++w) m = max_nan(m, s_cm[threadIdx.x * kWarpsPerCol + w]);
                colmax[jb] = m;
            }
        }
    }
}

template <typename T>
struct Screen {
    static constexpr int V = 16 / sizeof(T);
    static constexpr int BJ = 32 * V;

    // Append the entries of row i in this block that a prox step can touch: the
    // support (diagonal included) and every |W_ij| > lambda1 (NaN included).
    // (values by value, so callers' accumulators stay in registers)
    static __device__ __noinline__ void emit(int i, T a0, T a1, T a2, T a3, int rb, int re, int j0, int p,
                                             const int* __restrict__ ci, const T* __restrict__ cv, T lam1,
                                             Emit<T> em, Ctrl* ctrl, int lane) {
        const T acc[4] = {a0, a1, a2, a3};
        unsigned mbits = 0;
        T om[V];
#pragma unroll
        for (int v = 0; v < V; ++v) om[v] = T(0);
        for (int q = rb; q < re; q += 32) {
            const int c = (q + lane < re) ? ci[q + lane] : -1;
            unsigned bal = __ballot_sync(kFull, c >= j0 && c < j0 + BJ);
            while (bal) {
                const int src = __ffs(bal) - 1;
                bal &= bal - 1;
                const int o = __shfl_sync(kFull, c, src) - j0;
                if (lane == o / V) {
                    const T w = cv[q + src];
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (o % V == v) om[v] = w;
                    mbits |= 1u << (o % V);
                }
            }
        }
        bool emit_v[V];
        int c = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = j0 + lane * V + v;
            emit_v[v] = (j < p) && (((mbits >> v) & 1u) || !(fabs(acc[v]) <= lam1));
            c += emit_v[v] ? 1 : 0;
        }
        const int incl = warp_incl_scan(c, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        if (!total) return;
        int base_pos = 0;
        if (lane == 0) base_pos = atomicAdd(&ctrl->em_count, total);
        base_pos = __shfl_sync(kFull, base_pos, 0);
        int pos = base_pos + incl - c;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (emit_v[v]) {
                if (pos < em.cap) {
                    const int j = j0 + lane * V + v;
                    const bool sup = (mbits >> v) & 1u;
                    em.row[pos] = i;
                    em.col[pos] = sup ? (int)((unsigned)j | 0x80000000u) : j;
                    em.w[pos] = acc[v];
                    em.om[pos] = sup ? om[v] : T(0);
                }
                ++pos;
            }
        }
    }
};

// Append the entries a lane found in one tile: n records (row, col word, W, w_ij)
// staged in registers by the caller; one atomicAdd per warp.
template <typename T>
__device__ __forceinline__ int warp_reserve(int n, Ctrl* ctrl, int lane) {
    const int incl = warp_incl_scan(n, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    int base = 0;
    if (total && lane == 0) base = atomicAdd(&ctrl->em_count, total);
    base = __shfl_sync(kFull, base, 0);
    return base + incl - n;
}

template <typename T>
__device__ __forceinline__ void put_entry(const Emit<T>& em, int& pos, int i, unsigned colw, T w, T om) {
    if (pos < em.cap) {
        em.row[pos] = i;
        em.col[pos] = (int)colw;
        em.w[pos] = w;
        em.om[pos] = om;
    }
    ++pos;
}

template <typename T>
__global__ void __launch_bounds__(kScreenThreads, 1)
k_grad_screen(const __grid_constant__ CUtensorMap smap, int p, const long long* __restrict__ seqoff,
              const int4* __restrict__ rinfo, const T* __restrict__ rdv, const unsigned* __restrict__ pmask,
              int pairs_cap, Emit<T> em, Ctrl* __restrict__ ctrl) {
    using Sc = Screen<T>;
    constexpr int V = Sc::V;
    constexpr int BJ = Sc::BJ;
    constexpr int R = kScreenTileRows;
    constexpr int kTileBytes = R * BJ * (int)sizeof(T);
    constexpr int kColBytes = screen_col_bytes<T>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    T* tiles = reinterpret_cast<T*>(smem);
    uint8_t* cols = smem + kScreenStages * kTileBytes;       // per stage: BJ values, then 4 mask words
    int4* s_info = reinterpret_cast<int4*>(cols + kScreenStages * kColBytes);
    T* s_dv = reinterpret_cast<T*>(s_info + kScreenMaxChunks * R);
    uint64_t* full = reinterpret_cast<uint64_t*>(s_dv + kScreenMaxChunks * R);
    uint64_t* empty = full + kScreenStages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kScreenStages);

    if (2 * ctrl->n_offrows > p) return;      // dense rows: k_grad_screen_rows covers every row
    if (ctrl->n_pairs <= pairs_cap) return;   // the bound screening's items cover the pairs
    const T lam1 = (T)ctrl->lam1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const int nc = (p + R - 1) / R;
    const int nblocks = (p + BJ - 1) / BJ;
    // this CTA's contiguous share of the folded tile sequence
    const long long total = seqoff[nc];
    const long long lo = total * blockIdx.x / G, hi = total * (blockIdx.x + 1) / G;
    const int items = (int)(hi - lo);
    int s_first = 0, s_last = 0;
    if (items > 0) {
        int a = 0, b = nc - 1;                       // last s with seqoff[s] <= lo
        while (a < b) { const int m = (a + b + 1) >> 1; if (seqoff[m] <= lo) a = m; else b = m - 1; }
        s_first = a;
        a = s_first; b = nc - 1;                     // last s with seqoff[s] <= hi - 1
        while (a < b) { const int m = (a + b + 1) >> 1; if (seqoff[m] <= hi - 1) a = m; else b = m - 1; }
        s_last = a;
    }
    const int mine = items > 0 ? s_last - s_first + 1 : 0;   // <= kScreenMaxChunks (host-checked grid)
    const int jb_first = items > 0 ? (int)((long long)screen_seq_chunk(s_first, nc) * R / BJ + (lo - seqoff[s_first])) : 0;

    if (threadIdx.x == 0) {
        for (int st = 0; st < kScreenStages; ++st) {
            ptx::mbar_init(&full[st], 1);
            ptx::mbar_init(&empty[st], kWarps);
        }
        *abort_flag = 0;
        ptx::mbar_init_fence();
    }
    // cache the row set-up of this CTA's chunks (slot m: the chunk at position s_first + m)
    for (int t = threadIdx.x; t < mine * R; t += blockDim.x) {
        const int i = screen_seq_chunk(s_first + t / R, nc) * R + (t % R);
        s_info[t] = i < p ? rinfo[i] : make_int4(0, 0, -1, 0);
        s_dv[t] = i < p ? rdv[i] : T(0);
    }
    __syncthreads();

    if (warp == kWarps) {
        // ---------------- producer: one TMA tile per (row chunk, column block) item
        if (lane == 0) {
            ptx::prefetch_tensormap(&smap);
            int sq = s_first, jb = jb_first, chunk = screen_seq_chunk(s_first, nc);
            for (int t = 0; t < items; ++t) {
                const int st = t % kScreenStages;
                const uint32_t ph = (uint32_t)(t / kScreenStages) & 1u;
                if (!ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, abort_flag, kScreenWaitLimit)) break;
                ptx::mbar_expect_tx(&full[st], kTileBytes + kColBytes);
                ptx::tma_load_2d(reinterpret_cast<uint8_t*>(tiles) + st * kTileBytes, &smap, &full[st], jb * BJ,
                                 chunk * R);
                uint8_t* cdst = cols + st * kColBytes;
                ptx::bulk_load(cdst, rdv + (size_t)jb * BJ, BJ * (int)sizeof(T), &full[st]);
                ptx::bulk_load(cdst + BJ * sizeof(T), pmask + (((jb * BJ) >> 5) & ~3), 16, &full[st]);
                if (++jb == nblocks) {
                    ++sq;
                    chunk = sq < nc ? screen_seq_chunk(sq, nc) : 0;
                    jb = (int)((long long)chunk * R / BJ);
                }
            }
        }
    } else {
        // ---------------- consumers: warp w screens rows 8w .. 8w+7 of every tile
        int sq = s_first, jb = jb_first, chunk = screen_seq_chunk(s_first, nc);
        for (int t = 0; t < items; ++t) {
            const int st = t % kScreenStages;
            const uint32_t ph = (uint32_t)(t / kScreenStages) & 1u;
            const int j0 = jb * BJ;
            const int jl = j0 + lane * V;
            if (!ptx::mbar_wait_bounded(&full[st], ph, abort_flag, kScreenWaitLimit)) break;
            // column side, staged with the tile: diagonal values and purity of rows jl..jl+V-1
            const uint8_t* csrc = cols + st * kColBytes;
            T cdv[V];
            if constexpr (V == 4) {
                const float4 x = *reinterpret_cast<const float4*>(csrc + lane * 16);
                cdv[0] = x.x; cdv[1] = x.y; cdv[2] = x.z; cdv[3] = x.w;
            } else {
                const double2 x = *reinterpret_cast<const double2*>(csrc + lane * 16);
                cdv[0] = x.x; cdv[1] = x.y;
            }
            const unsigned* cw = reinterpret_cast<const unsigned*>(csrc + BJ * sizeof(T));
            const unsigned cbits = (cw[(jl >> 5) - ((j0 >> 5) & ~3)] >> (jl & 31)) & ((1u << V) - 1u);
            const int m = sq - s_first;
            const T* tile = tiles + (size_t)st * R * BJ;
            const int r0 = chunk * R + warp * 8;
            // Filter: off the diagonal band and the ragged edges, an element can emit only
            // if fl(max(|w_ii|, |w_jj|) |S_ij|) > lambda1 over the pure sides (rounding is
            // monotone, so this is the larger of the two products); warps with a hit, and
            // the tiles on the diagonal or at p, take the exact path below.
            const bool edge = (j0 < chunk * R + R) || (j0 + BJ > p) || (chunk * R + R > p);
            bool hit = edge;
            if (!edge) {
                T cm[V];
#pragma unroll
                for (int v = 0; v < V; ++v) cm[v] = ((cbits >> v) & 1u) ? fabs(cdv[v]) : T(0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const T rm = s_info[m * R + warp * 8 + q].w ? fabs(s_dv[m * R + warp * 8 + q]) : T(0);
                    T sv[V];
                    if constexpr (V == 4) {
                        const float4 x = *reinterpret_cast<const float4*>(tile + (warp * 8 + q) * BJ + lane * V);
                        sv[0] = x.x; sv[1] = x.y; sv[2] = x.z; sv[3] = x.w;
                    } else {
                        const double2 x = *reinterpret_cast<const double2*>(tile + (warp * 8 + q) * BJ + lane * V);
                        sv[0] = x.x; sv[1] = x.y;
                    }
#pragma unroll
                    for (int v = 0; v < V; ++v) hit |= !(fabs(mulT(fmax(rm, cm[v]), sv[v])) <= lam1);
                }
            }
            if (__any_sync(kFull, hit)) {
            // rows r0..r0+7 x columns jl..jl+V-1: count the records, then write them
            T av[8][V], bv[8][V];
            unsigned ea = 0, eb = 0;     // bit (q*V + v): emit row side / column side
            unsigned pairbits = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int r = r0 + q;
                const int4 info = s_info[m * R + warp * 8 + q];
                const T dv = s_dv[m * R + warp * 8 + q];
                const bool rpure = info.w != 0;
                T sv[V];
                if constexpr (V == 4) {
                    const float4 x = *reinterpret_cast<const float4*>(tile + (warp * 8 + q) * BJ + lane * V);
                    sv[0] = x.x; sv[1] = x.y; sv[2] = x.z; sv[3] = x.w;
                } else {
                    const double2 x = *reinterpret_cast<const double2*>(tile + (warp * 8 + q) * BJ + lane * V);
                    sv[0] = x.x; sv[1] = x.y;
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int j = jl + v;
                    const bool cpure = (cbits >> v) & 1u;
                    av[q][v] = mulT(dv, sv[v]);
                    bv[q][v] = mulT(cdv[v], sv[v]);
                    const unsigned bit = 1u << (q * V + v);
                    if (r < p && j < p && j > r) {
                        {
                            const bool ba = rpure && !(fabs(av[q][v]) <= lam1);
                            const bool bb = cpure && !(fabs(bv[q][v]) <= lam1);
                            if (rpure && cpure) {
                                if (ba || bb) { ea |= bit; eb |= bit; pairbits |= bit; }
                            } else {
                                if (ba) ea |= bit;
                                if (bb) eb |= bit;
                            }
                        }
                    }
                }
            }
            const int n = __popc(ea) + __popc(eb);
            if (__any_sync(kFull, n != 0)) {
                int pos = warp_reserve<T>(n, ctrl, lane);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const unsigned bit = 1u << (q * V + v);
                        const int r = r0 + q, j = jl + v;
                        const unsigned pf = (pairbits & bit) ? 0x40000000u : 0u;
                        if (ea & bit) put_entry(em, pos, r, (unsigned)j | pf, av[q][v], T(0));
                        if (eb & bit) put_entry(em, pos, j, (unsigned)r | pf, bv[q][v], T(0));
                    }
                }
            }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[st]);
            if (++jb == nblocks) {
                ++sq;
                chunk = sq < nc ? screen_seq_chunk(sq, nc) : 0;
                jb = (int)((long long)chunk * R / BJ);
            }
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) {
            atomicOr(&ctrl->flags, kFlagTimeout);
            // drain: bounded waits so that no TMA copy lands after the CTA exits
            for (int t = max(0, items - kScreenStages); t < items; ++t) {
                const int st = t % kScreenStages;
                const uint32_t ph = (uint32_t)(t / kScreenStages) & 1u;
                for (long long it = 0; it < (1ll << 22) && !ptx::mbar_try_wait(&full[st], ph); ++it) __nanosleep(64);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ bound screening
// Non-negative value rounded up to BF16 (an upper bound: 8 bits of mantissa kept,
// the rest carried upwards), and its float value.
__device__ __forceinline__ unsigned short bf16_up(float x) {
    if (!(x == x)) return 0x7fc0;
    unsigned u = __float_as_uint(x);
    if (u & 0xffffu) u += 0x10000u;
    return (unsigned short)(u >> 16);
}
__device__ __forceinline__ unsigned short bf16_up(double x) { return bf16_up(__double2float_ru(x)); }
__device__ __forceinline__ float bf16_val(unsigned short b) { return __uint_as_float((unsigned)b << 16); }

// Eight BF16 block maxima from one 16-byte load (element 0 in the low half of x).
__device__ __forceinline__ void bf16x8(const uint4 v, float (&f)[8]) {
    f[0] = __uint_as_float(v.x << 16);
    f[1] = __uint_as_float(v.x & 0xffff0000u);
    f[2] = __uint_as_float(v.y << 16);
    f[3] = __uint_as_float(v.y & 0xffff0000u);
    f[4] = __uint_as_float(v.z << 16);
    f[5] = __uint_as_float(v.z & 0xffff0000u);
    f[6] = __uint_as_float(v.w << 16);
    f[7] = __uint_as_float(v.w & 0xffff0000u);
}

// Once per data load: m1[i][jb] = max |S_ij| over the column block jb (width BJ),
// j != i, j < p, rounded up to BF16; NaN if the block holds a NaN.  One warp per row.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_rowblock_max(const T* __restrict__ S, int64_t ld, int p, int nbm, unsigned short* __restrict__ m1) {
    using Sc = Screen<T>;
    constexpr int V = Sc::V;
    constexpr int BJ = Sc::BJ;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < p; i += nw) {
        const T* row = S + (int64_t)i * ld;
        for (int jb = 0; jb < nbm; ++jb) {
            const int jl = jb * BJ + lane * V;
            T x[V];
            vload(x, row + jl);
            T mx = T(0);
            bool nan = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int j = jl + v;
                const T a = (j < p && j != i) ? fabs(x[v]) : T(0);
                nan |= !(a == a);
                mx = a > mx ? a : mx;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T y = __shfl_xor_sync(kFull, mx, o);
                mx = y > mx ? y : mx;
            }
            nan = __any_sync(kFull, nan);
            if (lane == 0) m1[(int64_t)i * nbm + jb] = nan ? (unsigned short)0x7fc0 : bf16_up(mx);
        }
    }
}

// Selection of the (row i, column block jb) items of the upper triangle (some j > i
// in the block) that can emit: with m = max(|w_ii| if row i is pure, max |w_jj| over
// the pure rows j of the block), an item is kept iff fl(m * m1[i][jb]) > lambda1.
// Rounding is monotone, so a dropped item has no j with fl(|w_ii| |S_ij|) > lambda1
// or fl(|w_jj| |S_ij|) > lambda1: the emitted set is exactly the full screen's.  The
// pure rows' diagonals (support) are emitted here.  Nothing happens when the rows
// with neighbours are the majority (k_grad_screen_rows then screens every row).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pair_select(const T* __restrict__ S, int64_t ld, int p, int nbm, const unsigned short* __restrict__ m1,
              const unsigned short* __restrict__ m1g, int ngl, const int4* __restrict__ rinfo,
              const T* __restrict__ rdv, const void* colmax_raw, int2* __restrict__ pairs, int cap, Emit<T> em,
              Ctrl* __restrict__ ctrl) {
    constexpr int BJ = Screen<T>::BJ;
    if (2 * ctrl->n_offrows > p) return;
    const T* colmax = static_cast<const T*>(colmax_raw);
    const T lam1 = (T)ctrl->lam1;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    // the pure diagonals, 32 rows per warp
    for (int base = gw * 32; base < p; base += nw * 32) {
        const int i = base + lane;
        const bool d = i < p && rinfo[i].w;
        T w = T(0), dv = T(0);
        if (d) {
            dv = rdv[i];
            w = mulT(dv, S[(int64_t)i * ld + i]);
        }
        int pos = warp_reserve<T>(d ? 1 : 0, ctrl, lane);
        if (d) put_entry(em, pos, i, (unsigned)i | 0x80000000u, w, dv);
    }
    if (m1g) {
        // the items, two-level: the column maxima and their group maxima (8 blocks) in
        // shared memory (the launch sizes it); one thread per (row, span of 8 groups).
        // A group is dropped when fl(max(|w_ii|, max colmax over the group) * m1g) <=
        // lambda1: both factors bound each block's, so no block of it could be kept.
        // Only the groups that pass load their 8 block maxima for the per-block test.
        extern __shared__ __align__(16) unsigned char ps_smem[];
        T* s_cm = reinterpret_cast<T*>(ps_smem);
        const int ng = nbm / 8;
        T* s_cg = s_cm + nbm;
        for (int t = threadIdx.x; t < nbm; t += blockDim.x) s_cm[t] = colmax[t];
        __syncthreads();
        for (int g = threadIdx.x; g < ng; g += blockDim.x) {
            T m = T(0);
#pragma unroll
            for (int v = 0; v < 8; ++v) m = max_nan(m, s_cm[8 * g + v]);
            s_cg[g] = m;
        }
        __syncthreads();
        const int nsp = (ng + 7) / 8;
        const int total = p * nsp;          // the launch checks that this fits an int
        for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
            const int it = base + threadIdx.x;
            unsigned long long bits = 0;
            int i = 0, g0 = 0;
            if (it < total) {
                i = it / nsp;
                g0 = (it - i * nsp) * 8;
                const int jb0 = (i + 1) / BJ;
                if (8 * (g0 + 8) > jb0) {
                    const T rm = rinfo[i].w ? fabs(rdv[i]) : T(0);
                    float gf[8];
                    bf16x8(*reinterpret_cast<const uint4*>(m1g + (int64_t)i * ngl + g0), gf);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int g = g0 + q;
                        if (g >= ng || 8 * (g + 1) <= jb0) continue;
                        const T mg = max_nan(rm, s_cg[g]);
                        if (mg == T(0) || mulT(mg, (T)gf[q]) <= lam1) continue;
                        float f[8];
                        bf16x8(*reinterpret_cast<const uint4*>(m1 + (int64_t)i * nbm + 8 * g), f);
#pragma unroll
                        for (int v = 0; v < 8; ++v) {
                            const int jb = 8 * g + v;
                            if ((i + 1) < min(p, (jb + 1) * BJ)) {
                                const T m = max_nan(rm, s_cm[jb]);
                                if ((m != T(0)) && !(mulT(m, (T)f[v]) <= lam1)) bits |= 1ull << (8 * q + v);
                            }
                        }
                    }
                }
            }
            const int c = __popcll(bits);
            if (!__any_sync(kFull, c != 0)) continue;
            const int incl = warp_incl_scan(c, lane);
            int q = 0;
            if (lane == 31) q = atomicAdd(&ctrl->n_pairs, incl);
            q = __shfl_sync(kFull, q, 31) + incl - c;
            while (bits) {
                const int b = __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                if (q < cap) pairs[q] = make_int2(i, 8 * g0 + b);
                ++q;
            }
        }
        return;
    }
    // the items, one warp per row, four 32-block chunks of loads in flight
    for (int i = m1 ? gw : p; i < p; i += nw) {
        const int4 ri = rinfo[i];
        const T rm = ri.w ? fabs(rdv[i]) : T(0);
        const int jb0 = (i + 1) / BJ;
        const unsigned short* mrow = m1 + (int64_t)i * nbm;
        for (int c0 = jb0; c0 < nbm; c0 += 128) {
            unsigned short mv[4];
            T cm[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jb = c0 + 32 * u + lane;
                mv[u] = jb < nbm ? mrow[jb] : (unsigned short)0;
                cm[u] = jb < nbm ? colmax[jb] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jb = c0 + 32 * u + lane;
                bool keep = false;
                if (jb < nbm && (i + 1) < min(p, (jb + 1) * BJ)) {
                    const T m = max_nan(rm, cm[u]);
                    keep = (m != T(0)) && !(mulT(m, (T)bf16_val(mv[u])) <= lam1);
                }
                const unsigned bal = __ballot_sync(kFull, keep);
                if (!bal) continue;
                int base = 0;
                if (lane == 0) base = atomicAdd(&ctrl->n_pairs, __popc(bal));
                base = __shfl_sync(kFull, base, 0);
                const int q = base + __popc(bal & ((1u << lane) - 1u));
                if (keep && q < cap) pairs[q] = make_int2(i, jb);
            }
        }
    }
}

// The kept items: for j > i in the block, W_ij = w_ii S_ij (row i pure) and W_ji =
// w_jj S_ij (row j pure), emitted as in the triangle stream (pairs of pure rows from
// both sides, flagged as paired).  Idle when the items overflowed their list: the
// triangle stream then covers every pair.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_pair_screen(const T* __restrict__ S, int64_t ld, int p, const int2* __restrict__ pairs, int cap,
              const int4* __restrict__ rinfo, const T* __restrict__ rdv, const unsigned* __restrict__ pmask,
              Emit<T> em, Ctrl* __restrict__ ctrl) {
    using Sc = Screen<T>;
    constexpr int V = Sc::V;
    constexpr int BJ = Sc::BJ;
    if (2 * ctrl->n_offrows > p) return;
    const int n = ctrl->n_pairs;
    if (n > cap) return;
    const T lam1 = (T)ctrl->lam1;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = gw; t < n; t += nw) {
        const int2 it = pairs[t];
        const int i = it.x;
        const int jl = it.y * BJ + lane * V;
        T sv[V], cdv[V];
        vload(sv, S + (int64_t)i * ld + jl);
        vload(cdv, rdv + jl);
        const unsigned cbits = (pmask[jl >> 5] >> (jl & 31)) & ((1u << V) - 1u);
        const bool rpure = rinfo[i].w != 0;
        const T dv = rdv[i];
        T av[V], bv[V];
        unsigned ea = 0, eb = 0, pb = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = jl + v;
            av[v] = mulT(dv, sv[v]);
            bv[v] = mulT(cdv[v], sv[v]);
            if (j > i && j < p) {
                const bool cpure = (cbits >> v) & 1u;
                const bool ba = rpure && !(fabs(av[v]) <= lam1);
                const bool bb = cpure && !(fabs(bv[v]) <= lam1);
                if (rpure && cpure) {
                    if (ba || bb) { ea |= 1u << v; eb |= 1u << v; pb |= 1u << v; }
                } else {
                    if (ba) ea |= 1u << v;
                    if (bb) eb |= 1u << v;
                }
            }
        }
        const int cnt = __popc(ea) + __popc(eb);
        if (!__any_sync(kFull, cnt != 0)) continue;
        int pos = warp_reserve<T>(cnt, ctrl, lane);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = jl + v;
            const unsigned pf = ((pb >> v) & 1u) ? 0x40000000u : 0u;
            if ((ea >> v) & 1u) put_entry(em, pos, i, (unsigned)j | pf, av[v], T(0));
            if ((eb >> v) & 1u) put_entry(em, pos, j, (unsigned)i | pf, bv[v], T(0));
        }
    }
}

// Rows with neighbours: which column blocks can emit.  For row i with terms t (the
// diagonal w_ii at k = i, then w_ik), W_ij is an FMA chain of m terms, so
// |fl(W_ij)| <= (1 + gamma_m) sum_t |w_t| |S_{k_t j}| <= (1 + gamma_m) B_jb with
// B_jb = sum_t |w_t| m1[k_t][jb] (m1 is an upper bound) and gamma_m = m u / (1 - m u).
// The bound is evaluated in FP32 with every operation rounded towards +inf (the
// operands are non-negative, so the result is at least the exact value) and
// compared with the emission threshold in T; for m u <= 2^-10, gamma_m <=
// m u (1 + 2^-9), and longer chains keep every block.  Columns j = k_t are the
// support (and i), whose blocks are always processed; for the other columns the
// bound holds because m1 excludes each row's diagonal.  Row i needs block jb iff
// the block holds a support column or !(bound <= lambda1) (NaN keeps it).
template <typename T>
__device__ __forceinline__ float abs_up(T x) {
    if constexpr (sizeof(T) == 4) return fabsf(x);
    else return __double2float_ru(fabs(x));
}

template <typename T>
__device__ __forceinline__ bool bound_keeps(float g1, float B, bool long_chain, T lam1) {
    const float bound = __fmul_ru(g1, B);
    bool below;
    if constexpr (sizeof(T) == 4) below = bound <= lam1;
    else below = (double)bound <= lam1;
    return long_chain || !below;
}

// The row kernel's item list: (8-row group, column block) items any of whose rows
// needs the block.  One CTA per group of 8 listed rows, warp w on the group's row w;
// the rows' block words (bit jb % 32 of word jb / 32) meet in shared memory and are
// ORed there.  VEC (nbm % 8 == 0, m1 rows 16-byte aligned): in each chunk of 256
// blocks lane l covers blocks c0 + 8l .. c0 + 8l + 7 with one 16-byte load of m1 per
// term, the row's terms fetched 32 at a time and broadcast (a slot that is not a
// term -- the diagonal's CSR position, the tail of the last fetch -- is the weight 0
// on row i itself, which adds 0, or the NaN that row i's own diagonal term already
// adds).  Otherwise lane l takes block 32 w + l of word w.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads)
k_rows_items(int p, int nbm, const unsigned short* __restrict__ m1, const int4* __restrict__ rinfo,
             const T* __restrict__ rdv, const int* __restrict__ offlist, const int* __restrict__ ci,
             const T* __restrict__ cv, int2* __restrict__ items, int cap, Ctrl* __restrict__ ctrl) {
    constexpr int BJ = Screen<T>::BJ;
    static_assert(kWarps == 8, "one warp per row of an 8-row group");
    extern __shared__ unsigned ri_words[];          // [kWarps][nwords]
    const float u = sizeof(T) == 4 ? 0x1p-24f : 0x1p-53f;
    const bool all_rows = 2 * ctrl->n_offrows > p;
    const int nrows = all_rows ? p : ctrl->n_offrows;
    const int ngroups = (nrows + 7) / 8;
    const int nwords = (nbm + 31) / 32;
    const T lam1 = (T)ctrl->lam1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned* my = ri_words + warp * nwords;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int pos = grp * 8 + warp;
        if (pos >= nrows) {
            for (int w = lane; w < nwords; w += 32) my[w] = 0u;
        } else {
            const int i = all_rows ? pos : offlist[pos];
            const int4 ri = rinfo[i];
            const float di = abs_up(rdv[i]);
            const int m = 1 + (ri.y - ri.x) - (ri.z >= 0 ? 1 : 0);
            const float mu = (float)m * u;                       // exact: m < 2^24, u a power of 2
            const float g1 = __fadd_ru(1.0f, __fmul_ru(mu, 1.001953125f));
            const bool long_chain = mu > 0x1p-10f;
            const int ib = i / BJ;
            if constexpr (VEC) {
                for (int c0 = 0; c0 < nbm; c0 += 256) {
                    const int jl = c0 + lane * 8;
                    const bool act = jl < nbm;
                    float B[8], f[8];
                    unsigned sup = (unsigned)(ib - jl) < 8u ? 1u << (ib - jl) : 0u;
                    bf16x8(act ? *reinterpret_cast<const uint4*>(m1 + (int64_t)i * nbm + jl) : make_uint4(0, 0, 0, 0),
                           f);
#pragma unroll
                    for (int v = 0; v < 8; ++v) B[v] = __fmul_ru(di, f[v]);
                    for (int q0 = ri.x; q0 < ri.y; q0 += 32) {
                        const int q = q0 + lane;
                        const bool term = q < ri.y && q != ri.z;
                        const int kq = term ? ci[q] : i;
                        const float wq = term ? abs_up(cv[q]) : 0.0f;
                        const int nt = min(32, ri.y - q0);
#pragma unroll 4
                        for (int t = 0; t < nt; ++t) {
                            const int k = __shfl_sync(kFull, kq, t);
                            const float w = __shfl_sync(kFull, wq, t);
                            bf16x8(act ? *reinterpret_cast<const uint4*>(m1 + (int64_t)k * nbm + jl)
                                       : make_uint4(0, 0, 0, 0),
                                   f);
#pragma unroll
                            for (int v = 0; v < 8; ++v) B[v] = __fadd_ru(B[v], __fmul_ru(w, f[v]));
                            const int kb = k / BJ;
                            if ((unsigned)(kb - jl) < 8u) sup |= 1u << (kb - jl);
                        }
                    }
                    unsigned bits = 0;
                    if (act) {
#pragma unroll
                        for (int v = 0; v < 8; ++v)
                            if (((sup >> v) & 1u) || bound_keeps<T>(g1, B[v], long_chain, lam1)) bits |= 1u << v;
                    }
                    unsigned word = bits << (8 * (lane & 3));
                    word |= __shfl_xor_sync(kFull, word, 1);
                    word |= __shfl_xor_sync(kFull, word, 2);
                    const int w = jl / 32;
                    if ((lane & 3) == 0 && w < nwords) my[w] = word;
                }
            } else {
                for (int w0 = 0; w0 < nwords; ++w0) {
                    const int jb = w0 * 32 + lane;
                    bool keep = false;
                    if (jb < nbm) {
                        float B = __fmul_ru(di, bf16_val(m1[(int64_t)i * nbm + jb]));
                        bool sup = ib == jb;
#pragma unroll 4
                        for (int q = ri.x; q < ri.y; ++q) {
                            const int k = ci[q];
                            if (q != ri.z) {
                                B = __fadd_ru(B, __fmul_ru(abs_up(cv[q]), bf16_val(m1[(int64_t)k * nbm + jb])));
                                sup |= (k / BJ) == jb;
                            }
                        }
                        keep = sup || bound_keeps<T>(g1, B, long_chain, lam1);
                    }
                    const unsigned word = __ballot_sync(kFull, keep);
                    if (lane == 0) my[w0] = word;
                }
            }
        }
        __syncthreads();
        // the group's items: warps take words w0 = warp, warp + 8, ...
        for (int w0 = warp; w0 < nwords; w0 += kWarps) {
            unsigned word = lane < 8 ? ri_words[lane * nwords + w0] : 0u;
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) word |= __shfl_xor_sync(kFull, word, o);
            word = __shfl_sync(kFull, word, 0);
            if (!word) continue;
            const bool keep = (word >> lane) & 1u;
            int base = 0;
            if (lane == 0) base = atomicAdd(&ctrl->n_row_items, __popc(word));
            base = __shfl_sync(kFull, base, 0);
            const int q = base + __popc(word & ((1u << lane) - 1u));
            if (keep && q < cap) items[q] = make_int2(grp, w0 * 32 + lane);
        }
        __syncthreads();
    }
}

// Rows with off-diagonal entries (or, when they are the majority, every row):
// persistent warps over items (column block, group of 8 listed rows), column
// block outermost so that in-flight warps share S[:, J] in L2.  The terms of the
// item's rows -- per row the diagonal term w_ii S[i, J] (0 if absent) followed by
// the off-diagonal terms w_ik S[k, J] in CSR order -- form one stream whose
// (k, w_ik) the lanes fetch 32 at a time; the S-row segments are then loaded
// kTermBatch at a time across row boundaries, so every batch keeps that many
// loads in flight whatever the row lengths, and each row still accumulates in
// the canonical order.
constexpr int kRowsPerItem = 8;
constexpr int kTermBatch = 8;

// MINB: resident CTAs per SM the registers are sized for (2: 128 registers; 3: 80,
// with a small spill); the tuning knob rows_ctas_per_sm >= 3 selects the second.
template <typename T, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
k_grad_screen_rows(const T* __restrict__ S, int64_t ld, int p, const int4* __restrict__ rinfo,
                   const T* __restrict__ rdv, const int* __restrict__ offlist, const int* __restrict__ ci,
                   const T* __restrict__ cv, const int2* __restrict__ row_items, int row_items_cap, Emit<T> em,
                   Ctrl* __restrict__ ctrl) {
    using Sc = Screen<T>;
    constexpr int V = Sc::V;
    constexpr int BJ = Sc::BJ;
    constexpr int R = kRowsPerItem;
    __shared__ int s_row[kWarps][R], s_rb[kWarps][R], s_re[kWarps][R], s_pd[kWarps][R], s_start[kWarps][R];
    __shared__ T s_dv[kWarps][R];
    __shared__ T s_acc[kWarps][R][V][32];
    __shared__ int s_sup[kWarps][R];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T lam1 = (T)ctrl->lam1;
    const bool all_rows = 2 * ctrl->n_offrows > p;
    const int nrows = all_rows ? p : ctrl->n_offrows;
    const int ngroups = (nrows + R - 1) / R;
    const int nblocks = (p + BJ - 1) / BJ;
    // the bound screening's list of kept items, unless it overflowed; else every item
    const bool listed = row_items && ctrl->n_row_items <= row_items_cap;
    const long long items = listed ? (long long)ctrl->n_row_items : (long long)ngroups * nblocks;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long it = gw; it < items; it += nw) {
        int jb, grp;
        if (listed) {
            const int2 x = row_items[it];
            grp = x.x;
            jb = x.y;
        } else {
            jb = (int)(it / ngroups);
            grp = (int)(it % ngroups);
        }
        const int j0 = jb * BJ;
        const int nr = min(R, nrows - grp * R);
        // lanes < nr: the row's set-up and the length of its term stream
        int slen = 0;
        __syncwarp();
        if (lane < nr) {
            const int row = all_rows ? grp * R + lane : offlist[grp * R + lane];
            const int4 inf = rinfo[row];
            s_row[warp][lane] = row;
            s_rb[warp][lane] = inf.x;
            s_re[warp][lane] = inf.y;
            s_pd[warp][lane] = inf.z;
            s_dv[warp][lane] = rdv[row];
            slen = 1 + (inf.y - inf.x) - (inf.z >= 0 ? 1 : 0);
        }
        const int incl = warp_incl_scan(slen, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        if (lane < nr) s_start[warp][lane] = incl - slen;
        __syncwarp();

        int cur = -1;
        T acc[V];
        bool sup = false;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = T(0);
        for (int w0 = 0; w0 < total; w0 += 32) {
            // lane l fetches term w0 + l: its row slot, S row k and weight
            const int x = w0 + lane;
            int tk = 0, tr = -1;
            T tw = T(0);
            if (x < total) {
                int r = 0;
                for (int q = 1; q < nr; ++q)
                    if (s_start[warp][q] <= x) r = q;
                const int y = x - s_start[warp][r];
                tr = r;
                if (y == 0) {
                    tk = s_row[warp][r];
                    tw = s_dv[warp][r];
                } else {
                    int qq = s_rb[warp][r] + y - 1;
                    if (s_pd[warp][r] >= 0 && qq >= s_pd[warp][r]) ++qq;
                    tk = ci[qq];
                    tw = cv[qq];
                }
            }
            const int nt = min(32, total - w0);
            for (int b0 = 0; b0 < nt; b0 += kTermBatch) {
                T sv[kTermBatch][V];
                int kk[kTermBatch], rr[kTermBatch];
                T ww[kTermBatch];
#pragma unroll
                for (int u = 0; u < kTermBatch; ++u) {
                    const int t = b0 + u;
                    kk[u] = __shfl_sync(kFull, tk, t & 31);
                    ww[u] = __shfl_sync(kFull, tw, t & 31);
                    rr[u] = __shfl_sync(kFull, tr, t & 31);
                    if (t >= nt) rr[u] = -1;
                    if (rr[u] >= 0) vload(sv[u], S + (int64_t)kk[u] * ld + j0 + lane * V);
                }
#pragma unroll
                for (int u = 0; u < kTermBatch; ++u) {
                    if (rr[u] < 0) break;
                    const bool in_blk = kk[u] >= j0 && kk[u] < j0 + BJ;
                    if (rr[u] != cur) {
                        if (cur >= 0) {
#pragma unroll
                            for (int v = 0; v < V; ++v) s_acc[warp][cur][v][lane] = acc[v];
                            if (lane == 0) s_sup[warp][cur] = sup ? 1 : 0;
                        }
                        cur = rr[u];
                        // a row's stream starts with its diagonal term
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = mulT(ww[u], sv[u][v]);
                        sup = in_blk;
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = fmaT(ww[u], sv[u][v], acc[v]);
                        sup |= in_blk;
                    }
                }
            }
        }
        if (cur >= 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) s_acc[warp][cur][v][lane] = acc[v];
            if (lane == 0) s_sup[warp][cur] = sup ? 1 : 0;
        }
        __syncwarp();
        // screen the item's rows
        for (int r = 0; r < nr; ++r) {
            T a[V];
            bool big = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                a[v] = s_acc[warp][r][v][lane];
                big |= !(fabs(a[v]) <= lam1);
            }
            if (__any_sync(kFull, big) || s_sup[warp][r])
                Sc::emit(s_row[warp][r], a[0], a[V > 1 ? 1 : 0], a[V > 2 ? 2 : 0], a[V > 3 ? 3 : 0], s_rb[warp][r],
                         s_re[warp][r], j0, p, ci, cv, lam1, em, ctrl, lane);
        }
    }
}

// ------------------------------------------------------------------ 2. candidates
// Each step of the candidate, line-search and accept chain is a device function
// over a grid of nb blocks of kThreads threads, this block being bid, so that the
// same code runs as a kernel of its own (bid = blockIdx.x, nb = gridDim.x) or as a
// phase of the fused iteration kernel k_iter_tail.  flags0 is the control block's
// flag word as the step sees it at its start.
template <typename T>
__device__ void bucket_count_body(const Emit<T>& em, const Buckets<T>& bk, Ctrl* ctrl, int bid, int nb) {
    const int total = ctrl->em_count;
    if (total > em.cap) {
        if (bid == 0 && threadIdx.x == 0) atomicOr(&ctrl->flags, kFlagEmOverflow);
        return;
    }
    for (int e = bid * kThreads + threadIdx.x; e < total; e += nb * kThreads) {
        const int i = em.row[e];
        const int cj = em.col[e];
        atomicAdd(&bk.cnt[i], 1);
        // off the support and not emitted from both sides: partner request in row j
        if (cj >= 0 && !(cj & 0x40000000)) atomicAdd(&bk.cnt[cj], 1);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bucket_count(Emit<T> em, Buckets<T> bk, Ctrl* ctrl) {
    bucket_count_body(em, bk, ctrl, blockIdx.x, gridDim.x);
}

// Line-search work units of a row with c candidate entries before de-dup: the
// pairs (a <= b) of its 32-entry chunks.
__device__ __forceinline__ long long ls_units(int c) {
    const long long t = (c + 31) >> 5;
    return t * (t + 1) / 2;
}

__device__ __forceinline__ long long warp_incl_scan64(long long x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Multi-block exclusive scan of n ints, out[n] = total; if total > cap, sets flag.
// With uoff (the bucket scan), also the list of long rows (more than kShortRow
// entries), in ascending order, into longlist, their count into ctrl->n_long, and
// the exclusive 64-bit prefix of their ls_units over that list into uoff
// (uoff[n_long] = total units).  Two kernels over tiles of kScanTile inputs (thread
// t of a tile owns 16 consecutive inputs, four 16-byte loads): k_scan_reduce writes
// each tile's sums, k_scan_apply adds the sums of the tiles before its own and
// writes the tile's prefixes.  No block waits on another.
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 16;
constexpr int kScanTile = kScanThreads * kScanPerThread;

// The 16 inputs of thread t (zero past n); in + base is 16-byte aligned.  The
// input is read through the coherent path: inside the fused iteration kernel it was
// written by the same launch.
__device__ __forceinline__ void scan_load16(const int* in, int n, int base, int (&v)[kScanPerThread]) {
#pragma unroll
    for (int q = 0; q < kScanPerThread; q += 4) {
        const int j = base + q;
        if (j + 4 <= n) {
            const int4 x = *reinterpret_cast<const int4*>(in + j);
            v[q] = x.x; v[q + 1] = x.y; v[q + 2] = x.z; v[q + 3] = x.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) v[q + r] = j + r < n ? in[j + r] : 0;
        }
    }
}

// Shared memory of one scan tile.
struct ScanSmem {
    int ws[kScanThreads / 32], wl[kScanThreads / 32];
    long long wu[kScanThreads / 32];
    int ps, pl;
    long long pu;
};

// Block-wide sums (with_long: also the long-row count and units) of the thread values.
template <bool INCL>
__device__ __forceinline__ void scan_block3(int& s, int& l, long long& u, bool with_long, int* ws, int* wl,
                                            long long* wu) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s0 = s, l0 = l;
    const long long u0 = u;
    s = warp_incl_scan(s, lane);
    if (with_long) { l = warp_incl_scan(l, lane); u = warp_incl_scan64(u, lane); }
    if (lane == 31) { ws[warp] = s; wl[warp] = l; wu[warp] = u; }
    __syncthreads();
    int ps = 0, pl = 0;
    long long pu = 0;
    for (int w = 0; w < warp; ++w) { ps += ws[w]; pl += wl[w]; pu += wu[w]; }
    s += ps; l += pl; u += pu;
    if (!INCL) { s -= s0; l -= l0; u -= u0; }
}

// Tile t of the first scan kernel: the tile's sums into part[t].
__device__ void scan_reduce_tile(const int* in, int n, int flags0, bool with_long, ScanPart* part, int t,
                                 ScanSmem& sm) {
    if (flags0 & ~kFlagLsFail & (kFlagEmOverflow | kFlagBucketOverflow)) return;
    int v[kScanPerThread];
    scan_load16(in, n, t * kScanTile + threadIdx.x * kScanPerThread, v);
    int s = 0, l = 0;
    long long u = 0;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        s += v[q];
        if (with_long && v[q] > kShortRow) { ++l; u += ls_units(v[q]); }
    }
    scan_block3<true>(s, l, u, with_long, sm.ws, sm.wl, sm.wu);
    if (threadIdx.x == kScanThreads - 1) part[t] = ScanPart{s, l, u};
    __syncthreads();   // sm is reused by the next tile of this block
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const int* in, int n, const Ctrl* __restrict__ ctrl, bool with_long, ScanPart* __restrict__ part) {
    __shared__ ScanSmem sm;
    scan_reduce_tile(in, n, ctrl->flags, with_long, part, blockIdx.x, sm);
}

// Tile t of ntiles of the second scan kernel: the tile's exclusive prefixes, and in
// the last tile the totals (and the stopping rule, for the compaction's scan).
__device__ void scan_apply_tile(const int* in, int* out, int n, int cap, Ctrl* ctrl, int flags0, int flag,
                                int* total_dst, long long* uoff, int* longlist, const ScanPart* part, int conv_cap,
                                double eps, int t, int ntiles, ScanSmem& sm) {
    if (flags0 & ~kFlagLsFail & (kFlagEmOverflow | kFlagBucketOverflow)) {
        if (t == 0 && threadIdx.x == 0) {
            out[n] = 0;
            if (uoff) { uoff[0] = 0; ctrl->n_long = 0; }
        }
        return;
    }
    const bool with_long = uoff != nullptr;
    const int base = t * kScanTile + threadIdx.x * kScanPerThread;
    int v[kScanPerThread];
    scan_load16(in, n, base, v);
    // the sums of the tiles before this one
    {
        int ps = 0, pl = 0;
        long long pu = 0;
        for (int b = threadIdx.x; b < t; b += kScanThreads) {
            const ScanPart q = part[b];
            ps += q.s; pl += q.l; pu += q.u;
        }
        scan_block3<true>(ps, pl, pu, with_long, sm.ws, sm.wl, sm.wu);
        if (threadIdx.x == kScanThreads - 1) { sm.ps = ps; sm.pl = pl; sm.pu = pu; }
        __syncthreads();
    }
    int s = 0, l = 0;
    long long u = 0;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        s += v[q];
        if (with_long && v[q] > kShortRow) { ++l; u += ls_units(v[q]); }
    }
    scan_block3<false>(s, l, u, with_long, sm.ws, sm.wl, sm.wu);
    int run = s + sm.ps, lrun = l + sm.pl;
    long long urun = u + sm.pu;
    __syncthreads();   // sm is reused by the next tile of this block
    int o[kScanPerThread];
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        o[q] = run;
        run += v[q];
        if (with_long && v[q] > kShortRow) {
            longlist[lrun] = base + q;
            uoff[lrun] = urun;
            ++lrun;
            urun += ls_units(v[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kScanPerThread; q += 4) {
        const int j = base + q;
        if (j + 4 <= n) {
            *reinterpret_cast<int4*>(out + j) = make_int4(o[q], o[q + 1], o[q + 2], o[q + 3]);
        } else {
            for (int r = 0; r < 4 && j + r < n; ++r) out[j + r] = o[q + r];
        }
    }
    if (t == ntiles - 1 && threadIdx.x == kScanThreads - 1) {
        // the inputs past n are zero, so this thread's running values are the totals
        const int total = run;
        out[n] = total;
        if (with_long) {
            uoff[lrun] = urun;
            ctrl->n_long = lrun;
        }
        if (total_dst) *total_dst = total;
        if (total > cap) atomicOr(&ctrl->flags, flag);
        // the compaction's scan (conv_cap >= 0) also takes the stopping-rule step once
        // a step is accepted: the new entry count against the CSR capacity, and the
        // relative change ||dOmega||_F / ||Omega||_F, both known before the write-out
        if (conv_cap >= 0 && ctrl->flags == 0 && ctrl->ls_accept >= 0) {
            ctrl->nnz_next = total;
            if (total > conv_cap) {
                ctrl->flags |= kFlagNnzOverflow;
            } else {
                const double rel = sqrt(ctrl->delta2) / sqrt(ctrl->norm2_cur);
                ctrl->rel = rel;
                ctrl->converged = rel < eps ? 1 : 0;
                ctrl->iter += 1;
            }
        }
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const int* in, int* __restrict__ out, int n, int cap, Ctrl* ctrl, int flag, int* total_dst,
             long long* __restrict__ uoff, int* __restrict__ longlist, const ScanPart* __restrict__ part,
             int conv_cap, double eps) {
    __shared__ ScanSmem sm;
    scan_apply_tile(in, out, n, cap, ctrl, ctrl->flags, flag, total_dst, uoff, longlist, part, conv_cap, eps,
                    blockIdx.x, gridDim.x, sm);
}

void launch_scan(const int* in, int* out, int n, int cap, Ctrl* ctrl, int flag, int* total_dst, long long* uoff,
                 int* longlist, ScanPart* part, cudaStream_t s, int conv_cap = -1, double eps = 0.0) {
    const int tiles = (int)std::max<int64_t>(1, ((int64_t)n + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<tiles, kScanThreads, 0, s>>>(in, n, ctrl, uoff != nullptr, part);
    k_scan_apply<<<tiles, kScanThreads, 0, s>>>(in, out, n, cap, ctrl, flag, total_dst, uoff, longlist, part, conv_cap,
                                                eps);
}

template <typename T>
__device__ void bucket_scatter_body(const Emit<T>& em, const Buckets<T>& bk, const Ctrl* ctrl, int flags0, int bid,
                                    int nb) {
    if (flags0) return;
    const int total = ctrl->em_count;
    for (int e = bid * kThreads + threadIdx.x; e < total; e += nb * kThreads) {
        const int i = em.row[e];
        const int cj = em.col[e];
        const int j = cj & 0x3fffffff;
        const int pos = bk.off[i] + atomicAdd(&bk.cur[i], 1);
        bk.col_a[pos] = j;
        bk.w_a[pos] = em.w[e];
        bk.om_a[pos] = em.om[e];
        bk.fl_a[pos] = (unsigned char)(kEntOwn | (cj < 0 ? kEntSupp : 0));
        if (cj >= 0 && !(cj & 0x40000000)) {
            const int q = bk.off[j] + atomicAdd(&bk.cur[j], 1);
            bk.col_a[q] = i;
            bk.w_a[q] = T(0);
            bk.om_a[q] = T(0);
            bk.fl_a[q] = kEntMirror;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bucket_scatter(Emit<T> em, Buckets<T> bk, const Ctrl* ctrl) {
    bucket_scatter_body(em, bk, ctrl, ctrl->flags, blockIdx.x, gridDim.x);
}

// Sort key of a scattered entry: column, own entry before the partner request.
template <typename T>
__device__ __forceinline__ unsigned sort_key(const Buckets<T>& bk, int pos) {
    return (unsigned)bk.col_a[pos] * 2u + ((bk.fl_a[pos] & kEntMirror) ? 1u : 0u);
}

template <typename T>
__device__ __forceinline__ unsigned sort_key_b(const Buckets<T>& bk, int pos) {
    return (unsigned)bk.col_b[pos] * 2u + ((bk.fl_b[pos] & kEntMirror) ? 1u : 0u);
}

// Append the kept partner entries of this warp (flag `mir`, final position pos in
// row i) to the fill list.
template <typename T>
__device__ __forceinline__ void push_mirrors(const Buckets<T>& bk, Ctrl* ctrl, bool mir, int pos, int i, int lane) {
    const unsigned mb = __ballot_sync(kFull, mir);
    if (!mb) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&ctrl->n_mirror, __popc(mb));
    base = __shfl_sync(kFull, base, 0);
    if (mir) bk.mir[base + __popc(mb & ((1u << lane) - 1u))] = make_int2(pos, i);
}

// Rows longer than one warp are sorted by a whole block in shared memory (bitonic
// on 64-bit (key, index) words) up to this many entries; beyond it, in chunks of
// this many that are then merged by ranks (binary searches in the other chunks).
constexpr int kSortSmem = 4096;
constexpr int kSortShort = 32;

// Sort by (column, own-before-partner) into the b arrays, then drop partner
// requests whose own entry exists (the own entry sorts just before).  Three
// tiers: rows of at most kShortRow entries one lane each (32 rows per warp);
// rows of at most 32 entries one warp each, in registers; longer rows (hub
// rows with thousands of candidates) one block each, so none serialises a warp.
// The last two tiers take their rows from the long-row list of the bucket scan.
struct SortSmem {
    unsigned long long key[kSortSmem];
    int cnt[kWarps];
    int out;
};

template <typename T>
__device__ void bucket_sort_body(const Buckets<T>& bk, int p, Ctrl* ctrl, int flags0, int bid, int nb,
                                 SortSmem& sm) {
    unsigned long long* s_key = sm.key;
    int* s_cnt = sm.cnt;
    int& s_out = sm.out;
    if (flags0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = (bid * kThreads + threadIdx.x) >> 5;
    const int nw = (nb * kThreads) >> 5;
    const int nlong = ctrl->n_long;

    // 1. short rows, one lane each
    for (int base = gw * 32; base < p; base += nw * 32) {
        const int i = base + lane;
        const int c = i < p ? bk.cnt[i] : kShortRow + 1;
        const bool sh = c <= kShortRow;
        int beg = 0, kept = 0;
        bool m0 = false, m1 = false;
        if (sh) {
            beg = bk.off[i];
            int e0 = 0, e1 = 1;
            bool drop1 = false;
            if (c == 2) {
                if (sort_key(bk, beg + 1) < sort_key(bk, beg)) { e0 = 1; e1 = 0; }
                drop1 = (bk.fl_a[beg + e1] & kEntMirror) && bk.col_a[beg + e1] == bk.col_a[beg + e0];
            }
            if (c >= 1) {
                bk.col_b[beg] = bk.col_a[beg + e0];
                bk.w_b[beg] = bk.w_a[beg + e0];
                bk.om_b[beg] = bk.om_a[beg + e0];
                bk.fl_b[beg] = bk.fl_a[beg + e0];
                m0 = bk.fl_a[beg + e0] & kEntMirror;
                kept = 1;
            }
            if (c == 2 && !drop1) {
                bk.col_b[beg + 1] = bk.col_a[beg + e1];
                bk.w_b[beg + 1] = bk.w_a[beg + e1];
                bk.om_b[beg + 1] = bk.om_a[beg + e1];
                bk.fl_b[beg + 1] = bk.fl_a[beg + e1];
                m1 = bk.fl_a[beg + e1] & kEntMirror;
                kept = 2;
            }
            bk.len[i] = kept;
        }
        push_mirrors(bk, ctrl, m0, beg, i, lane);
        push_mirrors(bk, ctrl, m1, beg + 1, i, lane);
    }

    // 2. rows of kShortRow+1 .. 32 entries, one warp each: rank by shuffles (keys are
    // distinct), drop a partner request whose predecessor in column order is the own
    // entry of that column, and write the kept entries in order
    for (int li = gw; li < nlong; li += nw) {
        const int i = bk.longlist[li];
        const int beg = bk.off[i];
        const int c = bk.cnt[i];
        if (c > kSortShort) continue;
        const bool valid = lane < c;
        int col = 0;
        T w = T(0), om = T(0);
        unsigned char fl = 0;
        if (valid) {
            col = bk.col_a[beg + lane];
            w = bk.w_a[beg + lane];
            om = bk.om_a[beg + lane];
            fl = bk.fl_a[beg + lane];
        }
        const int key = valid ? col * 2 + ((fl & kEntMirror) ? 1 : 0) : 0x7fffffff;
        int rank = 0;
        for (int t = 0; t < 32; ++t) rank += (__shfl_sync(kFull, key, t) < key) ? 1 : 0;
        int pred_col = -1;
        for (int t = 0; t < 32; ++t) {
            const int rt = __shfl_sync(kFull, rank, t);
            const int ct = __shfl_sync(kFull, col, t);
            if (t < c && rt == rank - 1) pred_col = ct;
        }
        const bool keep = valid && !((fl & kEntMirror) && rank > 0 && pred_col == col);
        const unsigned kb = __ballot_sync(kFull, keep);
        int pos = 0;
        for (int t = 0; t < 32; ++t) {
            const int rt = __shfl_sync(kFull, rank, t);
            pos += (((kb >> t) & 1u) && rt < rank) ? 1 : 0;
        }
        if (keep) {
            bk.col_b[beg + pos] = col;
            bk.w_b[beg + pos] = w;
            bk.om_b[beg + pos] = om;
            bk.fl_b[beg + pos] = fl;
        }
        push_mirrors(bk, ctrl, keep && (fl & kEntMirror), beg + pos, i, lane);
        if (lane == 0) bk.len[i] = __popc(kb);
    }

    // 3. rows over 32 entries, one block each
    for (int li = bid; li < nlong; li += nb) {
        const int i = bk.longlist[li];
        const int c = bk.cnt[i];
        if (c <= kSortShort) continue;
        const int beg = bk.off[i];
        __syncthreads();
        if (c <= kSortSmem) {
            int n2 = 1;
            while (n2 < c) n2 <<= 1;
            for (int e = threadIdx.x; e < n2; e += kThreads)
                s_key[e] = e < c ? ((unsigned long long)sort_key(bk, beg + e) << 32) | (unsigned)e : ~0ull;
            __syncthreads();
            for (int k = 2; k <= n2; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int t = threadIdx.x; t < n2; t += kThreads) {
                        const int u = t ^ j;
                        if (u > t) {
                            const unsigned long long x = s_key[t], y = s_key[u];
                            if ((x > y) == ((t & k) == 0)) { s_key[t] = y; s_key[u] = x; }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int q = threadIdx.x; q < c; q += kThreads) {
                const int e = beg + (int)(s_key[q] & 0xffffffffu);
                bk.col_b[beg + q] = bk.col_a[e];
                bk.w_b[beg + q] = bk.w_a[e];
                bk.om_b[beg + q] = bk.om_a[e];
                bk.fl_b[beg + q] = bk.fl_a[e];
            }
        } else {
            // (a) every chunk of kSortSmem entries sorted in shared memory into the b arrays
            for (int q0 = 0; q0 < c; q0 += kSortSmem) {
                const int cn = min(kSortSmem, c - q0);
                int n2 = 1;
                while (n2 < cn) n2 <<= 1;
                __syncthreads();
                for (int e = threadIdx.x; e < n2; e += kThreads)
                    s_key[e] = e < cn ? ((unsigned long long)sort_key(bk, beg + q0 + e) << 32) | (unsigned)e : ~0ull;
                __syncthreads();
                for (int k = 2; k <= n2; k <<= 1) {
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        for (int t = threadIdx.x; t < n2; t += kThreads) {
                            const int u = t ^ j;
                            if (u > t) {
                                const unsigned long long x = s_key[t], y = s_key[u];
                                if ((x > y) == ((t & k) == 0)) { s_key[t] = y; s_key[u] = x; }
                            }
                        }
                        __syncthreads();
                    }
                }
                for (int q = threadIdx.x; q < cn; q += kThreads) {
                    const int e = beg + q0 + (int)(s_key[q] & 0xffffffffu);
                    bk.col_b[beg + q0 + q] = bk.col_a[e];
                    bk.w_b[beg + q0 + q] = bk.w_a[e];
                    bk.om_b[beg + q0 + q] = bk.om_a[e];
                    bk.fl_b[beg + q0 + q] = bk.fl_a[e];
                }
            }
            __syncthreads();
            // (b) the rank of each entry in the row: its place in its own chunk plus, in every
            // other chunk, the number of keys below its own (a binary search; the keys are
            // distinct); the entry moves to that place in the a arrays (no longer needed)
            const int nck = (c + kSortSmem - 1) / kSortSmem;
            for (int e = threadIdx.x; e < c; e += kThreads) {
                const int qc = e / kSortSmem;
                const unsigned ke = sort_key_b(bk, beg + e);
                int rank = e - qc * kSortSmem;
                for (int r = 0; r < nck; ++r) {
                    if (r == qc) continue;
                    int lo = r * kSortSmem, hi = min(c, lo + kSortSmem);
                    const int first = lo;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (sort_key_b(bk, beg + mid) < ke) lo = mid + 1;
                        else hi = mid;
                    }
                    rank += lo - first;
                }
                bk.col_a[beg + rank] = bk.col_b[beg + e];
                bk.w_a[beg + rank] = bk.w_b[beg + e];
                bk.om_a[beg + rank] = bk.om_b[beg + e];
                bk.fl_a[beg + rank] = bk.fl_b[beg + e];
            }
            __syncthreads();
            for (int e = threadIdx.x; e < c; e += kThreads) {
                bk.col_b[beg + e] = bk.col_a[beg + e];
                bk.w_b[beg + e] = bk.w_a[beg + e];
                bk.om_b[beg + e] = bk.om_a[beg + e];
                bk.fl_b[beg + e] = bk.fl_a[beg + e];
            }
        }
        __syncthreads();
        // de-dup in place, chunk by chunk (a chunk only writes at or before the
        // positions it read, and the predecessor it compares with keeps its value)
        if (threadIdx.x == 0) s_out = 0;
        for (int c0 = 0; c0 < c; c0 += kThreads) {
            const int e = c0 + threadIdx.x;
            int col = 0;
            T w = T(0), om = T(0);
            unsigned char fl = 0;
            bool keep = false;
            if (e < c) {
                col = bk.col_b[beg + e];
                w = bk.w_b[beg + e];
                om = bk.om_b[beg + e];
                fl = bk.fl_b[beg + e];
                keep = !((fl & kEntMirror) && e > 0 && bk.col_b[beg + e - 1] == col);
            }
            const unsigned bal = __ballot_sync(kFull, keep);
            if (lane == 0) s_cnt[warp] = __popc(bal);
            __syncthreads();
            int before = s_out;
            for (int w2 = 0; w2 < warp; ++w2) before += s_cnt[w2];
            int total = 0;
            for (int w2 = 0; w2 < kWarps; ++w2) total += s_cnt[w2];
            const int q = before + __popc(bal & ((1u << lane) - 1u));
            if (keep) {
                bk.col_b[beg + q] = col;
                bk.w_b[beg + q] = w;
                bk.om_b[beg + q] = om;
                bk.fl_b[beg + q] = fl;
            }
            push_mirrors(bk, ctrl, keep && (fl & kEntMirror), beg + q, i, lane);
            __syncthreads();
            if (threadIdx.x == 0) s_out += total;
            __syncthreads();
        }
        if (threadIdx.x == 0) bk.len[i] = s_out;
    }
    __syncthreads();   // sm is reused by what follows in a fused launch
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bucket_sort(Buckets<T> bk, int p, Ctrl* ctrl) {
    __shared__ SortSmem sm;
    bucket_sort_body(bk, p, ctrl, ctrl->flags, blockIdx.x, gridDim.x, sm);
}

// W_ij for partner entries, one thread per entry of the fill list, by gathers in
// the CSR order of row i: diagonal term first, then the off-diagonals ascending
// (bitwise equal to the value the screening pass computes for that entry).
template <typename T>
__device__ void fill_w_body(const T* __restrict__ S, int64_t ld, const Csr<T>& om, const int4* __restrict__ rinfo,
                            const T* __restrict__ rdv, const Buckets<T>& bk, const Ctrl* ctrl, int flags0, int bid,
                            int nb) {
    if (flags0) return;
    const int nm = ctrl->n_mirror;
    for (int k = bid * kThreads + threadIdx.x; k < nm; k += nb * kThreads) {
        const int2 m = bk.mir[k];
        const int i = m.y;
        const int j = bk.col_b[m.x];
        const int4 ri = rinfo[i];
        T acc = mulT(rdv[i], S[(int64_t)i * ld + j]);
        for (int q = ri.x; q < ri.y; ++q)
            if (q != ri.z) acc = fmaT(om.cv[q], S[(int64_t)om.ci[q] * ld + j], acc);
        bk.w_b[m.x] = acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fill_w(const T* __restrict__ S, int64_t ld, Csr<T> om, const int4* __restrict__ rinfo, const T* __restrict__ rdv,
         Buckets<T> bk, const Ctrl* ctrl) {
    fill_w_body(S, ld, om, rinfo, rdv, bk, ctrl, ctrl->flags, blockIdx.x, gridDim.x);
}

// G_ij of one entry (position q of row i) and its share of the objective partials.
template <typename T, typename A>
__device__ __forceinline__ void gradient_entry(const Buckets<T>& bk, int i, int q, T lam1, T lam2, A& s_ow, A& s_o2,
                                               A& s_log, A& s_abs, int& bad) {
    const int j = bk.col_b[q];
    const T wij = bk.w_b[q];
    const T om = bk.om_b[q];
    const unsigned char fl = bk.fl_b[q];
    // W_ji: binary search for column i in row j
    const int jb = bk.off[j];
    int lo = 0, hi = bk.len[j] - 1, pos = -1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int cm = bk.col_b[jb + mid];
        if (cm == i) { pos = mid; break; }
        if (cm < i) lo = mid + 1; else hi = mid - 1;
    }
    if (pos < 0) { bad |= kFlagBadStructure; return; }
    const T wji = bk.w_b[jb + pos];
    // G_ij = (W_ij + W_ji)/2 + lambda2 w_ij - [i=j]/w_ii, one fixed rounding sequence
    T g = fmaT(lam2, om, T(0.5) * (wij + wji));
    if (i == j) g -= T(1) / om;
    bk.g[q] = g;
    const bool keep = (fl & kEntSupp) || (i == j) || !(fabs(g) <= lam1);
    if (keep) bk.fl_b[q] = fl | kEntKeep;
    if (!(g == g) || isinf((double)g)) bad |= kFlagNaN;
    if (fl & kEntSupp) {
        acc_add(s_ow, mulT(om, wij));
        acc_add(s_o2, mulT(om, om));
        if (i == j) acc_add(s_log, logT(om)); else acc_add(s_abs, fabs(om));
    }
}

// G on the candidates (Alg. 2 steps 5-6) and the objective partials of Omega^k:
// short rows one lane each, long rows (from the bucket scan's list) one warp each.
template <typename T>
__device__ void gradient_body(int p, const Buckets<T>& bk, int stride, double* part_obj, Ctrl* ctrl, int flags0,
                              int bid, int nb, double (&red)[kWarps][4]) {
    using A = typename AccOf<T>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = (bid * kThreads + threadIdx.x) >> 5;
    const int nw = (nb * kThreads) >> 5;
    const bool skip = flags0 != 0;
    const T lam1 = (T)ctrl->lam1, lam2 = (T)ctrl->lam2;
    const int nlong = skip ? 0 : ctrl->n_long;
    A s_ow{}, s_o2{}, s_log{}, s_abs{};
    int bad = 0;
    for (int base = skip ? p : gw * 32; base < p; base += nw * 32) {
        const int i = base + lane;
        if (i < p && bk.cnt[i] <= kShortRow) {
            const int beg = bk.off[i], L = bk.len[i];
            for (int e = 0; e < L; ++e) gradient_entry(bk, i, beg + e, lam1, lam2, s_ow, s_o2, s_log, s_abs, bad);
        }
    }
    for (int li = gw; li < nlong; li += nw) {
        const int i = bk.longlist[li];
        const int beg = bk.off[i], L = bk.len[i];
        for (int e = lane; e < L; e += 32) gradient_entry(bk, i, beg + e, lam1, lam2, s_ow, s_o2, s_log, s_abs, bad);
    }
    if (bad) atomicOr(&ctrl->flags, bad);
    s_ow = warp_sum(s_ow); s_o2 = warp_sum(s_o2); s_log = warp_sum(s_log); s_abs = warp_sum(s_abs);
    if (lane == 0) {
        red[warp][0] = acc_value(s_ow); red[warp][1] = acc_value(s_o2);
        red[warp][2] = acc_value(s_log); red[warp][3] = acc_value(s_abs);
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double a = 0.0;
        for (int w = 0; w < kWarps; ++w) a += red[w][threadIdx.x];
        part_obj[(size_t)threadIdx.x * stride + bid] = a;
    }
    __syncthreads();   // red is reused by what follows in a fused launch
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gradient(int p, Buckets<T> bk, int stride, double* part_obj, Ctrl* ctrl) {
    __shared__ double red[kWarps][4];
    gradient_body(p, bk, stride, part_obj, ctrl, ctrl->flags, blockIdx.x, gridDim.x, red);
}

// ------------------------------------------------------------------ 3. line search
constexpr int kMaxWindow = 16;

// What the last block of a line-search launch needs for the decision.
struct LsDecide {
    const double* part_obj;     // objective partials of the current iterate (k_gradient)
    int n_obj;                  // their count per quantity
    int stride;                 // quantity stride of both partial arrays
    int max_halvings;
    double tau0;
    int use_cond;               // 1: set the line-search loop's graph condition
    cudaGraphConditionalHandle cond;
};
template <int M>
__device__ void ls_finish(const double* __restrict__ part_ls, int n_ls, const LsDecide& d, Ctrl* ctrl);

// Row i of the unit-offset prefix containing unit u (uoff[i] <= u < uoff[i+1]): a
// 32-way search by the whole warp (each step narrows the range 32-fold).
__device__ __forceinline__ int find_unit_row(const long long* uoff, int p, long long u, int lane) {
    int lo = 0, hi = p;
    while (hi - lo > 1) {
        const int span = hi - lo;
        const int q = lo + (int)(((long long)span * (lane + 1)) >> 5);
        const bool le = lane < 31 && uoff[q] <= u;
        const unsigned bal = __ballot_sync(kFull, le);
        const int c = __popc(bal);
        const int nlo = c ? __shfl_sync(kFull, q, c - 1) : lo;
        const int nhi = c < 31 ? __shfl_sync(kFull, q, c) : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// tau = 2^-h in T, exactly (what ldexp(1, -h) rounds to, denormals and 0 included).
template <typename T> __device__ __forceinline__ T tau_pow2(int h);
template <> __device__ __forceinline__ float tau_pow2<float>(int h) {
    return h <= 126 ? __int_as_float((127 - h) << 23) : (h <= 149 ? __int_as_float(1 << (149 - h)) : 0.f);
}
template <> __device__ __forceinline__ double tau_pow2<double>(int h) {
    return h <= 1022 ? __longlong_as_double((long long)(1023 - h) << 52)
                     : (h <= 1074 ? __longlong_as_double(1ll << (1074 - h)) : 0.0);
}

__device__ __forceinline__ F2 to_acc(float x) { F2 a; a.hi = x; return a; }
__device__ __forceinline__ double to_acc(double x) { return x; }
__device__ __forceinline__ void acc_merge(F2& a, const F2& b) { acc_add(a, b.hi); a.lo = __fadd_rn(a.lo, b.lo); }
__device__ __forceinline__ void acc_merge(double& a, double b) { a += b; }

// Partials per block and per tau of the window, stored quantity-major
// (part_ls[(4 m + k) * stride + block]):
//   [0] sum_{e,f} D_e D_f S_{j_e j_f}   (= tr(D S D) restricted to row i, summed over rows)
//   [1] ||D||_F^2                       [2] sum_i phi(D_ii / w_ii)     [3] #{w+_ii <= 0}
// The quadratic form of row i is split into work units, the pairs (a <= b) of its
// 32-entry chunks; every warp takes an equal contiguous range of the units of all
// rows (prefix uoff), so rows with thousands of candidates spread over many warps.
// Terms [1]-[3] are per entry: each diagonal unit (a = b) warp-reduces them into
// the warp's shared accumulators, which keeps the register count (and so the
// number of resident warps on a persistent grid) where the gathers need it: three
// CTAs per SM for windows of up to 4 step sizes, two for wider ones.
template <typename T, int M>
struct LsSmem {
    using A = typename AccOf<T>::type;
    int col[kWarps][32];
    T del[kWarps][M][32];
    A acc[kWarps][M][2];
    int nb[kWarps][M];
    double red[kWarps][M][4];
};

template <typename T, int M>
__device__ void ls_eval_body(const T* __restrict__ S, int64_t ld, int p, const Buckets<T>& bk, int stride,
                             double* part_ls, Ctrl* ctrl, int flags0, int bid, int nblocks, LsSmem<T, M>& sm) {
    using A = typename AccOf<T>::type;
    auto& s_col = sm.col;
    auto& s_del = sm.del;
    auto& s_acc = sm.acc;
    auto& s_nb = sm.nb;
    auto& red = sm.red;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gw = (bid * (long long)kThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)nblocks * kThreads) >> 5;
    const bool skip = (flags0 != 0) || (ctrl->ls_accept >= 0);
    const T lam1 = (T)ctrl->lam1;
    const int h_base = ctrl->ls_base;
    if (lane < M) {
        s_acc[warp][lane][0] = A{};
        s_acc[warp][lane][1] = A{};
        s_nb[warp][lane] = 0;
    }
    __syncwarp();
    A q[M]{};

    // 1. short rows (at most kShortRow entries), one lane each: the quadratic form
    //    of a row with entries e0, e1 is d0^2 S_00 + d1^2 S_11 + 2 d0 d1 S_01
    for (int base = skip ? p : (int)gw * 32; base < p; base += (int)nw * 32) {
        const int i = base + lane;
        int L = 0, beg = 0;
        if (i < p && bk.cnt[i] <= kShortRow) {
            L = bk.len[i];
            beg = bk.off[i];
        }
        int j0 = 0, j1 = 0;
        T om0 = T(1), g0 = T(0), om1 = T(1), g1 = T(0);
        if (L >= 1) { j0 = bk.col_b[beg]; om0 = bk.om_b[beg]; g0 = bk.g[beg]; }
        if (L >= 2) { j1 = bk.col_b[beg + 1]; om1 = bk.om_b[beg + 1]; g1 = bk.g[beg + 1]; }
        const T s00 = L >= 1 ? S[(int64_t)j0 * ld + j0] : T(0);
        const T s11 = L >= 2 ? S[(int64_t)j1 * ld + j1] : T(0);
        const T s01 = L >= 2 ? S[(int64_t)j0 * ld + j1] : T(0);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const T tau = tau_pow2<T>(h_base + m);
            const T n0 = prox_entry(om0, g0, tau, tau * lam1, j0 == i);
            const T n1 = prox_entry(om1, g1, tau, tau * lam1, j1 == i);
            const T d0 = L >= 1 ? n0 - om0 : T(0);
            const T d1 = L >= 2 ? n1 - om1 : T(0);
            T qf = mulT(mulT(d0, d0), s00);
            qf = fmaT(mulT(d1, d1), s11, qf);
            qf = fmaT(T(2) * mulT(d0, d1), s01, qf);
            acc_add(q[m], qf);
            A n2 = to_acc(mulT(d0, d0));
            acc_add(n2, mulT(d1, d1));
            T ph = T(0);
            bool bad = false;
            if (L >= 1 && j0 == i) { if (!(n0 > T(0))) bad = true; else ph = phiT(d0 / om0); }
            if (L >= 2 && j1 == i) { if (!(n1 > T(0))) bad = true; else ph = phiT(d1 / om1); }
            const A n2w = warp_sum(n2);
            const A phw = warp_sum(to_acc(ph));
            const int nbad = __popc(__ballot_sync(kFull, bad));
            if (lane == 0) {
                acc_merge(s_acc[warp][m][0], n2w);
                acc_merge(s_acc[warp][m][1], phw);
                s_nb[warp][m] += nbad;
            }
        }
    }

    // 2. long rows: equal ranges of the work units of the long-row list
    const int nlong = skip ? 0 : ctrl->n_long;
    const long long U = nlong > 0 ? bk.uoff[nlong] : 0;
    long long u = U * gw / nw;
    const long long u1 = U * (gw + 1) / nw;
    int li = u < u1 ? find_unit_row(bk.uoff, nlong, u, lane) : 0;
    while (u < u1) {
        while (bk.uoff[li + 1] <= u) ++li;
        const int i = bk.longlist[li];
        const long long uend = min(bk.uoff[li + 1], u1);
        const int tc = (bk.cnt[i] + 31) >> 5;
        int k = (int)(u - bk.uoff[li]);
        int a = 0;
        while (k >= tc - a) { k -= tc - a; ++a; }
        int cb = a + k;
        const int beg = bk.off[i], L = bk.len[i];
        for (; u < uend; ++u) {
            const int eb = a * 32, fb = cb * 32;
            const bool diag_unit = (a == cb);
            if (fb < L) {
                const int e = eb + lane;
                T de[M];
                int je = 0;
                bool act_e = false;
                {
                    T om = T(0), g = T(0);
                    bool diag = false;
                    if (e < L) {
                        je = bk.col_b[beg + e];
                        om = bk.om_b[beg + e];
                        g = bk.g[beg + e];
                        diag = (je == i);
                    }
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const T tau = tau_pow2<T>(h_base + m);
                        const T np_ = prox_entry(om, g, tau, tau * lam1, diag);
                        de[m] = e < L ? np_ - om : T(0);
                        act_e |= (de[m] != T(0));
                    }
                    if (diag_unit) {
                        // per-entry terms of this chunk: ||D||^2, phi(D_ii / w_ii), #{w+_ii <= 0}
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            T ph = T(0);
                            bool bad = false;
                            if (diag) {
                                const T np_ = om + de[m];
                                if (!(np_ > T(0))) bad = true;
                                else ph = phiT(de[m] / om);
                            }
                            const A n2 = warp_sum(to_acc(mulT(de[m], de[m])));
                            const A pp = warp_sum(to_acc(ph));
                            const int nbad = __popc(__ballot_sync(kFull, bad));
                            if (lane == 0) {
                                acc_merge(s_acc[warp][m][0], n2);
                                acc_merge(s_acc[warp][m][1], pp);
                                s_nb[warp][m] += nbad;
                            }
                        }
                    }
                }
                __syncwarp();
                {
                    const int f = fb + lane;
                    int jf = -1;
                    if (f < L) {
                        jf = bk.col_b[beg + f];
                        const T om = bk.om_b[beg + f], g = bk.g[beg + f];
                        bool act = false;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const T tau = tau_pow2<T>(h_base + m);
                            const T d = prox_entry(om, g, tau, tau * lam1, jf == i) - om;
                            s_del[warp][m][lane] = d;
                            act |= (d != T(0));
                        }
                        if (!act) jf = -1;
                    } else {
#pragma unroll
                        for (int m = 0; m < M; ++m) s_del[warp][m][lane] = T(0);
                    }
                    s_col[warp][lane] = jf;
                }
                __syncwarp();
                if (act_e) {
                    T qf[M];
#pragma unroll
                    for (int m = 0; m < M; ++m) qf[m] = T(0);
                    const T* srow = S + (int64_t)je * ld;
#pragma unroll 4
                    for (int t = 0; t < 32; ++t) {
                        const int jf = s_col[warp][t];
                        const bool use = jf >= 0 && (!diag_unit || t >= lane);
                        const T sv = use ? srow[jf] : T(0);
                        const T wgt = (diag_unit && t == lane) ? T(1) : T(2);
#pragma unroll
                        for (int m = 0; m < M; ++m) qf[m] = fmaT(wgt * de[m] * s_del[warp][m][t], sv, qf[m]);
                    }
#pragma unroll
                    for (int m = 0; m < M; ++m) acc_add(q[m], qf[m]);
                }
            }
            if (++cb == tc) { ++a; cb = a; }
        }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const A a = warp_sum(q[m]);
        if (lane == 0) {
            red[warp][m][0] = acc_value(a);
            red[warp][m][1] = acc_value(s_acc[warp][m][0]);
            red[warp][m][2] = acc_value(s_acc[warp][m][1]);
            red[warp][m][3] = (double)s_nb[warp][m];
        }
    }
    __syncthreads();
    if (threadIdx.x < M * 4) {
        const int m = threadIdx.x / 4, k = threadIdx.x % 4;
        double a = 0.0;
        for (int w = 0; w < kWarps; ++w) a += red[w][m][k];
        part_ls[(size_t)(m * 4 + k) * stride + bid] = a;
    }
    __syncthreads();   // sm is reused by what follows in a fused launch
}

template <typename T, int M>
__global__ void __launch_bounds__(kThreads, (M <= 4) ? 3 : 2)
k_ls_eval(const T* __restrict__ S, int64_t ld, int p, Buckets<T> bk, int stride, double* part_ls,
          Ctrl* ctrl, LsDecide dec) {
    __shared__ LsSmem<T, M> sm;
    ls_eval_body<T, M>(S, ld, p, bk, stride, part_ls, ctrl, ctrl->flags, blockIdx.x, gridDim.x, sm);
    ls_finish<M>(part_ls, (int)gridDim.x, dec, ctrl);
}

// Obs form of the line-search partials (Alg. 3 step 11): tr(D S D) restricted to
// row i is ||X D_i||^2 / n with X D_i = sum_e D_e X^T[j_e, :]; lanes hold 4
// consecutive samples of each 128-sample chunk of n.  [1]-[3] as in k_ls_eval.
template <int M>
__device__ void ls_eval_obs_body(const float* __restrict__ Xt, int64_t ldx, int64_t n, int p,
                                 const Buckets<float>& bk, double tau0, int stride, double* part_ls, Ctrl* ctrl,
                                 int flags0, int bid, int nblocks, double (&red)[kWarps][M][4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = (bid * kThreads + threadIdx.x) >> 5;
    const int nw = (nblocks * kThreads) >> 5;
    const bool skip = (flags0 != 0) || (ctrl->ls_accept >= 0);
    const float lam1 = (float)ctrl->lam1;
    const int h_base = ctrl->ls_base;
    float tau[M], tl1[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        tau[m] = (float)ldexp(tau0, -(h_base + m));
        tl1[m] = tau[m] * lam1;
    }
    F2 q[M]{}, n2[M]{}, ph[M]{};
    int nb[M];
#pragma unroll
    for (int m = 0; m < M; ++m) nb[m] = 0;
    for (int i = skip ? p : gw; i < p; i += nw) {
        const int beg = bk.off[i], L = bk.len[i];
        for (int e = lane; e < L; e += 32) {
            const int je = bk.col_b[beg + e];
            const float om = bk.om_b[beg + e], g = bk.g[beg + e];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const float np_ = prox_entry(om, g, tau[m], tl1[m], je == i);
                const float d = np_ - om;
                acc_add(n2[m], mulT(d, d));
                if (je == i) {
                    if (!(np_ > 0.f)) nb[m] += 1;
                    else acc_add(ph[m], phiT(d / om));
                }
            }
        }
        for (int64_t c0 = 0; c0 < n; c0 += 128) {
            const int64_t c = c0 + lane * 4;
            float u[M][4];
#pragma unroll
            for (int m = 0; m < M; ++m) u[m][0] = u[m][1] = u[m][2] = u[m][3] = 0.f;
            bool any = false;
            for (int e = 0; e < L; ++e) {
                const int je = bk.col_b[beg + e];
                const float om = bk.om_b[beg + e], g = bk.g[beg + e];
                float d[M];
                bool act = false;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    d[m] = prox_entry(om, g, tau[m], tl1[m], je == i) - om;
                    act |= d[m] != 0.f;
                }
                if (!act) continue;
                any = true;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (c < ldx) x = __ldg(reinterpret_cast<const float4*>(Xt + (int64_t)je * ldx + c));
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    u[m][0] = fmaf(d[m], x.x, u[m][0]);
                    u[m][1] = fmaf(d[m], x.y, u[m][1]);
                    u[m][2] = fmaf(d[m], x.z, u[m][2]);
                    u[m][3] = fmaf(d[m], x.w, u[m][3]);
                }
            }
            if (!any) break;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                float sq = u[m][0] * u[m][0];
                sq = fmaf(u[m][1], u[m][1], sq);
                sq = fmaf(u[m][2], u[m][2], sq);
                sq = fmaf(u[m][3], u[m][3], sq);
                acc_add(q[m], sq);
            }
        }
    }
    const double inv_n = 1.0 / (double)n;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const F2 a = warp_sum(q[m]), b = warp_sum(n2[m]), c = warp_sum(ph[m]);
        int dd = nb[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(kFull, dd, o);
        if (lane == 0) {
            red[warp][m][0] = acc_value(a) * inv_n; red[warp][m][1] = acc_value(b);
            red[warp][m][2] = acc_value(c); red[warp][m][3] = (double)dd;
        }
    }
    __syncthreads();
    if (threadIdx.x < M * 4) {
        const int m = threadIdx.x / 4, k = threadIdx.x % 4;
        double a = 0.0;
        for (int w = 0; w < kWarps; ++w) a += red[w][m][k];
        part_ls[(size_t)(m * 4 + k) * stride + bid] = a;
    }
    __syncthreads();   // red is reused by what follows in a fused launch
}

template <int M>
__global__ void __launch_bounds__(kThreads)
k_ls_eval_obs(const float* __restrict__ Xt, int64_t ldx, int64_t n, int p, Buckets<float> bk, double tau0,
              int stride, double* part_ls, Ctrl* ctrl, LsDecide dec) {
    __shared__ double red[kWarps][M][4];
    ls_eval_obs_body<M>(Xt, ldx, n, p, bk, tau0, stride, part_ls, ctrl, ctrl->flags, blockIdx.x, gridDim.x, red);
    ls_finish<M>(part_ls, (int)gridDim.x, dec, ctrl);
}

// The sufficient-decrease decision of one window (thread 0 of the last block of k_ls_eval).
__device__ void decide_window(const double* sums, const double* obj, int M, int h_base, int max_halvings,
                              double tau0, double lam1, double lam2, int first, Ctrl* ctrl) {
    if (first) {
        // f = -sum log w_ii + tr(Omega S Omega)/2 + lambda2/2 ||Omega||^2, tr = sum w_ij W_ij
        ctrl->f_cur = -obj[2] + 0.5 * obj[0] + 0.5 * lam2 * obj[1];
        ctrl->pen_cur = lam1 * obj[3];
        ctrl->norm2_cur = obj[1];
    }
    for (int m = 0; m < M; ++m) {
        const int h = h_base + m;
        if (h > max_halvings) break;
        const double tau = ldexp(tau0, -h);
        const double qd = sums[m * 4 + 0], n2 = sums[m * 4 + 1], ph = sums[m * 4 + 2], nb = sums[m * 4 + 3];
        if (nb != 0.0) continue;                       // a diagonal entry left the domain
        const double excess = 0.5 * qd + 0.5 * lam2 * n2 + ph;
        if (excess <= n2 / (2.0 * tau)) {
            ctrl->ls_accept = h;
            ctrl->tau = tau;
            ctrl->delta2 = n2;
            ctrl->ls_trials += h + 1;
            return;
        }
        if (!(excess == excess)) { ctrl->flags |= kFlagNaN; return; }
    }
    ctrl->ls_base = h_base + M;
    if (h_base + M > max_halvings) ctrl->flags |= kFlagLsFail;
}

// The last block of a line-search launch to finish (every block has written its
// partials) reduces them in a fixed order -- one warp per quantity, lanes over
// strided blocks, then a butterfly -- and takes the decision of Alg. 1 step 9; the
// other blocks return.  The order does not depend on which block is last.
template <int M>
struct FinSmem {
    double sums[M * 4];
    double obj[4];
};

// Whole block: the window's partials (and, in the first window, the objective
// partials) reduced in the fixed order into sm; thread 0 then takes the decision
// (decide_window).  Called with no flag raised and nothing accepted yet.
template <int M>
__device__ void ls_reduce_decide(const double* part_ls, int n_ls, const LsDecide& d, Ctrl* ctrl, FinSmem<M>& sm) {
    double* sums = sm.sums;
    double* obj = sm.obj;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = kWarps;
    const int h_base = ctrl->ls_base;
    const int first = h_base == 0;
    const double lam1 = ctrl->lam1, lam2 = ctrl->lam2;
    const int nq = M * 4 + (first ? 4 : 0);
    for (int q = warp; q < nq; q += nwarps) {
        double a = 0.0;
        // eight loads in flight per lane; the additions keep their order
        if (q < M * 4) {
#pragma unroll 8
            for (int b = lane; b < n_ls; b += 32) a += __ldcg(part_ls + (size_t)q * d.stride + b);
        } else {
#pragma unroll 8
            for (int b = lane; b < d.n_obj; b += 32) a += __ldcg(d.part_obj + (size_t)(q - M * 4) * d.stride + b);
        }
        a = warp_sum(a);
        if (lane == 0) {
            if (q < M * 4) sums[q] = a; else obj[q - M * 4] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctrl->ls_windows += 1;
        decide_window(sums, obj, M, h_base, d.max_halvings, d.tau0, lam1, lam2, first, ctrl);
    }
    __syncthreads();
}

template <int M>
__device__ void ls_finish(const double* __restrict__ part_ls, int n_ls, const LsDecide& d, Ctrl* ctrl) {
    __shared__ int s_last;
    __shared__ FinSmem<M> sm;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctrl->ls_done, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (ctrl->flags != 0 || ctrl->ls_accept >= 0) {
        if (threadIdx.x == 0) {
            ctrl->ls_done = 0;
            if (d.use_cond) cudaGraphSetConditional(d.cond, 0);
        }
        return;
    }
    ls_reduce_decide<M>(part_ls, n_ls, d, ctrl, sm);
    if (threadIdx.x != 0) return;
    ctrl->ls_done = 0;
    // another window while nothing is accepted and nothing went wrong
    if (d.use_cond) cudaGraphSetConditional(d.cond, (ctrl->flags == 0 && ctrl->ls_accept < 0) ? 1u : 0u);
}

// ------------------------------------------------------------------ 4. accept
// Entries of the accepted iterate: the diagonal, and every candidate the prox
// at the accepted tau leaves nonzero.  Short rows one lane each, long rows one
// warp each.
template <typename T>
__device__ void compact_count_body(int p, const Buckets<T>& bk, int* cnt2, const Ctrl* ctrl, int flags0, int bid,
                                   int nb) {
    const int lane = threadIdx.x & 31;
    const int gw = (bid * kThreads + threadIdx.x) >> 5;
    const int nw = (nb * kThreads) >> 5;
    if (flags0 != 0 || ctrl->ls_accept < 0) return;
    const T tau = (T)ctrl->tau;
    const T tl1 = tau * (T)ctrl->lam1;
    const int nlong = ctrl->n_long;
    for (int base = gw * 32; base < p; base += nw * 32) {
        const int i = base + lane;
        if (i < p && bk.cnt[i] <= kShortRow) {
            const int beg = bk.off[i], L = bk.len[i];
            int c = 0;
            for (int e = 0; e < L; ++e) {
                const int j = bk.col_b[beg + e];
                const T v = prox_entry(bk.om_b[beg + e], bk.g[beg + e], tau, tl1, j == i);
                c += ((j == i) || (v != T(0))) ? 1 : 0;
            }
            cnt2[i] = c;
        }
    }
    for (int li = gw; li < nlong; li += nw) {
        const int i = bk.longlist[li];
        const int beg = bk.off[i], L = bk.len[i];
        int c = 0;
        for (int base = 0; base < L; base += 32) {
            const int e = base + lane;
            bool nz = false;
            if (e < L) {
                const int j = bk.col_b[beg + e];
                const T v = prox_entry(bk.om_b[beg + e], bk.g[beg + e], tau, tl1, j == i);
                nz = (j == i) || (v != T(0));
            }
            c += __popc(__ballot_sync(kFull, nz));
        }
        if (lane == 0) cnt2[i] = c;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_compact_count(int p, Buckets<T> bk, int* cnt2, const Ctrl* ctrl) {
    compact_count_body(p, bk, cnt2, ctrl, ctrl->flags, blockIdx.x, gridDim.x);
}

template <typename T>
__device__ void compact_write_body(int p, const Buckets<T>& bk, const Csr<T>& nx, int cap, const Ctrl* ctrl,
                                   int flags0, int bid, int nb) {
    const int lane = threadIdx.x & 31;
    const int gw = (bid * kThreads + threadIdx.x) >> 5;
    const int nw = (nb * kThreads) >> 5;
    if (flags0 != 0 || ctrl->ls_accept < 0) return;
    const T tau = (T)ctrl->tau;
    const T tl1 = tau * (T)ctrl->lam1;
    const int nlong = ctrl->n_long;
    for (int base = gw * 32; base < p; base += nw * 32) {
        const int i = base + lane;
        if (i < p && bk.cnt[i] <= kShortRow) {
            const int beg = bk.off[i], L = bk.len[i];
            int out = nx.rp[i];
            for (int e = 0; e < L; ++e) {
                const int j = bk.col_b[beg + e];
                const T v = prox_entry(bk.om_b[beg + e], bk.g[beg + e], tau, tl1, j == i);
                if ((j == i) || (v != T(0))) {
                    if (out < cap) { nx.ci[out] = j; nx.cv[out] = v; }
                    ++out;
                }
            }
        }
    }
    for (int li = gw; li < nlong; li += nw) {
        const int i = bk.longlist[li];
        const int beg = bk.off[i], L = bk.len[i];
        int out = nx.rp[i];
        for (int base = 0; base < L; base += 32) {
            const int e = base + lane;
            bool nz = false;
            int j = 0;
            T v = T(0);
            if (e < L) {
                j = bk.col_b[beg + e];
                v = prox_entry(bk.om_b[beg + e], bk.g[beg + e], tau, tl1, j == i);
                nz = (j == i) || (v != T(0));
            }
            const unsigned bal = __ballot_sync(kFull, nz);
            if (nz) {
                const int q = out + __popc(bal & ((1u << lane) - 1u));
                if (q < cap) { nx.ci[q] = j; nx.cv[q] = v; }
            }
            out += __popc(bal);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_compact_write(int p, Buckets<T> bk, Csr<T> nx, int cap, const Ctrl* ctrl) {
    compact_write_body(p, bk, nx, cap, ctrl, ctrl->flags, blockIdx.x, gridDim.x);
}

template <typename T>
__global__ void k_set_identity(Csr<T> c, int p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= p; i += gridDim.x * blockDim.x) {
        c.rp[i] = i;
        if (i < p) { c.ci[i] = i; c.cv[i] = T(1); }
    }
}

template <typename T, typename V>
__global__ void k_csr_export(const int* rp, const int* ci, const T* cv, int p, int nnz, int64_t* rp64,
                             int32_t* co, V* vo) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nnz || t <= p; t += gridDim.x * blockDim.x) {
        if (t <= p) rp64[t] = rp[t];
        if (t < nnz) { co[t] = ci[t]; vo[t] = (V)cv[t]; }
    }
}

__global__ void k_gather_s(const void* S, int is_f64, int64_t ld, int64_t m, const int64_t* rows,
                           const int64_t* cols, double* out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = rows[t] * ld + cols[t];
        out[t] = is_f64 ? static_cast<const double*>(S)[o] : (double)static_cast<const float*>(S)[o];
    }
}

// ------------------------------------------------------------------ 5. the fused iteration tail
// One cooperative launch runs steps 2-4 of an outer iteration: the candidate
// structure (count, scan, scatter, sort, partner fill), the gradient G on it
// (Alg. 2 steps 5-6), the line-search windows -- prox of eq. (2), the objective
// partials and the sufficient-decrease decision of Alg. 1 step 9 -- until a step
// is accepted, then the compaction of the accepted iterate into CSR and the
// stopping rule.  Every phase is the device function the separate kernels of
// the chain run, so each entry gets the same bits; grid-wide barriers stand where
// the chain has kernel boundaries.  The cooperative launch keeps every block of
// the grid resident, and every wait is bounded: a barrier that waits longer than
// kBarrierWaitNs raises kFlagTimeout, after which every block skips the remaining
// phases.

__device__ __forceinline__ long long tail_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *static_cast<const volatile int*>(p); }

constexpr long long kBarrierWaitNs = 4000000000ll;   // 4 s

// Barrier bookkeeping of one block, and the control block's state after a barrier.
struct TailSync {
    unsigned* count;             // the launch's arrival counter
    unsigned target;             // arrivals that complete this block's current barrier
    int last;
    int pre_flags, pre_accept;   // as the last block to arrive sees them
    int flags, accept;           // after the release
};
struct TailState {
    int flags;
    int accept;
};

__device__ __forceinline__ void tail_sync_init(TailSync& ss, unsigned* bar) {
    if (threadIdx.x != 0) return;
    ss.count = bar;
    ss.target = 0u;
}

// Grid-wide barrier over the launch's nb blocks on one arrival counter that only
// grows within the launch (k_iter_begin zeroes it before each iteration): the
// barrier is complete when the counter reaches the block's target, which grows
// by nb per barrier.  With a hook, the last block to arrive runs at_last (the
// whole block, with the state it read) and then adds one more arrival, which is
// what the others wait for.  Ordering: the arrival is an acq_rel atomic after the
// block's writes (CTA barrier first) and the waits are acquire loads, so every
// block leaves with the writes of every block before the barrier (and of the
// hook) visible.  A wait longer than kBarrierWaitNs, or a timeout raised
// elsewhere, raises kFlagTimeout and ends the wait.  (Measured on GB300: one such
// barrier over 304 blocks costs about what a kernel boundary inside a CUDA graph
// does; a two-level form with 16 group counters was slower.)
template <bool HOOK, typename F>
__device__ TailState grid_barrier_impl(Ctrl* ctrl, int nb, TailSync& ss, F&& at_last) {
    __syncthreads();
    if (threadIdx.x == 0) {
        ss.target += (unsigned)nb;
        const unsigned target = ss.target + (HOOK ? 1u : 0u);
        const unsigned prev = atom_add_acq_rel_gpu(ss.count, 1u);
        ss.last = prev + 1u == ss.target;
        if (ss.last && HOOK) {
            ss.pre_flags = ld_volatile_int(&ctrl->flags);
            ss.pre_accept = ld_volatile_int(&ctrl->ls_accept);
        } else if (!ss.last) {
            const long long t0 = tail_clock_ns();
            unsigned polls = 0;
            while ((int)(ld_acquire_gpu(ss.count) - target) < 0) {
                if ((++polls & 63u) == 0u &&
                    ((ld_volatile_int(&ctrl->flags) & kFlagTimeout) || tail_clock_ns() - t0 > kBarrierWaitNs)) {
                    atomicOr(&ctrl->flags, kFlagTimeout);
                    break;
                }
                __nanosleep(20);
            }
        }
        if (HOOK) ss.target += 1u;
    }
    __syncthreads();
    if (HOOK && ss.last) {
        at_last(ss.pre_flags, ss.pre_accept);
        __syncthreads();
        if (threadIdx.x == 0) atom_add_acq_rel_gpu(ss.count, 1u);
    }
    if (threadIdx.x == 0) {
        ss.flags = ld_volatile_int(&ctrl->flags);
        ss.accept = ld_volatile_int(&ctrl->ls_accept);
    }
    __syncthreads();
    return TailState{ss.flags, ss.accept};
}

template <typename F>
__device__ __forceinline__ TailState grid_barrier(Ctrl* ctrl, int nb, TailSync& ss, F&& at_last) {
    return grid_barrier_impl<true>(ctrl, nb, ss, at_last);
}

__device__ __forceinline__ TailState grid_barrier(Ctrl* ctrl, int nb, TailSync& ss) {
    return grid_barrier_impl<false>(ctrl, nb, ss, [](int, int) {});
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// Shared memory of the fused kernel: one phase at a time uses it.
template <typename T, int M, bool OBS>
constexpr size_t tail_smem_bytes() {
    return cmax(cmax(sizeof(ScanSmem), sizeof(SortSmem)),
                cmax(cmax(sizeof(double) * kWarps * 4, sizeof(FinSmem<M>)),
                     OBS ? sizeof(double) * kWarps * M * 4 : sizeof(LsSmem<T, M>)));
}

// Steps of the tail, each over the whole grid of the launch that runs it.
// 2. candidates and the gradient (ends with the objective partials written, one
//    per block of this grid).
template <typename T>
__device__ TailState tail_candidates(const IterBufs<T>& b, TailSync& ss, unsigned char* smem) {
    Ctrl* ctrl = b.ctrl;
    const int bid = blockIdx.x, nb = gridDim.x;
    const int p = b.p;
    const int ntiles = (int)(((int64_t)p + kScanTile - 1) / kScanTile);
    auto& scan_sm = *reinterpret_cast<ScanSmem*>(smem);
    const Buckets<T>& bk = b.bk;
    bucket_count_body(b.em, bk, ctrl, bid, nb);
    TailState st = grid_barrier(ctrl, nb, ss);
    if (!(st.flags & kFlagTimeout))
        for (int t = bid; t < ntiles; t += nb) scan_reduce_tile(bk.cnt, p, st.flags, true, b.scan_part, t, scan_sm);
    st = grid_barrier(ctrl, nb, ss);
    if (!(st.flags & kFlagTimeout))
        for (int t = bid; t < ntiles; t += nb)
            scan_apply_tile(bk.cnt, bk.off, p, bk.cap, ctrl, st.flags, kFlagBucketOverflow, &ctrl->bucket_total,
                            bk.uoff, bk.longlist, b.scan_part, -1, 0.0, t, ntiles, scan_sm);
    st = grid_barrier(ctrl, nb, ss);
    bucket_scatter_body(b.em, bk, ctrl, st.flags, bid, nb);
    st = grid_barrier(ctrl, nb, ss);
    bucket_sort_body(bk, p, ctrl, st.flags, bid, nb, *reinterpret_cast<SortSmem*>(smem));
    st = grid_barrier(ctrl, nb, ss);
    fill_w_body(b.S, b.ld, b.cur, b.rinfo, b.rdv, bk, ctrl, st.flags, bid, nb);
    st = grid_barrier(ctrl, nb, ss);
    gradient_body(p, bk, b.nblk, b.part_obj, ctrl, st.flags, bid, nb, *reinterpret_cast<double(*)[kWarps][4]>(smem));
    return st;
}

// 4. the accepted iterate into CSR (count, scan with the stopping rule, write),
//    entered with no flag raised and a step accepted.
template <typename T>
__device__ void tail_accept(const IterBufs<T>& b, TailSync& ss, unsigned char* smem, TailState st) {
    Ctrl* ctrl = b.ctrl;
    const int bid = blockIdx.x, nb = gridDim.x;
    const int p = b.p;
    const int ntiles = (int)(((int64_t)p + kScanTile - 1) / kScanTile);
    auto& scan_sm = *reinterpret_cast<ScanSmem*>(smem);
    compact_count_body(p, b.bk, b.cnt2, ctrl, st.flags, bid, nb);
    st = grid_barrier(ctrl, nb, ss);
    if (!(st.flags & kFlagTimeout))
        for (int t = bid; t < ntiles; t += nb) scan_reduce_tile(b.cnt2, p, st.flags, false, b.scan_part, t, scan_sm);
    st = grid_barrier(ctrl, nb, ss);
    if (!(st.flags & kFlagTimeout))
        for (int t = bid; t < ntiles; t += nb)
            scan_apply_tile(b.cnt2, b.next.rp, p, 0x7fffffff, ctrl, st.flags, 0, nullptr, nullptr, nullptr,
                            b.scan_part, b.csr_cap, b.eps, t, ntiles, scan_sm);
    st = grid_barrier(ctrl, nb, ss);
    compact_write_body(p, b.bk, b.next, b.csr_cap, ctrl, st.flags, bid, nb);
}

// The whole tail in one launch: candidates, gradient, every window (the last
// block at a window's barrier reduces the partials and decides), accept.
template <typename T, int M, bool OBS>
__global__ void __launch_bounds__(kThreads, OBS ? 1 : 2)
k_iter_tail(IterBufs<T> b) {
    __shared__ __align__(16) unsigned char smem[tail_smem_bytes<T, M, OBS>()];
    __shared__ TailSync ss;
    tail_sync_init(ss, b.bar);
    Ctrl* ctrl = b.ctrl;
    const int bid = blockIdx.x, nb = gridDim.x;
    TailState st = tail_candidates<T>(b, ss, smem);
    st = grid_barrier(ctrl, nb, ss);
    // 3. line-search windows until a step is accepted or a flag is raised
    const LsDecide dec{b.part_obj, nb, b.nblk, b.max_halvings, 1.0, 0, 0};
    while (st.flags == 0 && st.accept < 0) {
        if constexpr (OBS) {
            ls_eval_obs_body<M>(b.xt, b.ldx, b.n, b.p, b.bk, 1.0, b.nblk, b.part_ls, ctrl, st.flags, bid, nb,
                                *reinterpret_cast<double(*)[kWarps][M][4]>(smem));
        } else {
            ls_eval_body<T, M>(b.S, b.ld, b.p, b.bk, b.nblk, b.part_ls, ctrl, st.flags, bid, nb,
                               *reinterpret_cast<LsSmem<T, M>*>(smem));
        }
        st = grid_barrier(ctrl, nb, ss, [&](int f, int acc) {
            if (f == 0 && acc < 0) ls_reduce_decide<M>(b.part_ls, nb, dec, ctrl, *reinterpret_cast<FinSmem<M>*>(smem));
        });
    }
    if (st.flags != 0 || st.accept < 0) return;
    tail_accept<T>(b, ss, smem, st);
}

}  // namespace

// ------------------------------------------------------------------ launchers
template <typename T>
void launch_iter_begin(const IterBufs<T>& b, const LoopCond& lc, cudaStream_t s) {
    k_iter_begin<T><<<64, 256, 0, s>>>(b.bk, b.p, b.ctrl, lc.use, lc.ls, b.bar);
}

// Prefix of the folded tile sequence of the screening pass (seqoff, nc+1 entries)
// and its grid: one CTA per SM, more while some CTA's share would span more row
// chunks than its shared-memory row cache holds.
template <typename T>
int screen_plan(int p, int num_sms, std::vector<long long>& seqoff) {
    constexpr int R = kScreenTileRows;
    constexpr int BJ = 32 * (16 / (int)sizeof(T));
    const int nc = (p + R - 1) / R;
    const int nb = (p + BJ - 1) / BJ;
    seqoff.assign(nc + 1, 0);
    for (int q = 0; q < nc; ++q) {
        const int c = screen_seq_chunk(q, nc);
        seqoff[q + 1] = seqoff[q] + (nb - (int)((long long)c * R / BJ));
    }
    const long long total = seqoff[nc];
    auto last_le = [&](long long x) {
        return (int)(std::upper_bound(seqoff.begin(), seqoff.begin() + nc, x) - seqoff.begin()) - 1;
    };
    long long G = std::max<long long>(1, std::min<long long>(total, num_sms));
    for (;;) {
        int span = 0;
        for (long long g = 0; g < G; ++g) {
            const long long lo = total * g / G, hi = total * (g + 1) / G;
            if (hi > lo) span = std::max(span, last_le(hi - 1) - last_le(lo) + 1);
        }
        if (span <= kScreenMaxChunks || G >= total) break;
        G = std::min<long long>(total, G + num_sms);
    }
    return (int)G;
}

template <typename T>
void launch_grad_screen(const IterBufs<T>& b, cudaStream_t s) {
    constexpr int smem = screen_smem_bytes<T>();
    set_smem_once((const void*)k_grad_screen<T>, smem, sizeof(T) == 8 ? kSmemSlotScreenD : kSmemSlotScreenF);
    const int warps_grid = b.num_sms * 4;
    // one row per thread (the column maxima need every row of a block in one CTA)
    k_row_info<T><<<(b.p + 255) / 256, 256, 0, s>>>(b.p, b.cur, b.rinfo, b.rdv, b.pmask, b.offlist, b.ctrl,
                                                     b.m1 ? static_cast<T*>(b.colmax) : nullptr, b.nbm);
    // two-level item selection when the group maxima exist and the column maxima fit
    // in shared memory (and the item count fits an int)
    const int ngr = b.nbm / 8;
    const size_t ps_smem = (size_t)(b.nbm + ngr) * sizeof(T);
    const bool grp = b.m1 && b.m1g && ps_smem <= 48 * 1024 && (long long)b.p * ((ngr + 7) / 8) < (1ll << 30);
    k_pair_select<T><<<b.num_sms * 8, kThreads, grp ? ps_smem : 0, s>>>(
        b.S, b.ld, b.p, b.nbm, b.m1, grp ? b.m1g : nullptr, b.ngl, b.rinfo, b.rdv, b.colmax, b.pairs, b.pairs_cap,
        b.em, b.ctrl);
    if (b.m1)
        k_pair_screen<T><<<warps_grid, kThreads, 0, s>>>(b.S, b.ld, b.p, b.pairs, b.pairs_cap, b.rinfo, b.rdv, b.pmask,
                                                         b.em, b.ctrl);
    k_grad_screen<T><<<b.screen_grid, kScreenThreads, smem, s>>>(*b.smap, b.p, b.seqoff, b.rinfo, b.rdv, b.pmask,
                                                                 b.m1 ? b.pairs_cap : -1, b.em, b.ctrl);
    if (b.m1) {
        const int ngroups_max = (b.p + 7) / 8;
        const int grid = std::max(1, std::min(ngroups_max, b.num_sms * 4));
        const size_t words = (size_t)kWarps * ((b.nbm + 31) / 32) * sizeof(unsigned);
        if (b.nbm % 8 == 0)
            k_rows_items<T, true><<<grid, kThreads, words, s>>>(b.p, b.nbm, b.m1, b.rinfo, b.rdv, b.offlist, b.cur.ci,
                                                                b.cur.cv, b.row_items, b.row_items_cap, b.ctrl);
        else
            k_rows_items<T, false><<<grid, kThreads, words, s>>>(b.p, b.nbm, b.m1, b.rinfo, b.rdv, b.offlist,
                                                                 b.cur.ci, b.cur.cv, b.row_items, b.row_items_cap,
                                                                 b.ctrl);
    }
    const int rows_ctas = std::max(1, std::min(4, b.rows_ctas_per_sm));
    if (rows_ctas >= 3)
        k_grad_screen_rows<T, 3><<<b.num_sms * rows_ctas, kThreads, 0, s>>>(
            b.S, b.ld, b.p, b.rinfo, b.rdv, b.offlist, b.cur.ci, b.cur.cv, b.m1 ? b.row_items : nullptr,
            b.row_items_cap, b.em, b.ctrl);
    else
        k_grad_screen_rows<T, 2><<<b.num_sms * rows_ctas, kThreads, 0, s>>>(
            b.S, b.ld, b.p, b.rinfo, b.rdv, b.offlist, b.cur.ci, b.cur.cv, b.m1 ? b.row_items : nullptr,
            b.row_items_cap, b.em, b.ctrl);
}

// Group maxima of the block maxima: m1g[i][g] = max over the blocks 8g .. 8g+7 of
// m1[i][.].  For non-negative BF16 values (and the NaN pattern 0x7fc0, above +inf)
// the order of the bit patterns is the order of the values, so an unsigned maximum
// is exact and keeps NaN.  One thread per (row, group): one 16-byte load.
__global__ void k_group_max(const unsigned short* __restrict__ m1, int p, int nbm, unsigned short* __restrict__ m1g,
                            int ngl) {
    const int ng = nbm / 8;
    const long long total = (long long)p * ng;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / ng), g = (int)(t - (long long)i * ng);
        const uint4 v = *reinterpret_cast<const uint4*>(m1 + (int64_t)i * nbm + 8 * g);
        const unsigned m = max(max(max(v.x & 0xffffu, v.x >> 16), max(v.y & 0xffffu, v.y >> 16)),
                               max(max(v.z & 0xffffu, v.z >> 16), max(v.w & 0xffffu, v.w >> 16)));
        m1g[(int64_t)i * ngl + g] = (unsigned short)m;
    }
}

void launch_group_max(const unsigned short* m1, int p, int nbm, unsigned short* m1g, int ngl, cudaStream_t s) {
    const long long total = (long long)p * (nbm / 8);
    const int blocks = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152 * 32));
    k_group_max<<<blocks, 256, 0, s>>>(m1, p, nbm, m1g, ngl);
}

template <typename T>
void launch_rowblock_max(const T* S, int64_t ld, int p, int nbm, unsigned short* m1, cudaStream_t s) {
    k_rowblock_max<T><<<std::max(1, std::min((p + 7) / 8, 152 * 16)), kThreads, 0, s>>>(S, ld, p, nbm, m1);
}

template <typename T>
void launch_row_info(int p, Csr<T> om, int4* rinfo, T* rdv, cudaStream_t s) {
    k_row_info<T><<<(p + 255) / 256, 256, 0, s>>>(p, om, rinfo, rdv, nullptr, nullptr, nullptr, nullptr, 0);
}

// Blocks of k_gradient: one objective partial each (read back by ls_finish).
template <typename T>
static int gradient_grid(const IterBufs<T>& b) {
    return std::max(1, std::min(b.nblk, b.num_sms * 4));
}

template <typename T>
void launch_candidates(const IterBufs<T>& b, cudaStream_t s) {
    const int g = 152 * 4;
    k_bucket_count<T><<<g, 256, 0, s>>>(b.em, b.bk, b.ctrl);
    launch_scan(b.bk.cnt, b.bk.off, b.p, b.bk.cap, b.ctrl, kFlagBucketOverflow, &b.ctrl->bucket_total, b.bk.uoff,
                b.bk.longlist, b.scan_part, s);
    k_bucket_scatter<T><<<g, 256, 0, s>>>(b.em, b.bk, b.ctrl);
    k_bucket_sort<T><<<b.nblk, kThreads, 0, s>>>(b.bk, b.p, b.ctrl);
    k_fill_w<T><<<b.num_sms * 8, kThreads, 0, s>>>(b.S, b.ld, b.cur, b.rinfo, b.rdv, b.bk, b.ctrl);
    k_gradient<T><<<gradient_grid(b), kThreads, 0, s>>>(b.p, b.bk, b.nblk, b.part_obj, b.ctrl);
}

// Persistent grid of the line-search evaluation: resident blocks x SMs (at most
// nblk, the partial arrays' stride).
template <typename T, int M>
static int ls_eval_grid(const IterBufs<T>& b) {
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_ls_eval<T, M>, kThreads, 0) != cudaSuccess || v < 1)
            v = 1;
        per_sm = v;
    }
    const int want = b.ls_blocks_per_sm > 0 ? std::min(b.ls_blocks_per_sm, per_sm) : per_sm;
    return std::max(1, std::min(b.nblk, want * b.num_sms));
}

template <typename T>
static LsDecide ls_decide_args(const IterBufs<T>& b, const LoopCond& lc) {
    return LsDecide{b.part_obj, gradient_grid(b), b.nblk, b.max_halvings, 1.0, lc.use, lc.ls};
}

template <typename T, int M>
static int ls_eval_m(const IterBufs<T>& b, const LoopCond& lc, cudaStream_t s) {
    const int g = ls_eval_grid<T, M>(b);
    k_ls_eval<T, M><<<g, kThreads, 0, s>>>(b.S, b.ld, b.p, b.bk, b.nblk, b.part_ls, b.ctrl, ls_decide_args(b, lc));
    return g;
}

static int window_m(int M) { return M == 1 || M == 2 || M == 4 || M == 8 ? M : 16; }

template <typename T>
void launch_ls_window(const IterBufs<T>& b, const LoopCond& lc, cudaStream_t s) {
    const int M = window_m(b.ls_window);
    // one launch per window: its last block to finish takes the decision (ls_finish)
    switch (M) {
        case 1: ls_eval_m<T, 1>(b, lc, s); break;
        case 2: ls_eval_m<T, 2>(b, lc, s); break;
        case 4: ls_eval_m<T, 4>(b, lc, s); break;
        case 8: ls_eval_m<T, 8>(b, lc, s); break;
        default: ls_eval_m<T, 16>(b, lc, s); break;
    }
}

template <int M>
static void ls_eval_obs_m(const IterBufs<float>& b, const LoopCond& lc, cudaStream_t s) {
    k_ls_eval_obs<M><<<b.nblk, kThreads, 0, s>>>(b.xt, b.ldx, b.n, b.p, b.bk, 1.0, b.nblk, b.part_ls, b.ctrl,
                                                 ls_decide_args(b, lc));
}

void launch_ls_window_obs(const IterBufs<float>& b, const LoopCond& lc, cudaStream_t s) {
    const int M = window_m(b.ls_window);
    switch (M) {
        case 1: ls_eval_obs_m<1>(b, lc, s); break;
        case 2: ls_eval_obs_m<2>(b, lc, s); break;
        case 4: ls_eval_obs_m<4>(b, lc, s); break;
        case 8: ls_eval_obs_m<8>(b, lc, s); break;
        default: ls_eval_obs_m<16>(b, lc, s); break;
    }
}

template <typename T>
void launch_accept(const IterBufs<T>& b, cudaStream_t s) {
    k_compact_count<T><<<b.nblk, kThreads, 0, s>>>(b.p, b.bk, b.cnt2, b.ctrl);
    launch_scan(b.cnt2, b.next.rp, b.p, 0x7fffffff, b.ctrl, 0, nullptr, nullptr, nullptr, b.scan_part, s, b.csr_cap,
                b.eps);
    k_compact_write<T><<<b.nblk, kThreads, 0, s>>>(b.p, b.bk, b.next, b.csr_cap, b.ctrl);
}

// The fused tail's grid: resident blocks per SM (capped by the tuning's
// ls_blocks_per_sm, as for the window kernel) x SMs, at most nblk (the stride of
// the partial arrays).  0 if the kernel cannot be resident at all.
template <typename T, int M, bool OBS>
static int tail_grid_m(const IterBufs<T>& b) {
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_iter_tail<T, M, OBS>, kThreads, 0) != cudaSuccess)
            v = 0;
        per_sm = std::max(0, v);
    }
    if (per_sm < 1) return 0;
    const int want = b.ls_blocks_per_sm > 0 ? std::min(b.ls_blocks_per_sm, per_sm) : per_sm;
    return std::max(1, std::min(b.nblk, want * b.num_sms));
}

template <typename T, int M, bool OBS>
static cudaError_t tail_m(const IterBufs<T>& b, cudaStream_t s) {
    const int g = tail_grid_m<T, M, OBS>(b);
    if (g < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_iter_tail<T, M, OBS>, b);
}

template <typename T, bool OBS>
static cudaError_t tail_window(const IterBufs<T>& b, cudaStream_t s, int* grid) {
    switch (window_m(b.ls_window)) {
        case 1: return grid ? (*grid = tail_grid_m<T, 1, OBS>(b), cudaSuccess) : tail_m<T, 1, OBS>(b, s);
        case 2: return grid ? (*grid = tail_grid_m<T, 2, OBS>(b), cudaSuccess) : tail_m<T, 2, OBS>(b, s);
        case 4: return grid ? (*grid = tail_grid_m<T, 4, OBS>(b), cudaSuccess) : tail_m<T, 4, OBS>(b, s);
        case 8: return grid ? (*grid = tail_grid_m<T, 8, OBS>(b), cudaSuccess) : tail_m<T, 8, OBS>(b, s);
        default: return grid ? (*grid = tail_grid_m<T, 16, OBS>(b), cudaSuccess) : tail_m<T, 16, OBS>(b, s);
    }
}

template <typename T>
static cudaError_t tail_dispatch(const IterBufs<T>& b, bool obs, cudaStream_t s, int* grid) {
    if constexpr (std::is_same<T, float>::value) {
        if (obs) return tail_window<float, true>(b, s, grid);
    } else {
        if (obs) return cudaErrorInvalidValue;
    }
    return tail_window<T, false>(b, s, grid);
}

template <typename T>
cudaError_t launch_tail(const IterBufs<T>& b, bool obs, cudaStream_t s) {
    return tail_dispatch<T>(b, obs, s, nullptr);
}

template <typename T>
int tail_grid(const IterBufs<T>& b, bool obs) {
    int g = 0;
    return tail_dispatch<T>(b, obs, nullptr, &g) == cudaSuccess ? g : 0;
}

// A cooperative launch of one block that counts itself and, inside a graph,
// ends its conditional loop: the device-loop capture checks with it once that
// cooperative kernels can run in a conditional node's body.
__global__ void k_tail_probe(int* out, int use_cond, cudaGraphConditionalHandle cond) {
    if (threadIdx.x == 0) {
        atomicAdd(out, 1);
        if (use_cond) cudaGraphSetConditional(cond, 0u);
    }
}

cudaError_t launch_tail_probe(int* out, cudaGraphConditionalHandle cond, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tail_probe, out, 1, cond);
}

template <typename T>
void launch_commit(const IterBufs<T>& b, const LoopCond& lc, cudaStream_t s) {
    k_csr_commit<T><<<b.num_sms * 2, 256, 0, s>>>(b.next, b.cur, b.p, b.ctrl, lc.use, lc.iter);
}

void launch_stamp(Ctrl* ctrl, int end, cudaStream_t s) { k_stamp<<<1, 1, 0, s>>>(ctrl, end); }

// ------------------------------------------------------------------ lambda path in one launch
__device__ __forceinline__ long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ __forceinline__ int status_of_flags(int f) {
    if (f & kFlagNaN) return HPC_ERR_NAN;
    if (f & kFlagLsFail) return HPC_ERR_LS_FAIL;
    if (f & kFlagTimeout) return HPC_ERR_DEVICE_TIMEOUT;
    return HPC_ERR_CUDA;
}

// Start point pt of the path: its lambda1, fresh counters (unless the point resumes
// after a host-side regrow), and the iteration loop armed.
__global__ void k_point_begin(Ctrl* ctrl, PathOut out, cudaGraphConditionalHandle iter_cond) {
    ctrl->path_pt = ctrl->path_pt_next;
    ctrl->path_off = ctrl->path_off_next;
    const int pt = ctrl->path_pt;
    ctrl->lam1 = out.lam1[pt];
    if (!ctrl->path_keep) {
        ctrl->iter = 0;
        ctrl->ls_trials = 0;
        ctrl->converged = 0;
        ctrl->t_point = globaltimer_ns();
    }
    ctrl->path_keep = 0;
    cudaGraphSetConditional(iter_cond, ctrl->iter_limit > ctrl->iter ? 1u : 0u);
}

// End of point pt: its statistics, optionally a copy of the estimate, and the
// decision to go on.  Every block reads the point index and the staging offset,
// which only the next k_point_begin advances.  An overflow flag ends the launch
// without advancing: the host grows the buffers and resumes this point.
template <typename T>
__global__ void k_point_end(Csr<T> cu, int p, PathOut out, Ctrl* ctrl, cudaGraphConditionalHandle path_cond) {
    const int flags = ctrl->flags;
    const int pt = ctrl->path_pt;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = gridDim.x * blockDim.x;
    const bool overflow = flags & (kFlagEmOverflow | kFlagBucketOverflow | kFlagNnzOverflow);
    if (overflow) {
        if (tid == 0) cudaGraphSetConditional(path_cond, 0u);
        return;
    }
    const long long nnz = ctrl->nnz_cur;
    const long long base = ctrl->path_off;
    const bool fits = base + nnz <= out.cap;
    if (out.rp && fits) {
        int64_t* rp = out.rp + (size_t)pt * (p + 1);
        for (int i = tid; i <= p; i += nt) rp[i] = cu.rp[i];
        for (long long q = tid; q < nnz; q += nt) {
            out.ci[base + q] = cu.ci[q];
            out.cv[base + q] = (float)cu.cv[q];
        }
    }
    if (tid != 0) return;
    hpc_path_point r;
    r.lambda1 = out.lam1[pt];
    r.iterations = ctrl->iter;
    r.ls_trials = ctrl->ls_trials;
    r.nnz = nnz;
    r.status = flags ? status_of_flags(flags) : (ctrl->converged ? HPC_OK : HPC_NOT_CONVERGED);
    r.pad_ = 0;
    r.f = ctrl->f_cur;
    r.F = ctrl->f_cur + ctrl->pen_cur;
    r.rel_change = ctrl->rel;
    r.ms = 1e-6 * (double)(globaltimer_ns() - ctrl->t_point);
    out.points[pt] = r;
    bool more = flags == 0 && pt + 1 < out.k;
    if (out.rp) {
        if (fits) {
            ctrl->path_off_next = base + nnz;
        } else {
            ctrl->path_need = base + nnz;
            ctrl->path_full = 1;
            more = false;
        }
    }
    ctrl->path_pt_next = pt + 1;
    cudaGraphSetConditional(path_cond, more ? 1u : 0u);
}

void launch_point_begin(Ctrl* ctrl, PathOut out, const LoopCond& lc, cudaStream_t s) {
    k_point_begin<<<1, 1, 0, s>>>(ctrl, out, lc.iter);
}

template <typename T>
void launch_point_end(const IterBufs<T>& b, PathOut out, cudaGraphConditionalHandle path_cond, cudaStream_t s) {
    k_point_end<T><<<b.num_sms * 2, 256, 0, s>>>(b.cur, b.p, out, b.ctrl, path_cond);
}

template <typename T>
void launch_set_identity(Csr<T> c, int p, cudaStream_t s) {
    k_set_identity<T><<<64, 256, 0, s>>>(c, p);
}

template <typename T>
void launch_csr_export(const int* rp, const int* ci, const T* cv, int p, int nnz, int64_t* rp64,
                       int32_t* co, void* val, int vdt, cudaStream_t s) {
    if (vdt == HPC_F64)
        k_csr_export<T, double><<<256, 256, 0, s>>>(rp, ci, cv, p, nnz, rp64, co, static_cast<double*>(val));
    else
        k_csr_export<T, float><<<256, 256, 0, s>>>(rp, ci, cv, p, nnz, rp64, co, static_cast<float*>(val));
}

void launch_gather_s(const void* S, int is_f64, int64_t ld, int64_t m, const int64_t* rows,
                     const int64_t* cols, double* out, cudaStream_t s) {
    k_gather_s<<<128, 256, 0, s>>>(S, is_f64, ld, m, rows, cols, out);
}

#define HPC_INSTANTIATE(T)                                                                       \
    template void launch_iter_begin<T>(const IterBufs<T>&, const LoopCond&, cudaStream_t);         \
    template void launch_commit<T>(const IterBufs<T>&, const LoopCond&, cudaStream_t);             \
    template void launch_point_end<T>(const IterBufs<T>&, PathOut, cudaGraphConditionalHandle, cudaStream_t); \
    template void launch_grad_screen<T>(const IterBufs<T>&, cudaStream_t);                         \
    template void launch_candidates<T>(const IterBufs<T>&, cudaStream_t);                          \
    template void launch_ls_window<T>(const IterBufs<T>&, const LoopCond&, cudaStream_t);          \
    template void launch_accept<T>(const IterBufs<T>&, cudaStream_t);                              \
    template cudaError_t launch_tail<T>(const IterBufs<T>&, bool, cudaStream_t);                     \
    template int tail_grid<T>(const IterBufs<T>&, bool);                                             \
    template void launch_set_identity<T>(Csr<T>, int, cudaStream_t);                               \
    template void launch_row_info<T>(int, Csr<T>, int4*, T*, cudaStream_t);                        \
    template void launch_rowblock_max<T>(const T*, int64_t, int, int, unsigned short*, cudaStream_t); \
    template int screen_plan<T>(int, int, std::vector<long long>&);                                 \
    template void launch_csr_export<T>(const int*, const int*, const T*, int, int, int64_t*, int32_t*, \
                                       void*, int, cudaStream_t);

HPC_INSTANTIATE(float)
HPC_INSTANTIATE(double)

}  // namespace hpc
