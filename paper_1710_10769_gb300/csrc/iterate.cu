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
#include <cstdio>

#include "internal.cuh"

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
__global__ void k_iter_begin(Buckets<T> bk, int p, Ctrl* ctrl) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = tid; i < p; i += gridDim.x * blockDim.x) {
        bk.cnt[i] = 0;
        bk.cur[i] = 0;
    }
    if (tid == 0) {
        ctrl->em_count = 0;
        ctrl->bucket_total = 0;
        ctrl->flags = 0;
        ctrl->ls_accept = -1;
        ctrl->ls_base = 0;
        ctrl->nnz_next = 0;
        ctrl->converged = 0;
        ctrl->tau = 0.0;
        ctrl->delta2 = 0.0;
    }
}

// ------------------------------------------------------------------ 1. screening SpMM
// Grid: x = chunks of 128 rows, y = column blocks of BJ = 32*V columns.  x runs
// fastest, so the CTAs in flight share a few column blocks S[:, J] (p*BJ*sizeof(T)
// bytes each), which stay in L2 while every row gathers its d rows of them: S is
// read from HBM about once per pass.  Lane l of a warp holds columns J*BJ + l*V
// .. +V-1 and loads them as one 16-byte vector per CSR entry.  A warp owns 16
// consecutive rows and walks their CSR entries as one stream, kScreenUnroll
// loads in flight at a time; when the stream crosses a row boundary the
// finished row is screened and its emitted entries appended.
constexpr int kScreenRowsPerWarp = 16;
constexpr int kScreenRows = kScreenRowsPerWarp * kWarps;
constexpr int kScreenUnroll = 8;

template <typename T>
struct ScreenRow {
    static constexpr int V = 16 / sizeof(T);
    static constexpr int BJ = 32 * V;

    // Screen row i of the block: emit the support entries, the diagonal and every
    // |W_ij| > lambda1 (NaN included).  Warp-collective.
    static __device__ __forceinline__ void finalize(int i, int rb, int re, const T (&acc)[V], int j0, int p,
                                                    const int* __restrict__ ci, const T* __restrict__ cv, T lam1,
                                                    const Emit<T>& em, Ctrl* ctrl, int lane) {
        unsigned mbits = 0;
        T om[V];
        bool big = false;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            om[v] = T(0);
            big |= !(fabs(acc[v]) <= lam1);
        }
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
        if (!__any_sync(kFull, big || mbits != 0)) return;
        bool emit[V];
        int c = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = j0 + lane * V + v;
            emit[v] = (j < p) && (((mbits >> v) & 1u) || !(fabs(acc[v]) <= lam1));
            c += emit[v] ? 1 : 0;
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
            if (emit[v]) {
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

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_grad_screen(const T* __restrict__ S, int64_t ld, int p, const int* __restrict__ rp,
              const int* __restrict__ ci, const T* __restrict__ cv, T lam1, Emit<T> em,
              Ctrl* __restrict__ ctrl) {
    using R = ScreenRow<T>;
    constexpr int V = R::V;
    constexpr int BJ = R::BJ;
    constexpr int U = kScreenUnroll;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = blockIdx.y * BJ;
    const int rbase = blockIdx.x * kScreenRows + warp * kScreenRowsPerWarp;
    if (rbase >= p) return;
    const int nr = min(kScreenRowsPerWarp, p - rbase);
    const T* sblk = S + j0 + lane * V;
    // lanes 0..nr hold the row pointers of the warp's rows (lane nr: end of the last row)
    const int my_rp = (lane <= nr) ? rp[rbase + lane] : 0;
    const int e_beg = __shfl_sync(kFull, my_rp, 0);
    const int e_end = __shfl_sync(kFull, my_rp, nr);
    int cur = 0;
    int cur_beg = e_beg;
    int cur_end = __shfl_sync(kFull, my_rp, 1);
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = T(0);

    for (int eb = e_beg; eb < e_end; eb += 32) {
        const int e = eb + lane;
        const int k_l = (e < e_end) ? ci[e] : 0;
        const T w_l = (e < e_end) ? cv[e] : T(0);
        const int cnt = min(32, e_end - eb);
        for (int t = 0; t < cnt; t += U) {
            const int g = min(U, cnt - t);          // entries in this group
            const int gbase = eb + t;               // stream index of the group's first entry
            T sv[U][V];
            T wv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (u < g) {
                    const int k = __shfl_sync(kFull, k_l, t + u);
                    wv[u] = __shfl_sync(kFull, w_l, t + u);
                    vload(sv[u], sblk + (int64_t)k * ld);
                }
            }
            int u0 = 0;
            while (true) {
                // entries [u0, stop) of the group belong to row cur (CSR order kept)
                const int stop = min(g, cur_end - gbase);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (u >= u0 && u < stop) {
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = fmaT(wv[u], sv[u][v], acc[v]);
                    }
                }
                u0 = max(u0, stop);
                if (u0 >= g) break;
                // the stream left row cur: screen it and move on
                R::finalize(rbase + cur, cur_beg, cur_end, acc, j0, p, ci, cv, lam1, em, ctrl, lane);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = T(0);
                ++cur;
                cur_beg = cur_end;
                cur_end = __shfl_sync(kFull, my_rp, cur + 1);
            }
        }
    }
    while (cur < nr) {
        R::finalize(rbase + cur, cur_beg, cur_end, acc, j0, p, ci, cv, lam1, em, ctrl, lane);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = T(0);
        ++cur;
        cur_beg = cur_end;
        cur_end = __shfl_sync(kFull, my_rp, min(cur + 1, nr));
    }
}

// ------------------------------------------------------------------ 2. candidates
template <typename T>
__global__ void k_bucket_count(Emit<T> em, Buckets<T> bk, Ctrl* ctrl) {
    const int total = ctrl->em_count;
    if (total > em.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctrl->flags, kFlagEmOverflow);
        return;
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int i = em.row[e];
        const int cj = em.col[e];
        atomicAdd(&bk.cnt[i], 1);
        if (cj >= 0) atomicAdd(&bk.cnt[cj], 1);   // off the support: partner request in row j
    }
}

// Single-block exclusive scan of n ints (chunks of 4096), out[n] = total.
// If total > cap, sets flag.
__global__ void __launch_bounds__(1024)
k_scan(const int* __restrict__ in, int* __restrict__ out, int n, int cap, Ctrl* ctrl, int flag,
       int* total_dst) {
    __shared__ int wsum[32];
    __shared__ int carry;
    if (ctrl->flags & ~kFlagLsFail & (kFlagEmOverflow | kFlagBucketOverflow)) {
        if (threadIdx.x == 0) out[n] = 0;
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 4096) {
        const int idx = base + threadIdx.x * 4;
        int v[4];
        int s = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = (idx + q < n) ? in[idx + q] : 0;
            s += v[q];
        }
        const int x = warp_incl_scan(s, lane);
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int y = warp_incl_scan(wsum[lane], lane);
            wsum[lane] = y;
        }
        __syncthreads();
        int run = x - s + (warp ? wsum[warp - 1] : 0) + carry;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (idx + q < n) out[idx + q] = run;
            run += v[q];
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[n] = carry;
        if (total_dst) *total_dst = carry;
        if (carry > cap) atomicOr(&ctrl->flags, flag);
    }
}

template <typename T>
__global__ void k_bucket_scatter(Emit<T> em, Buckets<T> bk, const Ctrl* ctrl) {
    if (ctrl->flags) return;
    const int total = ctrl->em_count;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int i = em.row[e];
        const int cj = em.col[e];
        const int j = cj & 0x7fffffff;
        const int pos = bk.off[i] + atomicAdd(&bk.cur[i], 1);
        bk.col_a[pos] = j;
        bk.w_a[pos] = em.w[e];
        bk.om_a[pos] = em.om[e];
        bk.fl_a[pos] = (unsigned char)(kEntOwn | (cj < 0 ? kEntSupp : 0));
        if (cj >= 0) {
            const int q = bk.off[j] + atomicAdd(&bk.cur[j], 1);
            bk.col_a[q] = i;
            bk.w_a[q] = T(0);
            bk.om_a[q] = T(0);
            bk.fl_a[q] = kEntMirror;
        }
    }
}

// Warp per row: rank sort by (column, own-before-partner) into the b arrays, then
// drop partner requests whose own entry exists.  Rows are short (the support plus
// a few screened entries), so an O(c^2) rank sort is cheap and deterministic.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_bucket_sort(Buckets<T> bk, int p, const Ctrl* ctrl) {
    if (ctrl->flags) return;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < p; i += nw) {
        const int beg = bk.off[i];
        const int c = bk.cnt[i];
        for (int e = lane; e < c; e += 32) {
            const int ke = bk.col_a[beg + e] * 2 + ((bk.fl_a[beg + e] & kEntMirror) ? 1 : 0);
            int rank = 0;
            for (int f = 0; f < c; ++f) {
                const int kf = bk.col_a[beg + f] * 2 + ((bk.fl_a[beg + f] & kEntMirror) ? 1 : 0);
                rank += (kf < ke) ? 1 : 0;
            }
            bk.col_b[beg + rank] = bk.col_a[beg + e];
            bk.w_b[beg + rank] = bk.w_a[beg + e];
            bk.om_b[beg + rank] = bk.om_a[beg + e];
            bk.fl_b[beg + rank] = bk.fl_a[beg + e];
        }
        __syncwarp();
        int out = 0;
        for (int base = 0; base < c; base += 32) {
            const int e = base + lane;
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
            __syncwarp();
            if (keep) {
                const int q = out + __popc(bal & ((1u << lane) - 1u));
                bk.col_b[beg + q] = col;
                bk.w_b[beg + q] = w;
                bk.om_b[beg + q] = om;
                bk.fl_b[beg + q] = fl;
            }
            out += __popc(bal);
            __syncwarp();
        }
        if (lane == 0) bk.len[i] = out;
    }
}

// W_ij for partner entries, by gathers in the CSR order of row i (bitwise equal to
// the value the screening pass computes for that entry).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fill_w(const T* __restrict__ S, int64_t ld, int p, Csr<T> om, Buckets<T> bk, const Ctrl* ctrl) {
    if (ctrl->flags) return;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < p; i += nw) {
        const int beg = bk.off[i], L = bk.len[i];
        const int rb = om.rp[i], re = om.rp[i + 1];
        for (int e = lane; e < L; e += 32) {
            if (!(bk.fl_b[beg + e] & kEntMirror)) continue;
            const int j = bk.col_b[beg + e];
            T acc = T(0);
            for (int q = rb; q < re; ++q) acc = fmaT(om.cv[q], S[(int64_t)om.ci[q] * ld + j], acc);
            bk.w_b[beg + e] = acc;
        }
    }
}

// G on the candidates (Alg. 2 steps 5-6) and the objective partials of Omega^k.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gradient(int p, Buckets<T> bk, T lam1, T lam2, double* part_obj, Ctrl* ctrl) {
    __shared__ double red[kWarps][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const bool skip = ctrl->flags != 0;
    double s_ow = 0.0, s_o2 = 0.0, s_log = 0.0, s_abs = 0.0;
    int bad = 0;
    for (int i = skip ? p : gw; i < p; i += nw) {
        const int beg = bk.off[i], L = bk.len[i];
        for (int e = lane; e < L; e += 32) {
            const int j = bk.col_b[beg + e];
            const T wij = bk.w_b[beg + e];
            const T om = bk.om_b[beg + e];
            const unsigned char fl = bk.fl_b[beg + e];
            // W_ji: binary search for column i in row j
            const int jb = bk.off[j];
            int lo = 0, hi = bk.len[j] - 1, pos = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int cm = bk.col_b[jb + mid];
                if (cm == i) { pos = mid; break; }
                if (cm < i) lo = mid + 1; else hi = mid - 1;
            }
            if (pos < 0) { bad |= kFlagBadStructure; continue; }
            const T wji = bk.w_b[jb + pos];
            T g = T(0.5) * (wij + wji) + lam2 * om;
            if (i == j) g -= T(1) / om;
            bk.g[beg + e] = g;
            const bool keep = (fl & kEntSupp) || (i == j) || !(fabs(g) <= lam1);
            if (keep) bk.fl_b[beg + e] = fl | kEntKeep;
            if (!(g == g) || isinf((double)g)) bad |= kFlagNaN;
            if (fl & kEntSupp) {
                const double od = (double)om;
                s_ow += od * (double)wij;
                s_o2 += od * od;
                if (i == j) s_log += log(od); else s_abs += fabs(od);
            }
        }
    }
    if (bad) atomicOr(&ctrl->flags, bad);
    s_ow = warp_sum(s_ow); s_o2 = warp_sum(s_o2); s_log = warp_sum(s_log); s_abs = warp_sum(s_abs);
    if (lane == 0) { red[warp][0] = s_ow; red[warp][1] = s_o2; red[warp][2] = s_log; red[warp][3] = s_abs; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double a = 0.0;
        for (int w = 0; w < kWarps; ++w) a += red[w][threadIdx.x];
        part_obj[blockIdx.x * 4 + threadIdx.x] = a;
    }
}

// ------------------------------------------------------------------ 3. line search
constexpr int kMaxWindow = 16;
template <int M> __host__ __device__ constexpr int ls_chunk() { return M >= 16 ? 32 : 64; }

// Partials per block and per tau of the window:
//   [0] sum_{e,f} D_e D_f S_{j_e j_f}   (= tr(D S D) restricted to row i, summed over rows)
//   [1] ||D||_F^2                       [2] sum_i phi(D_ii / w_ii)     [3] #{w+_ii <= 0}
template <typename T, int M>
__global__ void __launch_bounds__(kThreads)
k_ls_eval(const T* __restrict__ S, int64_t ld, int p, Buckets<T> bk, T lam1, double tau0, int h_base,
          double* part_ls, const Ctrl* ctrl) {
    constexpr int kChunk = ls_chunk<M>();
    __shared__ int s_col[kWarps][kChunk];
    __shared__ T s_del[kWarps][M][kChunk];
    __shared__ double red[kWarps][M][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const bool skip = (ctrl->flags != 0) || (ctrl->ls_accept >= 0);

    T tau[M], tl1[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        tau[m] = (T)ldexp(tau0, -(h_base + m));
        tl1[m] = tau[m] * lam1;
    }
    double q[M], n2[M], ph[M], nb[M];
#pragma unroll
    for (int m = 0; m < M; ++m) { q[m] = 0.0; n2[m] = 0.0; ph[m] = 0.0; nb[m] = 0.0; }

    for (int i = skip ? p : gw; i < p; i += nw) {
        const int beg = bk.off[i], L = bk.len[i];
        for (int eb = 0; eb < L; eb += 32) {
            const int e = eb + lane;
            T de[M];
            int je = 0;
            bool act_e = false;
            if (e < L) {
                je = bk.col_b[beg + e];
                const T om = bk.om_b[beg + e], g = bk.g[beg + e];
                const bool diag = (je == i);
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const T np_ = prox_entry(om, g, tau[m], tl1[m], diag);
                    de[m] = np_ - om;
                    act_e |= (de[m] != T(0));
                    const double dd = (double)de[m];
                    n2[m] += dd * dd;
                    if (diag) {
                        if (!(np_ > T(0))) nb[m] += 1.0;
                        else {
                            const double x = dd / (double)om;
                            ph[m] += x - log1p(x);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < M; ++m) de[m] = T(0);
            }
            for (int fb = eb; fb < L; fb += kChunk) {
                __syncwarp();
                for (int t = lane; t < kChunk; t += 32) {
                    const int f = fb + t;
                    int jf = -1;
                    if (f < L) {
                        jf = bk.col_b[beg + f];
                        const T om = bk.om_b[beg + f], g = bk.g[beg + f];
                        bool act = false;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const T d = prox_entry(om, g, tau[m], tl1[m], jf == i) - om;
                            s_del[warp][m][t] = d;
                            act |= (d != T(0));
                        }
                        if (!act) jf = -1;
                    }
                    s_col[warp][t] = jf;
                }
                __syncwarp();
                if (act_e) {
                    T qf[M];
#pragma unroll
                    for (int m = 0; m < M; ++m) qf[m] = T(0);
                    const T* srow = S + (int64_t)je * ld;
                    const int tmax = min(kChunk, L - fb);
                    for (int t = 0; t < tmax; ++t) {
                        const int f = fb + t;
                        const int jf = s_col[warp][t];
                        if (f < e || jf < 0) continue;
                        const T s = srow[jf];
                        const T wgt = (f == e) ? T(1) : T(2);
#pragma unroll
                        for (int m = 0; m < M; ++m) qf[m] = fmaT(wgt * de[m] * s_del[warp][m][t], s, qf[m]);
                    }
#pragma unroll
                    for (int m = 0; m < M; ++m) q[m] += (double)qf[m];
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const double a = warp_sum(q[m]), b = warp_sum(n2[m]), c = warp_sum(ph[m]), d = warp_sum(nb[m]);
        if (lane == 0) { red[warp][m][0] = a; red[warp][m][1] = b; red[warp][m][2] = c; red[warp][m][3] = d; }
    }
    __syncthreads();
    if (threadIdx.x < M * 4) {
        const int m = threadIdx.x / 4, k = threadIdx.x % 4;
        double a = 0.0;
        for (int w = 0; w < kWarps; ++w) a += red[w][m][k];
        part_ls[(size_t)blockIdx.x * kMaxWindow * 4 + m * 4 + k] = a;
    }
}

// Reduce the partials in a fixed order and take the decision of Alg. 1 step 9.
__global__ void __launch_bounds__(128)
k_ls_decide(const double* __restrict__ part_ls, const double* __restrict__ part_obj, int nblk, int M,
            int h_base, int max_halvings, double tau0, double lam1, double lam2, int first,
            Ctrl* ctrl) {
    __shared__ double sums[kMaxWindow * 4];
    __shared__ double obj[4];
    const int t = threadIdx.x;
    if (ctrl->flags != 0 || ctrl->ls_accept >= 0) return;
    if (t < M * 4) {
        double a = 0.0;
        for (int b = 0; b < nblk; ++b) a += part_ls[(size_t)b * kMaxWindow * 4 + t];
        sums[t] = a;
    }
    if (first && t >= 64 && t < 68) {
        double a = 0.0;
        for (int b = 0; b < nblk; ++b) a += part_obj[b * 4 + (t - 64)];
        obj[t - 64] = a;
    }
    __syncthreads();
    if (t != 0) return;
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

// ------------------------------------------------------------------ 4. accept
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_compact_count(int p, Buckets<T> bk, T lam1, int* cnt2, const Ctrl* ctrl) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (ctrl->flags != 0 || ctrl->ls_accept < 0) return;
    const T tau = (T)ctrl->tau;
    const T tl1 = tau * lam1;
    for (int i = gw; i < p; i += nw) {
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
__global__ void __launch_bounds__(kThreads)
k_compact_write(int p, Buckets<T> bk, T lam1, Csr<T> nx, int cap, const Ctrl* ctrl) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (ctrl->flags != 0 || ctrl->ls_accept < 0) return;
    const T tau = (T)ctrl->tau;
    const T tl1 = tau * lam1;
    for (int i = gw; i < p; i += nw) {
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

__global__ void k_converge(const int* rp_next, int p, int cap, double eps, Ctrl* ctrl) {
    if (ctrl->flags != 0 || ctrl->ls_accept < 0) return;
    const int nnz = rp_next[p];
    ctrl->nnz_next = nnz;
    if (nnz > cap) { ctrl->flags |= kFlagNnzOverflow; return; }
    const double rel = sqrt(ctrl->delta2) / sqrt(ctrl->norm2_cur);
    ctrl->rel = rel;
    ctrl->converged = rel < eps ? 1 : 0;
    ctrl->iter += 1;
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

}  // namespace

// ------------------------------------------------------------------ launchers
template <typename T>
void launch_iter_begin(const IterBufs<T>& b, cudaStream_t s) {
    k_iter_begin<T><<<64, 256, 0, s>>>(b.bk, b.p, b.ctrl);
}

template <typename T>
void launch_grad_screen(const IterBufs<T>& b, cudaStream_t s) {
    constexpr int BJ = 32 * (16 / sizeof(T));
    dim3 grid((b.p + kScreenRows - 1) / kScreenRows, (b.p + BJ - 1) / BJ);
    k_grad_screen<T><<<grid, kThreads, 0, s>>>(b.S, b.ld, b.p, b.cur.rp, b.cur.ci, b.cur.cv, b.lam1,
                                               b.em, b.ctrl);
}

template <typename T>
void launch_candidates(const IterBufs<T>& b, cudaStream_t s) {
    const int g = 152 * 4;
    k_bucket_count<T><<<g, 256, 0, s>>>(b.em, b.bk, b.ctrl);
    k_scan<<<1, 1024, 0, s>>>(b.bk.cnt, b.bk.off, b.p, b.bk.cap, b.ctrl, kFlagBucketOverflow,
                              &b.ctrl->bucket_total);
    k_bucket_scatter<T><<<g, 256, 0, s>>>(b.em, b.bk, b.ctrl);
    k_bucket_sort<T><<<b.nblk, kThreads, 0, s>>>(b.bk, b.p, b.ctrl);
    k_fill_w<T><<<b.nblk, kThreads, 0, s>>>(b.S, b.ld, b.p, b.cur, b.bk, b.ctrl);
    k_gradient<T><<<b.nblk, kThreads, 0, s>>>(b.p, b.bk, b.lam1, b.lam2, b.part_obj, b.ctrl);
}

template <typename T, int M>
static void ls_eval_m(const IterBufs<T>& b, int h_base, cudaStream_t s) {
    k_ls_eval<T, M><<<b.nblk, kThreads, 0, s>>>(b.S, b.ld, b.p, b.bk, b.lam1, 1.0, h_base, b.part_ls, b.ctrl);
}

template <typename T>
void launch_ls_window(const IterBufs<T>& b, int h_base, bool first, cudaStream_t s) {
    const int M = b.ls_window;
    switch (M) {
        case 1: ls_eval_m<T, 1>(b, h_base, s); break;
        case 2: ls_eval_m<T, 2>(b, h_base, s); break;
        case 4: ls_eval_m<T, 4>(b, h_base, s); break;
        case 8: ls_eval_m<T, 8>(b, h_base, s); break;
        default: ls_eval_m<T, 16>(b, h_base, s); break;
    }
    k_ls_decide<<<1, 128, 0, s>>>(b.part_ls, b.part_obj, b.nblk, M == 1 || M == 2 || M == 4 || M == 8 ? M : 16,
                                  h_base, b.max_halvings, 1.0, (double)b.lam1, (double)b.lam2, first ? 1 : 0,
                                  b.ctrl);
}

template <typename T>
void launch_accept(const IterBufs<T>& b, cudaStream_t s) {
    k_compact_count<T><<<b.nblk, kThreads, 0, s>>>(b.p, b.bk, b.lam1, b.cnt2, b.ctrl);
    k_scan<<<1, 1024, 0, s>>>(b.cnt2, b.next.rp, b.p, 0x7fffffff, b.ctrl, 0, nullptr);
    k_compact_write<T><<<b.nblk, kThreads, 0, s>>>(b.p, b.bk, b.lam1, b.next, b.csr_cap, b.ctrl);
    k_converge<<<1, 1, 0, s>>>(b.next.rp, b.p, b.csr_cap, b.eps, b.ctrl);
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
    template void launch_iter_begin<T>(const IterBufs<T>&, cudaStream_t);                          \
    template void launch_grad_screen<T>(const IterBufs<T>&, cudaStream_t);                         \
    template void launch_candidates<T>(const IterBufs<T>&, cudaStream_t);                          \
    template void launch_ls_window<T>(const IterBufs<T>&, int, bool, cudaStream_t);                \
    template void launch_accept<T>(const IterBufs<T>&, cudaStream_t);                              \
    template void launch_set_identity<T>(Csr<T>, int, cudaStream_t);                               \
    template void launch_csr_export<T>(const int*, const int*, const T*, int, int, int64_t*, int32_t*, \
                                       void*, int, cudaStream_t);

HPC_INSTANTIATE(float)
HPC_INSTANTIATE(double)

}  // namespace hpc
