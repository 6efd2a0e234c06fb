// Obs variant (Alg. 3): the products that replace S.
//
//   Y^T = Omega X^T (p x n)            row-split SpMM (adjoint.cu), canonical order
//   Z   = Y X / n = Y^T (X^T)^T / n    this file: tcgen05 GEMM on K-major panels
//
// Z equals W = Omega S, so the screening rule of the Cov pass applies: an entry
// can enter a prox step only if it is in the support or |G_ij| > lambda1, and
// |G_ij| > lambda1 needs max(|Z_ij|, |Z_ji|) > lambda1.  Persistent CTAs walk the
// tile pairs Z[I, J] and Z[J, I] (I <= J, 128 x 128 tiles), each into one of two
// TMEM accumulator pairs; the epilogue warps transpose the second tile through
// shared memory and emit both (i, j) and (j, i) -- flagged as paired, so no
// partner request follows -- for every pair in the support or above the
// threshold (Alg. 3 steps 4-6 with the transpose done inside the CTA), while the
// next pair accumulates.  Z is never stored.
//
// Operands are BF16 hi/lo panels (BF16X3: hi*hi + hi*lo + lo*hi) or TF32
// panels, K-major, zero padded; loaded by TMA (128-byte swizzle) through an
// mbarrier ring; every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "ptx.cuh"

namespace hpc {
namespace {

constexpr int kT = 128;                    // tile edge (UMMA M = N = 128)
constexpr int kRowB = 128;                 // bytes per swizzle row
constexpr int kPanelTile = kT * kRowB;     // 16 KB
constexpr uint32_t kTmemCols = 256;        // one accumulator pair: two 128-column FP32 accumulators
constexpr long long kWaitLimit = 1ll << 22;     // polls of at most 1 us each

enum : int { kObsBf16x3 = 0, kObsTf32 = 1 };

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void ptx_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int MODE>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if constexpr (MODE == kObsTf32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     ptx::smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// K-major, 128-byte swizzle, 8-row groups 1024 bytes apart, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

template <int MODE>
__host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4) | ((MODE == kObsTf32 ? 2u : 1u) << 7) | ((MODE == kObsTf32 ? 2u : 1u) << 10) |
           ((uint32_t)(kT >> 3) << 17) | ((uint32_t)(kT >> 4) << 24);
}

template <int MODE>
struct ObsCfg {
    static constexpr int kPieces = MODE == kObsBf16x3 ? 2 : 1;
    static constexpr int kTerms = MODE == kObsBf16x3 ? 3 : 1;
    static constexpr int kElem = MODE == kObsTf32 ? 4 : 2;
    static constexpr int kBK = kRowB / kElem;
    static constexpr int kMmaK = 32 / kElem;
    static constexpr int kStageBytes = kPieces * 2 * kPanelTile;    // A and B tiles, each piece
    static constexpr int kStages = MODE == kObsBf16x3 ? 3 : 5;
    static constexpr int kRing = 8;                                  // pair slots between the roles
    static constexpr int kLook = 4;                                  // pairs published ahead of the loads
    static constexpr int kSupBytes = kRing * kT * (16 + 4);          // support masks (uint4) and CSR starts
    static constexpr int kCtlBytes = 512;                            // barriers, pair slots, TMEM address
    static constexpr int kSmem = kStages * kStageBytes + kSupBytes + kCtlBytes + 1024;
};

constexpr int kEpiWarps = 8;
constexpr int kObsThreads = 128 + 32 * kEpiWarps;     // warpgroup 0: roles; warpgroups 1-2: epilogue
constexpr int kHelpThreads = 64;                      // warps 2-3: support masks
// Registers per thread after setmaxnreg (warpgroup 0 down, the epilogue warpgroups up);
// the host checks that the launch's pool covers both (kMinLaunchRegs) before launching.
constexpr int kRegsSmall = 56;
constexpr int kRegsEpi = 216;
constexpr int kMinLaunchRegs = (128 * kRegsSmall + 32 * kEpiWarps * kRegsEpi + kObsThreads - 1) / kObsThreads;


// 32 TMEM lanes x 16 consecutive 32-bit columns: thread t gets lane (base + t).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// v[O + b] for a run-time b in 0..31 without indexing registers dynamically: a
// five-level tree of selects on the bits of b.
template <int O>
__device__ __forceinline__ float pick32(const float (&v)[64], int b) {
    float t16[16], t8[8], t4[4], t2[2];
#pragma unroll
    for (int i = 0; i < 16; ++i) t16[i] = (b & 16) ? v[O + 16 + i] : v[O + i];
#pragma unroll
    for (int i = 0; i < 8; ++i) t8[i] = (b & 8) ? t16[8 + i] : t16[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) t4[i] = (b & 4) ? t8[4 + i] : t8[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) t2[i] = (b & 2) ? t4[2 + i] : t4[i];
    return (b & 1) ? t2[1] : t2[0];
}

// Support of row g in the columns j0 .. j0 + 127: a 128-bit mask and the CSR position
// of the row's first entry at or after column j0 (columns ascend, so the k-th set bit
// of the mask is entry qs + k).  A binary search narrows long rows; the entries are
// then read eight at a time with independent loads.
__device__ __forceinline__ void row_tile_support(const int* __restrict__ rp, const int* __restrict__ ci, int g, int j0,
                                                 uint4& mask, int& qs) {
    uint32_t m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
    int lo = rp[g];
    const int e = rp[g + 1];
    int hi = e;
    while (hi - lo > 8) {
        const int mid = (lo + hi) >> 1;
        if (ci[mid] < j0) lo = mid + 1;
        else hi = mid;
    }
    // lower_bound lies in [lo, hi]; entries before lo are < j0
    int q = lo;
    bool more = true;
    int first = -1;
    while (more) {
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = q + u < e ? ci[q + u] : 0x7fffffff;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = v[u] - j0;
            if (first < 0 && v[u] >= j0) first = q + u;
            const uint32_t bit = (c >= 0 && c < kT) ? 1u << (c & 31) : 0u;
            const int w = c >> 5;
            m0 |= w == 0 ? bit : 0u;
            m1 |= w == 1 ? bit : 0u;
            m2 |= w == 2 ? bit : 0u;
            m3 |= w == 3 ? bit : 0u;
        }
        more = q + 8 < e && v[7] < j0 + kT;
        q += 8;
    }
    qs = first < 0 ? e : first;
    mask = make_uint4(m0, m1, m2, m3);
}

// Persistent pair kernel: one CTA per SM takes block pairs (I <= J) from a shared
// counter, in the pair list's order (bands of row blocks, so the pairs in flight
// across the GPU share their panels in L2).  For pair (I, J) it forms, in TMEM,
//   phase 0:  Y^T[I] X^T[J]^T = n Z[I, J]          (row r, column c: n Z_{I0+r, J0+c})
//   phase 1:  X^T[I] Y^T[J]^T = n Z[J, I]^T        (row r, column c: n Z_{J0+c, I0+r})
// so that the thread holding row r of the tile has both n Z_ij and n Z_ji of every
// pair (i, j) = (I0 + r, J0 + c) in its registers: the transpose of Alg. 3 step 6
// costs nothing, and the screening test and the emission of both (i, j) and (j, i)
// happen in one thread.
//
// Chunked accumulation, as in the Gram: the K loop of a pair is cut into chunks
// (chunk_start), each chunk accumulates both tiles from zero into one TMEM
// accumulator pair, and the epilogue adds the chunk sums in FP32 round-to-nearest in
// registers, so the bias of the tensor core's truncating accumulation scales with
// the chunk, not with n.
//
// Roles:
//   warp 0      thread 0: takes the CTA's next pair from the counter, publishes it in
//               a ring of kRing pair slots, and streams per chunk the stages of
//               (Y^T[I], X^T[J]), then of (X^T[I], Y^T[J]) through TMA;
//   warp 1      MMA issuer (thread 32) and TMEM owner: chunk c of the CTA's sequence
//               into accumulator pair c & 1 (columns 256 (c & 1) + {0, 128});
//   warps 2-3   the support of the pair's rows in its columns (row_tile_support),
//               into the slot's masks, ahead of the epilogue;
//   warps 4-11  running sums (warp w: TMEM lanes 32 (w % 4) .. + 31, one row per
//               thread; warps 4-7 columns 0-63, warps 8-11 columns 64-127 of both
//               tiles), then the screening test and the emission.
// pair_full / pair_empty hand the pair slots around, sup_full the masks, acc_full /
// acc_empty the accumulator pairs.  Every wait is bounded; after an abort every
// role stops, the loads in flight drain and TMEM is freed.
template <int MODE>
__global__ void __launch_bounds__(kObsThreads, 1)
k_obs_pair(const __grid_constant__ CUtensorMap ya, const __grid_constant__ CUtensorMap yb,
           const __grid_constant__ CUtensorMap xa, const __grid_constant__ CUtensorMap xb, const int2* __restrict__ pairs,
           int npairs, int k_tiles, int p, int64_t n, const int* __restrict__ rp, const int* __restrict__ ci,
           const float* __restrict__ cv, Emit<float> em, Ctrl* __restrict__ ctrl, int chunk_kt, int lead_kt) {
    using C = ObsCfg<MODE>;
    constexpr int R = C::kRing;
    const float lam1 = (float)ctrl->lam1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint4* s_mask = reinterpret_cast<uint4*>(smem + C::kStages * C::kStageBytes);           // [R][kT]
    int* s_qs = reinterpret_cast<int*>(s_mask + R * kT);                                   // [R][kT]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStageBytes + C::kSupBytes);
    uint64_t* empty = full + C::kStages;
    uint64_t* acc_full = empty + C::kStages;     // [2]
    uint64_t* acc_empty = acc_full + 2;          // [2]
    uint64_t* pair_full = acc_empty + 2;         // [R]
    uint64_t* pair_empty = pair_full + R;        // [R]
    uint64_t* sup_full = pair_empty + R;         // [R]
    int2* s_pair = reinterpret_cast<int2*>(sup_full + R);                                  // [R]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(s_pair + R);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    static_assert(8 * (2 * C::kStages + 4 + 3 * R) + 8 * R + 8 <= C::kCtlBytes, "control area");
    static_assert(C::kSmem <= 232448, "shared memory per block");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (chunk_kt < 1) chunk_kt = 1;
    if (lead_kt < chunk_kt) lead_kt = chunk_kt;
    const int nch = num_chunks(k_tiles, chunk_kt, lead_kt);

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) { ptx::mbar_init(&full[s], 1); ptx::mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { ptx::mbar_init(&acc_full[b], 1); ptx::mbar_init(&acc_empty[b], kEpiWarps); }
        for (int s = 0; s < R; ++s) {
            ptx::mbar_init(&pair_full[s], 1);
            ptx::mbar_init(&pair_empty[s], 1 + 2 + kEpiWarps);      // MMA issuer, helper warps, epilogue warps
            ptx::mbar_init(&sup_full[s], kHelpThreads);
        }
        *abort_flag = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 2 * kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    long long issued = 0;
    if (warp < 4) {
        // producer, MMA issuer and the helpers: one warpgroup that gives registers away
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsSmall));
        if (threadIdx.x == 0) {
            // ---------------- scheduler and producer
            // Pairs are published kLook ahead of the loads, so that the counter's and the
            // pair list's latency, and the helpers' mask work, stay off the MMA's path.
            long long g = 0;
            bool ok = true, pub_done = false;
            int pub = 0;
            int nxt = atomicAdd(&ctrl->obs_next, 1);
            auto publish = [&]() -> bool {
                const int slot = pub % R;
                if (!ptx::mbar_wait_bounded(&pair_empty[slot], ((uint32_t)(pub / R) & 1u) ^ 1u, abort_flag,
                                            kWaitLimit))
                    return false;
                const int idx = nxt;
                const int2 pr = idx < npairs ? pairs[idx] : make_int2(-1, -1);
                if (idx < npairs) nxt = atomicAdd(&ctrl->obs_next, 1);
                s_pair[slot] = pr;
                ptx::mbar_arrive(&pair_full[slot]);
                ++pub;
                pub_done = pr.x < 0;
                return true;
            };
            for (int q = 0; q < C::kLook && ok && !pub_done; ++q) ok = publish();
            for (int t = 0; ok && t < pub; ++t) {
                const int2 pr = s_pair[t % R];
                if (pr.x < 0) break;
                if (!pub_done && !publish()) break;            // pair t + kLook
                const int I0 = pr.x * kT, J0 = pr.y * kT;
                for (int c = 0; c < nch && ok; ++c) {
                    const int kt0 = chunk_start(c, k_tiles, chunk_kt, lead_kt);
                    const int kt1 = chunk_start(c + 1, k_tiles, chunk_kt, lead_kt);
                    for (int phase = 0; phase < 2 && ok; ++phase) {
                        // phase 0: A = Y^T[I], B = X^T[J]; phase 1: A = X^T[I], B = Y^T[J]
                        const CUtensorMap* ma = phase == 0 ? &ya : &xa;
                        const CUtensorMap* mb = phase == 0 ? &xa : &ya;
                        const CUtensorMap* la = phase == 0 ? &yb : &xb;
                        const CUtensorMap* lb = phase == 0 ? &xb : &yb;
                        for (int kt = kt0; kt < kt1; ++kt, ++g) {
                            const int s = (int)(g % C::kStages);
                            const uint32_t ph = (uint32_t)(g / C::kStages) & 1u;
                            if (!ptx::mbar_wait_bounded(&empty[s], ph ^ 1u, abort_flag, kWaitLimit)) {
                                ok = false;
                                break;
                            }
                            uint8_t* st = smem + s * C::kStageBytes;
                            ptx::mbar_expect_tx(&full[s], C::kStageBytes);
                            const int kc = kt * C::kBK;
                            ptx::tma_load_2d(st, ma, &full[s], kc, I0);
                            ptx::tma_load_2d(st + kPanelTile, mb, &full[s], kc, J0);
                            if (C::kPieces > 1) {
                                ptx::tma_load_2d(st + 2 * kPanelTile, la, &full[s], kc, I0);
                                ptx::tma_load_2d(st + 3 * kPanelTile, lb, &full[s], kc, J0);
                            }
                            ++issued;
                        }
                    }
                }
            }
        } else if (threadIdx.x == 32) {
            // ---------------- MMA issuer
            constexpr uint32_t idesc = instr_desc<MODE>();
            long long g = 0, gc = 0;
            bool ok = true;
            for (int t = 0; ok; ++t) {
                const int slot = t % R;
                if (!ptx::mbar_wait_bounded(&pair_full[slot], (uint32_t)(t / R) & 1u, abort_flag, kWaitLimit)) break;
                const int2 pr = s_pair[slot];
                ptx::mbar_arrive(&pair_empty[slot]);
                if (pr.x < 0) break;
                for (int c = 0; c < nch && ok; ++c, ++gc) {
                    const int b = (int)(gc & 1);
                    if (!ptx::mbar_wait_bounded(&acc_empty[b], ((uint32_t)(gc >> 1) & 1u) ^ 1u, abort_flag,
                                                kWaitLimit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int kt0 = chunk_start(c, k_tiles, chunk_kt, lead_kt);
                    const int kt1 = chunk_start(c + 1, k_tiles, chunk_kt, lead_kt);
                    for (int phase = 0; phase < 2 && ok; ++phase) {
                        const uint32_t d = tmem + (uint32_t)(b * 2 * kT + phase * kT);
                        for (int kt = kt0; kt < kt1; ++kt, ++g) {
                            const int s = (int)(g % C::kStages);
                            const uint32_t ph = (uint32_t)(g / C::kStages) & 1u;
                            if (!ptx::mbar_wait_bounded(&full[s], ph, abort_flag, kWaitLimit)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t st = ptx::smem_u32(smem + s * C::kStageBytes);
                            const uint32_t a_hi = st, b_hi = st + kPanelTile, a_lo = st + 2 * kPanelTile,
                                           b_lo = st + 3 * kPanelTile;
#pragma unroll
                            for (int kk = 0; kk < C::kBK / C::kMmaK; ++kk) {
                                const uint32_t off = kk * 32;
                                const uint32_t acc0 = (kt > kt0 || kk > 0) ? 1u : 0u;
                                umma<MODE>(d, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_hi + off), idesc, acc0);
                                if constexpr (C::kTerms == 3) {
                                    umma<MODE>(d, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_lo + off), idesc, 1u);
                                    umma<MODE>(d, smem_desc_sw128(a_lo + off), smem_desc_sw128(b_hi + off), idesc, 1u);
                                }
                            }
                            umma_commit(&empty[s]);
                        }
                    }
                    if (ok) umma_commit(&acc_full[b]);
                }
            }
        } else if (warp >= 2) {
            // ---------------- support masks of the pair's rows (two rows per thread)
            const int ht = threadIdx.x - 64;
            for (int t = 0;; ++t) {
                const int slot = t % R;
                if (!ptx::mbar_wait_bounded(&pair_full[slot], (uint32_t)(t / R) & 1u, abort_flag, kWaitLimit)) break;
                const int2 pr = s_pair[slot];
                if (pr.x < 0) break;
                const int I0 = pr.x * kT, J0 = pr.y * kT;
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int rr = ht + kHelpThreads * h2;
                    const int g = I0 + rr;
                    uint4 m = make_uint4(0u, 0u, 0u, 0u);
                    int qs = 0;
                    if (g < p) row_tile_support(rp, ci, g, J0, m, qs);
                    s_mask[slot * kT + rr] = m;
                    s_qs[slot * kT + rr] = qs;
                }
                ptx::mbar_arrive(&sup_full[slot]);
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&pair_empty[slot]);
            }
        }
    } else {
        // the epilogue warpgroups take them: 2 x 64 running sums live in registers
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsEpi));
        // ---------------- epilogue
        // Thread (q4, lane) of warp w owns row r = 32 q4 + lane of the tile (g = I0 + r)
        // and the columns c0 .. c0 + 63 (c0 = 64 half).  For each column it holds
        // a = n Z_ij and b = n Z_ji (j = J0 + c).  The pair {(i, j), (j, i)} is emitted
        // when it is in the support, on the diagonal, or when |a| or |b| exceeds lambda1 n;
        // (i, j) carries a / n and (j, i) carries b / n, both flagged as paired (each is the
        // other's partner) and both with w_ij (the iterate is symmetric).  In a diagonal
        // pair (I = J) each thread emits only its own row's entry: (j, i) is the row of
        // another thread of the same tile.
        const int q4 = warp & 3;
        const int half = (warp - 4) >> 2;
        const int r = q4 * 32 + lane;
        const int c0 = half * 64;
        const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0;
        // Z = (Y X) / n: the sums are tested against lambda1 n and only the emitted entries
        // are scaled.  The threshold is lowered by 2^-20 relative, so that the entries
        // emitted include every one whose scaled value exceeds lambda1 in FP32; an extra
        // entry at the threshold is harmless (its prox step leaves it at zero).
        const float inv_n = 1.0f / (float)n;
        const float thr = (float)((double)lam1 * (double)n * (1.0 - 0x1p-20));
        long long gc = 0;
        for (int t = 0;; ++t) {
            const int slot = t % R;
            const uint32_t rph = (uint32_t)(t / R) & 1u;
            bool got = !*abort_flag && ptx::mbar_wait_bounded(&pair_full[slot], rph, abort_flag, kWaitLimit);
            got = __all_sync(kFull, got);
            if (!got) break;
            const int2 pr = s_pair[slot];
            if (pr.x < 0) break;
            const int I0 = pr.x * kT, J0 = pr.y * kT;
            const bool diag_pair = pr.x == pr.y;
            const int g = I0 + r;
            float za[64], zb[64];
            bool have = true;
            for (int c = 0; c < nch; ++c, ++gc) {
                const int b = (int)(gc & 1);
                bool ok = have && !*abort_flag &&
                          ptx::mbar_wait_bounded(&acc_full[b], (uint32_t)(gc >> 1) & 1u, abort_flag, kWaitLimit);
                ok = __all_sync(kFull, ok);
                if (!ok) { have = false; continue; }
                tc_fence_after();
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) {
                    uint32_t va[16], vb[16];
                    tmem_ld16(lane_base + (uint32_t)(b * 2 * kT + s4 * 16), va);
                    tmem_ld16(lane_base + (uint32_t)(b * 2 * kT + kT + s4 * 16), vb);
                    tmem_ld_wait();
                    if (c == 0) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            za[s4 * 16 + q] = __uint_as_float(va[q]);
                            zb[s4 * 16 + q] = __uint_as_float(vb[q]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            za[s4 * 16 + q] += __uint_as_float(va[q]);
                            zb[s4 * 16 + q] += __uint_as_float(vb[q]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx_arrive(&acc_empty[b]);
            }
            if (!have) break;
            bool sok = ptx::mbar_wait_bounded(&sup_full[slot], rph, abort_flag, kWaitLimit);
            sok = __all_sync(kFull, sok);
            if (!sok) break;
            const uint4 m4 = s_mask[slot * kT + r];
            const int qs = s_qs[slot * kT + r];
            const uint32_t sm[2] = {half ? m4.z : m4.x, half ? m4.w : m4.y};
            const int before0 = half ? __popc(m4.x) + __popc(m4.y) : 0;
            const bool mine = g < p;
            uint32_t eb[2];
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                uint32_t w = 0u;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const bool big = !(fabsf(za[32 * k + q]) <= thr) || !(fabsf(zb[32 * k + q]) <= thr);
                    w |= (uint32_t)big << q;
                }
                w |= sm[k];
                const int lim = p - (J0 + c0 + 32 * k);                 // columns J0 + c0 + 32 k + q < p
                if (lim < 32) w &= lim > 0 ? (1u << lim) - 1u : 0u;
                if (diag_pair && (r >> 5) == 2 * half + k) w |= 1u << (r & 31);      // the diagonal
                eb[k] = mine ? w : 0u;
                cnt += __popc(eb[k]);
            }
            if (!diag_pair) cnt *= 2;
            // one atomic per warp: an inclusive scan of the lanes' counts, the last lane takes
            // the warp's total from the emission counter and every lane writes from its offset
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            int base = 0;
            if (lane == 31 && incl > 0) base = atomicAdd(&ctrl->em_count, incl);
            base = __shfl_sync(kFull, base, 31);
            int pos = base + incl - cnt;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                uint32_t bits = eb[k];
                const uint32_t sw = sm[k];
                const int before = before0 + (k ? __popc(sm[0]) : 0);
                while (bits) {
                    const int q = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int j = J0 + c0 + 32 * k + q;
                    const bool sup = (sw >> q) & 1u;
                    const float om = sup ? cv[qs + before + __popc(sw & ((1u << q) - 1u))] : 0.f;
                    const unsigned fl = 0x40000000u | (sup ? 0x80000000u : 0u);
                    if (pos < em.cap) {
                        em.row[pos] = g;
                        em.col[pos] = (int)((unsigned)j | fl);
                        em.w[pos] = __fmul_rn(k ? pick32<32>(za, q) : pick32<0>(za, q), inv_n);
                        em.om[pos] = om;
                    }
                    ++pos;
                    if (!diag_pair) {
                        if (pos < em.cap) {
                            em.row[pos] = j;
                            em.col[pos] = (int)((unsigned)g | fl);
                            em.w[pos] = __fmul_rn(k ? pick32<32>(zb, q) : pick32<0>(zb, q), inv_n);
                            em.om[pos] = om;
                        }
                        ++pos;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&pair_empty[slot]);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) {
            atomicOr(&ctrl->flags, kFlagTimeout);
            for (long long g = issued > C::kStages ? issued - C::kStages : 0; g < issued; ++g) {
                const int s = (int)(g % C::kStages);
                const uint32_t ph = (uint32_t)(g / C::kStages) & 1u;
                for (long long it = 0; it < (1ll << 22) && !ptx::mbar_try_wait(&full[s], ph); ++it) __nanosleep(64);
            }
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kTmemCols);
    }
}

// FP32 rows (rows x ldi, K contiguous) -> K-major panels (rows_pad x n_pad) of the MMA input type.
template <int MODE>
__global__ void k_obs_split(const float* __restrict__ in, int64_t rows, int64_t cols, int64_t ldi, void* hi, void* lo,
                            int64_t rows_pad, int64_t n_pad) {
    const int64_t total = rows_pad * n_pad;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / n_pad, k = t % n_pad;
        const float x = (r < rows && k < cols) ? in[r * ldi + k] : 0.f;
        if constexpr (MODE == kObsTf32) {
            uint32_t u;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
            static_cast<float*>(hi)[t] = __uint_as_float(u);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            static_cast<__nv_bfloat16*>(hi)[t] = h;
            static_cast<__nv_bfloat16*>(lo)[t] = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
size_t obs_panel_bytes(int precision, int64_t n, int64_t p) {
    const int64_t p_pad = (p + kT - 1) / kT * kT, n_pad = (n + 63) / 64 * 64;
    const int es = precision == HPC_PREC_TF32 ? 4 : 2;
    return ((size_t)p_pad * n_pad * es + 1023) / 1024 * 1024;
}

int obs_pieces(int precision) { return precision == HPC_PREC_TF32 ? 1 : 2; }

int64_t obs_npairs(int64_t p) {
    const int64_t nb = (p + kT - 1) / kT;
    return nb * (nb + 1) / 2;
}

void obs_pair_list(int64_t p, std::vector<int2>& out) {
    const int64_t nb = (p + kT - 1) / kT;
    out.clear();
    // bands of 8 row blocks, columns left to right: pairs in flight share panels in L2
    for (int64_t b0 = 0; b0 < nb; b0 += 8)
        for (int64_t bj = 0; bj < nb; ++bj)
            for (int64_t bi = b0; bi < std::min<int64_t>(b0 + 8, nb); ++bi)
                if (bi <= bj) out.push_back(make_int2((int)bi, (int)bj));
}

void launch_obs_split(int precision, const float* in, int64_t rows, int64_t cols, int64_t ldi, void* hi, void* lo,
                      int64_t n, int64_t p, cudaStream_t s) {
    const int64_t rows_pad = (p + kT - 1) / kT * kT, n_pad = (n + 63) / 64 * 64;
    if (precision == HPC_PREC_TF32)
        k_obs_split<kObsTf32><<<2048, 256, 0, s>>>(in, rows, cols, ldi, hi, lo, rows_pad, n_pad);
    else
        k_obs_split<kObsBf16x3><<<2048, 256, 0, s>>>(in, rows, cols, ldi, hi, lo, rows_pad, n_pad);
}

bool obs_make_maps(int precision, const void* y_hi, const void* y_lo, const void* x_hi, const void* x_lo, int64_t n,
                   int64_t p, CUtensorMap* maps /*4: ya, yb, xa, xb*/) {
    const int64_t p_pad = (p + kT - 1) / kT * kT, n_pad = (n + 63) / 64 * 64;
    const int es = precision == HPC_PREC_TF32 ? 4 : 2;
    const void* bases[4] = {y_hi, precision == HPC_PREC_TF32 ? y_hi : y_lo, x_hi,
                            precision == HPC_PREC_TF32 ? x_hi : x_lo};
    for (int t = 0; t < 4; ++t)
        if (!encode_tensor_map_2d_sw128(&maps[t], bases[t], es, (uint64_t)n_pad, (uint64_t)p_pad,
                                        (uint64_t)n_pad * es, (uint32_t)(kRowB / es), (uint32_t)kT))
            return false;
    return true;
}

// K elements -> whole stages of kbk elements, at least one.
static int kt_of(int64_t k, int kbk) { return (int)std::max<int64_t>(1, std::min<int64_t>(k / kbk, 1 << 30)); }

cudaError_t launch_obs_pairs(int precision, const CUtensorMap* maps, const int2* pairs, int64_t npairs, int64_t n,
                             int p, const int* rp, const int* ci, const float* cv, Emit<float> em,
                             Ctrl* ctrl, cudaStream_t s, int64_t chunk_k, int64_t lead_k) {
    const int64_t n_pad = (n + 63) / 64 * 64;
    // K elements per accumulation chunk (the Gram's BF16X3 / TF32 default when none is given)
    if (chunk_k <= 0) chunk_k = 256;
    if (lead_k <= 0) lead_k = 4 * chunk_k;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || sms < 1)
            sms = 1;
    }
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(npairs, sms));   // one CTA per SM
    // setmaxnreg moves registers between the warpgroups of a block: the kernel must have
    // been built with enough registers per thread for both shares (else it would wait)
    static int regs[2] = {-1, -1};
    const int mi = precision == HPC_PREC_TF32 ? 1 : 0;
    if (regs[mi] < 0) {
        cudaFuncAttributes fa;
        const cudaError_t e = cudaFuncGetAttributes(
            &fa, mi ? (const void*)k_obs_pair<kObsTf32> : (const void*)k_obs_pair<kObsBf16x3>);
        if (e != cudaSuccess) return e;
        regs[mi] = fa.numRegs;
    }
    if (regs[mi] < kMinLaunchRegs) return cudaErrorNotSupported;
    if (precision == HPC_PREC_TF32) {
        using C = ObsCfg<kObsTf32>;
        cudaError_t e = set_smem_once((const void*)k_obs_pair<kObsTf32>, C::kSmem, kSmemSlotObsTf32);
        if (e != cudaSuccess) return e;
        k_obs_pair<kObsTf32><<<grid, kObsThreads, C::kSmem, s>>>(maps[0], maps[1], maps[2], maps[3], pairs,
                                                                 (int)npairs, (int)(n_pad / C::kBK), p, n, rp, ci,
                                                                 cv, em, ctrl, kt_of(chunk_k, C::kBK),
                                                                 kt_of(lead_k, C::kBK));
    } else {
        using C = ObsCfg<kObsBf16x3>;
        cudaError_t e = set_smem_once((const void*)k_obs_pair<kObsBf16x3>, C::kSmem, kSmemSlotObsBf16x3);
        if (e != cudaSuccess) return e;
        k_obs_pair<kObsBf16x3><<<grid, kObsThreads, C::kSmem, s>>>(maps[0], maps[1], maps[2], maps[3], pairs,
                                                                   (int)npairs, (int)(n_pad / C::kBK), p, n, rp, ci,
                                                                   cv, em, ctrl, kt_of(chunk_k, C::kBK),
                                                                   kt_of(lead_k, C::kBK));
    }
    return cudaGetLastError();
}


}  // namespace hpc
