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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
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
    static constexpr int kTransBytes = 2 * 2 * kT * 4 * 4;          // threshold bits, transposed: [side][buffer][kT][4]
    static constexpr int kSmem = kStages * kStageBytes + kTransBytes + 1024 + 256;
};

constexpr int kEpiWarps = 8;
constexpr int kObsThreads = 128 + 32 * kEpiWarps;     // warpgroup 0: roles; warpgroups 1-2: epilogue
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

// Persistent pair kernel: one CTA per SM walks the pairs blockIdx.x, blockIdx.x +
// grid, ... of the pair list (bi <= bj, bands of row blocks).  For pair (I, J)
// it forms Z[I, J] = Y^T[I] X^T[J]^T / n and Z[J, I] = Y^T[J] X^T[I]^T / n and emits
// both sides.
//
// Chunked accumulation, as in the Gram: the K loop of a pair is cut into chunks
// (chunk_start), each chunk accumulates both tiles from zero into one TMEM
// accumulator pair, and the epilogue adds the chunk sums in FP32 round-to-nearest in
// registers, so the bias of the tensor core's truncating accumulation scales with
// the chunk, not with n.
//
// Roles:
//   warp 0      TMA producer (thread 0), running ahead across pairs: per chunk the
//               stages of (Y^T[I], X^T[J]), then of (Y^T[J], X^T[I]);
//   warp 1      MMA issuer (thread 32) and TMEM owner: chunk c of the CTA's sequence
//               into accumulator pair c & 1 (columns 256 (c & 1) + {0, 128} for
//               Z[I, J], Z[J, I]);
//   warps 2-3   idle (they complete warpgroup 0, which hands registers to the
//               epilogue with setmaxnreg);
//   warps 4-7   running sums of Z[I, J] (warp w: TMEM lanes 32 (w % 4) .. + 31, one
//               row of 128 columns per thread), and after the last chunk the
//               emission of the pair, row by row;
//   warps 8-11  running sums of Z[J, I] (the same lanes), staged after the last chunk
//               through shared memory, half the tile at a time, for the transpose;
//               for a diagonal pair (I = J) warps 4-7 stage their own rows.
// acc_full[b] (one commit) and acc_empty[b] (eight epilogue warps) hand the
// accumulator pairs over.  Every wait is bounded; after an abort every role stops,
// the epilogue warps keep meeting at their barriers, the loads in flight drain and
// TMEM is freed.
template <int MODE>
__global__ void __launch_bounds__(kObsThreads, 1)
k_obs_pair(const __grid_constant__ CUtensorMap ya, const __grid_constant__ CUtensorMap yb,
           const __grid_constant__ CUtensorMap xa, const __grid_constant__ CUtensorMap xb, const int2* __restrict__ pairs,
           int npairs, int k_tiles, int p, int64_t n, const int* __restrict__ rp, const int* __restrict__ ci,
           const float* __restrict__ cv, Emit<float> em, Ctrl* __restrict__ ctrl, int chunk_kt, int lead_kt) {
    using C = ObsCfg<MODE>;
    const float lam1 = (float)ctrl->lam1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint32_t* tbits = reinterpret_cast<uint32_t*>(smem + C::kStages * C::kStageBytes);   // [2][2][kT][4]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStageBytes + C::kTransBytes);
    uint64_t* empty = full + C::kStages;
    uint64_t* acc_full = empty + C::kStages;     // [2]
    uint64_t* acc_empty = acc_full + 2;          // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    static_assert(8 * (2 * C::kStages + 4) + 8 <= 256, "barrier area");
    static_assert(C::kSmem <= 232448, "shared memory per block");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int my_pairs = (int)blockIdx.x < npairs ? (npairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (chunk_kt < 1) chunk_kt = 1;
    if (lead_kt < chunk_kt) lead_kt = chunk_kt;
    const int nch = num_chunks(k_tiles, chunk_kt, lead_kt);

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) { ptx::mbar_init(&full[s], 1); ptx::mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { ptx::mbar_init(&acc_full[b], 1); ptx::mbar_init(&acc_empty[b], kEpiWarps); }
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
        // producer, MMA issuer and two idle warps: one warpgroup that gives registers away
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsSmall));
        if (threadIdx.x == 0) {
            // ---------------- producer: per chunk, phase 0 streams (Y^T[I], X^T[J]), phase 1 (Y^T[J], X^T[I])
            long long g = 0;
            bool ok = true;
            for (int lt = 0; lt < my_pairs && ok; ++lt) {
                const int2 pr = pairs[blockIdx.x + (long long)lt * gridDim.x];
                const int I0 = pr.x * kT, J0 = pr.y * kT;
                const int phases = pr.x == pr.y ? 1 : 2;
                for (int c = 0; c < nch && ok; ++c) {
                    const int kt0 = chunk_start(c, k_tiles, chunk_kt, lead_kt);
                    const int kt1 = chunk_start(c + 1, k_tiles, chunk_kt, lead_kt);
                    for (int phase = 0; phase < phases && ok; ++phase) {
                        const int ra = phase == 0 ? I0 : J0, rb = phase == 0 ? J0 : I0;
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
                            ptx::tma_load_2d(st, &ya, &full[s], kc, ra);
                            ptx::tma_load_2d(st + kPanelTile, &xa, &full[s], kc, rb);
                            if (C::kPieces > 1) {
                                ptx::tma_load_2d(st + 2 * kPanelTile, &yb, &full[s], kc, ra);
                                ptx::tma_load_2d(st + 3 * kPanelTile, &xb, &full[s], kc, rb);
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
            for (int lt = 0; lt < my_pairs && ok; ++lt) {
                const int2 pr = pairs[blockIdx.x + (long long)lt * gridDim.x];
                const int phases = pr.x == pr.y ? 1 : 2;
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
                    for (int phase = 0; phase < phases && ok; ++phase) {
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
        }
    } else {
        // the epilogue warpgroups take them: the running sums of 128 columns live in registers
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsEpi));
        // ---------------- epilogue
        // Thread (side, row-local r) owns row g = (side ? J0 : I0) + r of its tile and the
        // tile's columns c = 0..127 of the other block (column k0 + c).  The entry pair
        // {(i, j), (j, i)} is emitted when it is in the support, on the diagonal, or when
        // n |Z_ij| or n |Z_ji| exceeds lambda1 n; each side emits its own entry with its own
        // value, flagged as paired (the other side emits the partner).  A side's threshold
        // bits reach the other side transposed: per column, a warp ballot over its 32 rows
        // (tbits), so no value crosses between the warps.  A diagonal pair is one tile,
        // held by side 0, whose bits meet their own transpose.
        const int q4 = warp & 3;
        const int side = (warp - 4) >> 2;            // 0: Z[I, J] rows, 1: Z[J, I] rows
        const int r = q4 * 32 + lane;                // TMEM lane = local row
        const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(side * kT);
        // Z = (Y X) / n: the sums are tested against lambda1 n and only the emitted entries
        // are scaled.  The threshold is lowered by 2^-20 relative, so that the entries
        // emitted include every one whose scaled value exceeds lambda1 in FP32; an extra
        // entry at the threshold is harmless (its prox step leaves it at zero).
        const float inv_n = 1.0f / (float)n;
        const float thr = (float)((double)lam1 * (double)n * (1.0 - 0x1p-20));
        long long gc = 0;
        for (int lt = 0; lt < my_pairs; ++lt) {
            const int2 pr = pairs[blockIdx.x + (long long)lt * gridDim.x];
            const int I0 = pr.x * kT, J0 = pr.y * kT;
            const bool diag_pair = pr.x == pr.y;
            const bool active = side == 0 || !diag_pair;
            const int g = (side ? J0 : I0) + r;          // this thread's row
            const int k0 = side ? I0 : J0;               // its tile's first column
            // the row's support in the columns k0 .. k0 + 127: a 128-bit mask, and the CSR
            // position of its first entry there (columns ascend, so entry k of the mask sits
            // at qs + k); read before the accumulator is waited for, so that the loads'
            // latency overlaps it
            uint32_t smask[4] = {0u, 0u, 0u, 0u};
            int qs = 0;
            if (active && g < p) {
                int q = rp[g];
                const int qe = rp[g + 1];
                while (q < qe && ci[q] < k0) ++q;
                qs = q;
                for (; q < qe && ci[q] < k0 + kT; ++q) {
                    const int c = ci[q] - k0;
                    smask[c >> 5] |= 1u << (c & 31);
                }
            }
            float acc[kT];
#pragma unroll
            for (int q = 0; q < kT; ++q) acc[q] = 0.f;
            bool have = true;
            for (int c = 0; c < nch; ++c, ++gc) {
                const int b = (int)(gc & 1);
                bool got = have && !*abort_flag &&
                           ptx::mbar_wait_bounded(&acc_full[b], (uint32_t)(gc >> 1) & 1u, abort_flag, kWaitLimit);
                got = __all_sync(kFull, got);
                if (!got) { have = false; continue; }
                tc_fence_after();
                if (active) {
#pragma unroll
                    for (int s8 = 0; s8 < kT / 16; ++s8) {
                        uint32_t v[16];
                        tmem_ld16(lane_base + (uint32_t)(b * 2 * kT + s8 * 16), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc[s8 * 16 + q] += __uint_as_float(v[q]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx_arrive(&acc_empty[b]);
            }
            // own threshold bits, and their transpose by ballots: column c's word (bit l = row
            // 32 q4 + l of this warp) is kept by lane c % 32
            uint32_t own[4] = {0u, 0u, 0u, 0u}, tw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int c = 0; c < kT; ++c) {
                const bool big = active && have && g < p && !(fabsf(acc[c]) <= thr);
                own[c >> 5] |= (uint32_t)big << (c & 31);
                const uint32_t word = __ballot_sync(kFull, big);
                if ((c & 31) == lane) tw[c >> 5] = word;
            }
            // layout [side][buffer][column][warp]; the buffer alternates by pair, so the next
            // pair's words cannot overwrite words another thread still reads
            uint32_t* tb = tbits + (size_t)(lt & 1) * kT * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) tb[((side * 2) * kT + 32 * k + lane) * 4 + q4] = tw[k];
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");     // every side's bits are in
            const bool mine = active && have && g < p;
            // the other side's bits for this row: its words for column r (a diagonal pair: this side's)
            const int other = diag_pair ? 0 : 1 - side;
            uint32_t emb[4];
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t e = own[k] | tb[((other * 2) * kT + r) * 4 + k] | smask[k];
                const int lim = p - (k0 + 32 * k);              // columns k0 + 32 k + b < p
                if (lim < 32) e &= lim > 0 ? (1u << lim) - 1u : 0u;
                if (diag_pair && (r >> 5) == k) e |= 1u << (r & 31);      // the diagonal
                emb[k] = mine ? e : 0u;
                cnt += __popc(emb[k]);
            }
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
            if (!mine) continue;
            int pos = base + incl - cnt;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t em_bits = emb[k];
                while (em_bits) {
                    const int b = __ffs(em_bits) - 1;
                    em_bits &= em_bits - 1u;
                    const int c = 32 * k + b;
                    float a = 0.f;                              // acc[32 k + b] without dynamic indexing
#pragma unroll
                    for (int t = 0; t < 32; ++t) a = (t == b) ? acc[32 * k + t] : a;
                    const uint32_t sw = smask[k];
                    const bool sup = (sw >> b) & 1u;
                    int before = __popc(sw & ((1u << b) - 1u));
#pragma unroll
                    for (int t = 0; t < k; ++t) before += __popc(smask[t]);
                    if (pos < em.cap) {
                        em.row[pos] = g;
                        em.col[pos] = (int)((unsigned)(k0 + c) | 0x40000000u | (sup ? 0x80000000u : 0u));
                        em.w[pos] = __fmul_rn(a, inv_n);
                        em.om[pos] = sup ? cv[qs + before] : 0.f;
                    }
                    ++pos;
                }
            }
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
