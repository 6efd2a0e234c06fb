// Tensor-core Gram S = X^T X / n (Alg. 2 step 2) for sm_103a: tcgen05.mma with the
// accumulator in tensor memory, operands staged in shared memory by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) through an mbarrier pipeline.
//
// Operands.  The Gram is a "TN" product of X^T with itself, so X (n x p,
// row-major) is first transposed into K-major panels A = X^T (p_pad x n_pad,
// zero padded) in the MMA input type:
//   BF16X3 on FP32 X : x = hi + lo, hi = bf16(x), lo = bf16(x - hi); the tile
//                      accumulates hi*hi^T + hi*lo^T + lo*hi^T in FP32 (the
//                      dropped lo*lo^T term is below FP32 rounding of S);
//   BF16 X           : one panel, one product (bf16 x bf16 is exact in FP32);
//   TF32             : FP32 panel rounded to TF32, kind::tf32 products.
//
// Tiles.  A 128 x 256 tile S[I, J] (UMMA M = 128, N = 256) is accumulated in
// chunks of K (each from a zero TMEM accumulator, the chunk sums added in FP32
// round-to-nearest in registers).  Only the tiles that touch the upper triangle
// run, in bands of row blocks (a tuning knob) so that the tiles in flight share A
// and B panels in L2.  The product kernel writes S_ij for i <= j; a second pass
// (k_mirror_max) writes S_ji = S_ij, so S is bitwise symmetric by construction, and
// optionally the block maxima of |S| for the bound screening.
//
// Persistent kernel (384 threads, one CTA per SM): warp 0 takes tiles and issues
// TMA loads into a ring of stages, warp 1 issues MMAs from one lane and owns the
// TMEM allocation (two 256-column accumulators, so the epilogue of one chunk
// overlaps the MMAs of the next), warps 4-11 drain the accumulators (TMEM lanes
// 32 (w % 4) .. + 31, one column half each), sum the chunks, scale by 1/n and store
// the upper part of the tile.  Every mbarrier wait is bounded; on timeout the CTA
// records an error word, stops issuing, waits (bounded) for its own copies and
// MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace hpc {
namespace {

constexpr int kBM = 128;           // rows of A per tile (UMMA M)
constexpr int kBN = 256;           // rows of B per tile (UMMA N)
constexpr int kRowBytes = 128;     // one swizzle row = one K-slab of a panel row
constexpr int kABytes = kBM * kRowBytes;   // 16 KB
constexpr int kBBytes = kBN * kRowBytes;   // 32 KB
constexpr int kBand = 16;          // row blocks per band of the tile order
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitLimit = 1ll << 26;

enum : int { kModeBf16 = 0, kModeBf16x3 = 1, kModeTf32 = 2 };


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false on timeout or when another role raised the abort flag.
// The first wait to give up records its code in the launch's error word.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int code,
                                          int* err) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255) {
            if (*abort_flag) return false;
            __nanosleep(64);
        }
    }
    *abort_flag = 1;
    atomicCAS(err, 0, code);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int MODE>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
    if constexpr (MODE == kModeTf32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns: thread t gets lane (base + t).
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
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05 format): K-major, 128-byte swizzle,
// 8-row core groups 1024 bytes apart (SBO), version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // SWIZZLE_128B
    return d;
}

// Instruction descriptor: D = F32, A/B = BF16 (kind::f16) or TF32 (kind::tf32),
// both K-major, N = 256, M = 128.
template <int MODE>
__host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4)                                          // D format F32
           | ((MODE == kModeTf32 ? 2u : 1u) << 7)             // A format
           | ((MODE == kModeTf32 ? 2u : 1u) << 10)            // B format
           | ((uint32_t)(kBN >> 3) << 17)                     // N >> 3
           | ((uint32_t)(kBM >> 4) << 24);                    // M >> 4
}

template <int MODE>
struct Cfg {
    static constexpr int kPieces = (MODE == kModeBf16x3) ? 2 : 1;       // panels in smem per stage
    static constexpr int kTerms = (MODE == kModeBf16x3) ? 3 : 1;        // products per K step
    static constexpr int kElem = (MODE == kModeTf32) ? 4 : 2;
    static constexpr int kBK = kRowBytes / kElem;                      // K elements per stage
    static constexpr int kMmaK = 32 / kElem;                           // K per instruction
    static constexpr int kStageBytes = kPieces * (kABytes + kBBytes);
    static constexpr int kStages = (MODE == kModeBf16x3) ? 2 : 4;
    static constexpr int kSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers and flags*/
                                 + 8 * 32 * 17 * 4 /*per-warp staging of the row stores*/;
};

// Non-negative float rounded up to BF16 (an upper bound).
__device__ __forceinline__ uint16_t bf16_up_f(float x) {
    uint32_t u = __float_as_uint(x);
    if (u & 0xffffu) u += 0x10000u;
    return (uint16_t)(u >> 16);
}

__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent form: one CTA per SM walks the banded order of the tile list, so the
// tiles running together share X panels in L2.  Dynamic: the CTAs take tiles from a
// counter they share, so the tiles in flight stay a contiguous window of the order
// however the CTAs drift; static: CTA g takes tiles g, g + grid, ...
//
// Chunked accumulation.  The tensor core adds each MMA's K slice into the FP32
// accumulator with truncation, so a sum over the whole K = n carries a bias that
// grows with the number of MMAs chained into one accumulator (about -1.4e-4
// relative on S_ii at n = 32768).  The K loop of a tile is therefore cut into
// chunks (chunk_start): each chunk starts from a zero accumulator, and the epilogue
// adds the chunk sums in FP32 with round-to-nearest, in chunk order, in registers.
// The bias then scales with the chunk lengths instead of n (the sum over chunks of
// length^2 / K).  A chunk longer than K gives one chunk per tile.
//
// Roles:
//   warp 0      TMA producer: takes the next tile, publishes its index in a ring of
//               kTileRing slots (tid_full / tid_empty), loads its K slices ahead;
//   warp 1      MMA issuer: chunk c of the CTA's sequence into TMEM accumulator
//               c & 1 (columns 0 / 256), so a chunk accumulates while the previous
//               one is read out;
//   warps 2-3   idle (they complete warpgroup 0, which hands registers to the
//               epilogue with setmaxnreg);
//   warps 4-11  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 and the column
//               half (w - 4) / 4 of the tile (128 columns), keeps the running
//               sums of its row's 128 columns in registers, and after a tile's last
//               chunk scales by 1/n and stores the entries with i <= j (the lower
//               triangle and the block maxima come from the mirror pass).
// acc_full[b] (one commit) and acc_empty[b] (eight epilogue warps) hand the
// buffers over.  Every wait is bounded; an abort stops all roles, drains the
// loads in flight and frees TMEM.
constexpr int kEpiWarps = 8;
constexpr int kPersistThreads = 128 + 32 * kEpiWarps;     // warpgroup 0: roles; warpgroups 1-2: epilogue
// Registers per thread after setmaxnreg: warpgroup 0 gives down to kRegsSmall, the two
// epilogue warpgroups take up to kRegsEpi.  The launch's pool (threads x registers per
// thread at launch) must cover both, which the host checks before the first launch
// (kMinLaunchRegs), so that the increase never waits for registers that do not exist.
constexpr int kRegsSmall = 56;
constexpr int kRegsEpi = 216;
constexpr int kMinLaunchRegs = (128 * kRegsSmall + 32 * kEpiWarps * kRegsEpi + kPersistThreads - 1) / kPersistThreads;
constexpr int kTileRing = 4;
constexpr int kHalf = kBN / 2;          // columns per epilogue warp

// The launch's control words in the scratch's slack: the shared tile counter and the
// error word of the bounded waits, reset before each launch (by a kernel, so the reset
// is not queued behind copies on a copy engine).  Each scratch has its own, so an error
// is reported by the call whose launch hit it.
__global__ void k_zero_ctl(unsigned* ctl) { ctl[0] = 0u; ctl[1] = 0u; }

template <int MODE>
__global__ void __launch_bounds__(kPersistThreads, 1)
k_gram_tc_persist(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                  const int2* __restrict__ tiles, int ntiles, int k_tiles, int64_t p, int64_t n,
                  float* __restrict__ S, int64_t lds, unsigned* __restrict__ tile_ctr, int* __restrict__ err,
                  int dynamic, int chunk_kt, int lead_kt) {
    using C = Cfg<MODE>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStageBytes);
    uint64_t* empty = full + C::kStages;
    uint64_t* acc_full = empty + C::kStages;     // [2]
    uint64_t* acc_empty = acc_full + 2;          // [2]
    uint64_t* tid_full = acc_empty + 2;          // [kTileRing]
    uint64_t* tid_empty = tid_full + kTileRing;  // [kTileRing]: MMA thread + one epilogue thread
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tid_empty + kTileRing);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* s_tid = reinterpret_cast<volatile int*>(tmem_slot + 2);      // [kTileRing]
    volatile int* s_epi = s_tid + kTileRing;                                    // [2]
    float* s_stage = reinterpret_cast<float*>(smem + C::kStages * C::kStageBytes + 256);   // [kEpiWarps][32][17]
    static_assert(8 * (2 * C::kStages + 4 + 2 * kTileRing) + 4 * (2 + kTileRing + 2) <= 256, "barrier area");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (chunk_kt < 1) chunk_kt = 1;
    if (lead_kt < chunk_kt) lead_kt = chunk_kt;
    const int nch = num_chunks(k_tiles, chunk_kt, lead_kt);     // chunks per tile

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], kEpiWarps); }
        for (int r = 0; r < kTileRing; ++r) { mbar_init(&tid_full[r], 1); mbar_init(&tid_empty[r], 2); }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_hi)) : "memory");
        if (C::kPieces > 1) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_lo)) : "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 2 * kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    long long issued = 0;   // stages whose TMA loads were issued (producer thread)
    if (warp < 4) {
        // producer, MMA issuer and two idle warps: one warpgroup that gives registers away
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsSmall));
        if (threadIdx.x == 0) {
            // ---------------- TMA producer
            long long g = 0;
            bool ok = true;
            for (int lt = 0; ok; ++lt) {
                // the next tile of the shared order, published to the MMA and epilogue roles
                const int slot = lt % kTileRing;
                if (!mbar_wait(&tid_empty[slot], ((uint32_t)(lt / kTileRing) & 1u) ^ 1u, abort_flag, 15, err)) break;
                // dynamic: the counter shared by the CTAs; static: tiles blockIdx.x + lt * grid
                const unsigned t = dynamic ? atomicAdd(tile_ctr, 1u)
                                           : (unsigned)blockIdx.x + (unsigned)lt * (unsigned)gridDim.x;
                const int tt = t < (unsigned)ntiles ? (int)t : -1;
                s_tid[slot] = tt;
                mbar_arrive_local(&tid_full[slot]);
                if (tt < 0) break;
                const int2 tile = tiles[tt];
                const int I0 = tile.x * kBM, J0 = tile.y * kBN;
                for (int kt = 0; kt < k_tiles; ++kt, ++g) {
                    const int s = (int)(g % C::kStages);
                    const uint32_t ph = (uint32_t)(g / C::kStages) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, 11, err)) { ok = false; break; }
                    uint8_t* st = smem + s * C::kStageBytes;
                    mbar_expect_tx(&full[s], C::kStageBytes);
                    const int kc = kt * C::kBK;
                    for (int pc = 0; pc < C::kPieces; ++pc) {
                        const CUtensorMap* m = pc == 0 ? &map_hi : &map_lo;
                        uint8_t* a = st + pc * (kABytes + kBBytes);
                        uint8_t* b = a + kABytes;
                        tma_load_2d(a, m, &full[s], kc, I0);
                        tma_load_2d(b, m, &full[s], kc, J0);
                        tma_load_2d(b + kABytes, m, &full[s], kc, J0 + kBM);
                    }
                    ++issued;
                }
            }
        } else if (threadIdx.x == 32) {
            // ---------------- MMA issuer: chunk after chunk, alternating the two accumulators
            constexpr uint32_t idesc = instr_desc<MODE>();
            long long g = 0, gc = 0;
            bool ok = true;
            for (int lt = 0; ok; ++lt) {
                const int slot = lt % kTileRing;
                if (!mbar_wait(&tid_full[slot], (uint32_t)(lt / kTileRing) & 1u, abort_flag, 16, err)) break;
                const int tt = s_tid[slot];
                mbar_arrive_local(&tid_empty[slot]);
                if (tt < 0) break;
                for (int c = 0; c < nch && ok; ++c, ++gc) {
                    const int b = (int)(gc & 1);
                    if (!mbar_wait(&acc_empty[b], ((uint32_t)(gc >> 1) & 1u) ^ 1u, abort_flag, 12, err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)(b * kTmemCols);
                    const int kt0 = chunk_start(c, k_tiles, chunk_kt, lead_kt);
                    const int kt1 = chunk_start(c + 1, k_tiles, chunk_kt, lead_kt);
                    for (int kt = kt0; kt < kt1; ++kt, ++g) {
                        const int s = (int)(g % C::kStages);
                        const uint32_t ph = (uint32_t)(g / C::kStages) & 1u;
                        if (!mbar_wait(&full[s], ph, abort_flag, 13, err)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t st = smem_u32(smem + s * C::kStageBytes);
                        const uint32_t a_hi = st, b_hi = st + kABytes;
                        const uint32_t a_lo = st + (kABytes + kBBytes), b_lo = a_lo + kABytes;
    #pragma unroll
                        for (int kk = 0; kk < C::kBK / C::kMmaK; ++kk) {
                            const uint32_t off = kk * 32;
                            const uint32_t acc0 = (kt > kt0 || kk > 0) ? 1u : 0u;
                            umma<MODE>(acc, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_hi + off), idesc, acc0);
                            if constexpr (C::kTerms == 3) {
                                umma<MODE>(acc, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_lo + off), idesc, 1u);
                                umma<MODE>(acc, smem_desc_sw128(a_lo + off), smem_desc_sw128(b_hi + off), idesc, 1u);
                            }
                        }
                        umma_commit(&empty[s]);
                    }
                    if (ok) umma_commit(&acc_full[b]);
                }
            }
        }
    } else {
        // the epilogue warpgroups take them: the running sums of 128 columns live in registers
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsEpi));
        // ---------------- epilogue: chunk sums -> registers; after a tile's last chunk, the
        // scaled sums S_ij with i <= j (the owner rule; the lower triangle is written by
        // the mirror pass that follows the kernel)
        const float inv_n = 1.0f / (float)n;
        const int q4 = warp & 3;
        const int hc = (warp - 4) >> 2;                     // column half of the tile
        const int et = threadIdx.x - 128;                   // 0..255 over the epilogue warps
        const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(hc * kHalf);
        float* stg = s_stage + (warp - 4) * 32 * 17;
        // After an abort a warp keeps walking its tiles (every wait then fails at once)
        // without touching TMEM or memory, so the eight epilogue warps always meet at
        // the named barrier the same number of times.
        long long gc = 0;
        for (int lt = 0;; ++lt) {
            // the round's tile: one thread takes it from the ring, all eight warps read it
            // after the barrier (double-buffered, so the next round's write cannot race
            // this round's reads); -1 (no tile left, or an abort) ends every warp's loop
            // at the same round
            if (et == 0) {
                const int slot = lt % kTileRing;
                int tt = -1;
                if (!*abort_flag && mbar_wait(&tid_full[slot], (uint32_t)(lt / kTileRing) & 1u, abort_flag, 17, err)) {
                    tt = s_tid[slot];
                    mbar_arrive_local(&tid_empty[slot]);
                }
                s_epi[lt & 1] = tt;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
            const int tt = s_epi[lt & 1];
            if (tt < 0) break;
            float acc[kHalf];
#pragma unroll
            for (int q = 0; q < kHalf; ++q) acc[q] = 0.f;
            bool have = true;
            for (int c = 0; c < nch; ++c, ++gc) {
                const int b = (int)(gc & 1);
                bool got = have && !*abort_flag &&
                           mbar_wait(&acc_full[b], (uint32_t)(gc >> 1) & 1u, abort_flag, 14, err);
                got = __all_sync(kFull, got);
                if (!got) { have = false; continue; }
                tc_fence_after();
#pragma unroll
                for (int s4 = 0; s4 < kHalf / 16; ++s4) {
                    uint32_t v[16];
                    tmem_ld16(lane_base + (uint32_t)(b * kTmemCols + s4 * 16), v);
                    tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[s4 * 16 + q] += __uint_as_float(v[q]);
                }
                // this warp's lanes of buffer b are read: hand the buffer back
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_local(&acc_empty[b]);
            }
            if (!have) continue;
            const int2 tile = tiles[tt];
            const int I0 = tile.x * kBM, J0 = tile.y * kBN + hc * kHalf;   // this warp's columns
            // 16 columns at a time, staged through this warp's shared buffer so that each
            // store covers two rows x 64 contiguous bytes (a lane per row would write 32
            // rows x 16 bytes per instruction)
            const int ri0 = I0 + q4 * 32 + (lane >> 4);            // store row for k = 0
            const int ci = lane & 15;                              // store column in the piece
#pragma unroll
            for (int s16 = 0; s16 < kHalf / 16; ++s16) {
                const int c0 = s16 * 16;
                __syncwarp();
#pragma unroll
                for (int q = 0; q < 16; ++q) stg[lane * 17 + q] = __fmul_rn(acc[c0 + q], inv_n);
                __syncwarp();
                const int cj = J0 + c0 + ci;
                float* dst = S + (int64_t)ri0 * lds + cj;
#pragma unroll 4
                for (int k = 0; k < 16; ++k) {
                    const int ri = ri0 + 2 * k;
                    if (ri < p && cj < p && cj >= ri) dst[(int64_t)(2 * k) * lds] = stg[(2 * k + (lane >> 4)) * 17 + ci];
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) {
        // drain: bounded waits for the loads this CTA issued, so no copy lands after exit
        for (long long g = issued > C::kStages ? issued - C::kStages : 0; g < issued; ++g) {
            const int s = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)(g / C::kStages) & 1u;
            for (long long it = 0; it < (1ll << 22) && !mbar_try_wait(&full[s], ph); ++it) __nanosleep(64);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kTmemCols);
    }
}

// The lower triangle and, with m1, the block maxima, after the product kernel wrote
// S_ij for i <= j: S_ji = S_ij for i < j (bitwise, so S is exactly symmetric), and
// m1[i][jb] = max |S_ij| over the 128-column block jb with j != i and j < p, rounded
// up to BF16 (an upper bound; 0x7fc0 when the block holds a NaN).  One block of 256
// threads per 128 x 128 block pair (I <= J) of the upper triangle, in triangle order:
// the tile is read row by row (row maxima on the way), staged in shared memory, and
// written transposed row by row (column maxima on the way); both passes are
// coalesced.  A diagonal pair reads and writes only its strictly upper part, and its
// maxima combine the row (j > i) and column (j < i) parts.
constexpr int kMirT = 128;
constexpr int kMirSmem = kMirT * (kMirT + 1) * 4 + kMirT * 8;

__device__ __forceinline__ void nanmax_warp(float& mx, bool& nan) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    nan = __any_sync(kFull, nan);
}

// max that returns NaN when either operand is NaN (so a block's maximum flags a NaN)
__device__ __forceinline__ float max_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

__device__ __forceinline__ float warp_max_nan(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max_nan(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// An interior block pair (I < J, both blocks whole; rows 16-byte aligned): rows read as float4 (lane l takes
// columns 4 l .. 4 l + 3), their maxima taken from the registers, and staged in shared
// memory with column c at c + c / 32 of a 131-float row, so that both the row stores
// (eight lanes per 128-byte phase) and the column reads (32 rows of one column) hit 32
// different banks.
constexpr int kMirRow = 131;
static_assert(kMirT * kMirRow * 4 <= kMirSmem, "interior staging fits the block's shared memory");

template <bool MAXIMA>
__device__ __forceinline__ void mirror_interior(float* __restrict__ S, int64_t lds, int I0, int J0, int bi, int bj,
                                                uint16_t* __restrict__ m1, int nbm, float* t) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cs = 4 * lane + (lane >> 3);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = warp + 8 * (8 * h + q);
            v[q] = *reinterpret_cast<const float4*>(S + (int64_t)(I0 + r) * lds + J0 + 4 * lane);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = warp + 8 * (8 * h + q);
            float* row = t + r * kMirRow + cs;
            row[0] = v[q].x;
            row[1] = v[q].y;
            row[2] = v[q].z;
            row[3] = v[q].w;
            if constexpr (MAXIMA) {
                float mx = max_nan(max_nan(fabsf(v[q].x), fabsf(v[q].y)), max_nan(fabsf(v[q].z), fabsf(v[q].w)));
                mx = warp_max_nan(mx);
                if (lane == 0) m1[(int64_t)(I0 + r) * nbm + bj] = mx != mx ? (uint16_t)0x7fc0 : bf16_up_f(mx);
            }
        }
    }
    __syncthreads();
    for (int c = warp; c < kMirT; c += 8) {
        const int pc = c + (c >> 5);
        float mx = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r = lane + 32 * m;
            const float x = t[r * kMirRow + pc];
            S[(int64_t)(J0 + c) * lds + I0 + r] = x;
            if constexpr (MAXIMA) mx = max_nan(mx, fabsf(x));
        }
        if constexpr (MAXIMA) {
            mx = warp_max_nan(mx);
            if (lane == 0) m1[(int64_t)(J0 + c) * nbm + bi] = mx != mx ? (uint16_t)0x7fc0 : bf16_up_f(mx);
        }
    }
}

template <bool MAXIMA>
__global__ void __launch_bounds__(256)
k_mirror_max(float* __restrict__ S, int64_t lds, int p, int nb, uint16_t* __restrict__ m1, int nbm, int vec) {
    extern __shared__ float mir[];
    float* t = mir;                                               // [kMirT][kMirT + 1]
    float* rmax = mir + kMirT * (kMirT + 1);                      // [kMirT] upper-part row maxima
    int* rnan = reinterpret_cast<int*>(rmax + kMirT);             // [kMirT]
    // block pair (bi <= bj) of this CTA: t = bj (bj + 1) / 2 + bi
    const long long tix = blockIdx.x;
    int bj = (int)((sqrt(8.0 * (double)tix + 1.0) - 1.0) * 0.5);
    while ((long long)(bj + 1) * (bj + 2) / 2 <= tix) ++bj;
    while ((long long)bj * (bj + 1) / 2 > tix) --bj;
    const int bi = (int)(tix - (long long)bj * (bj + 1) / 2);
    if (bj >= nb) return;
    const bool dg = bi == bj;
    const int I0 = bi * kMirT, J0 = bj * kMirT;
    if (vec && !dg && J0 + kMirT <= p) {
        mirror_interior<MAXIMA>(S, lds, I0, J0, bi, bj, m1, nbm, t);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a diagonal or ragged block pair: rows of S[I, J]: warp w takes rows w, w + 8, ...; lane l columns l + 32 m.  Only
    // loads and shared stores here, so that the loads of several rows are in flight.
#pragma unroll 4
    for (int r = warp; r < kMirT; r += 8) {
        const int i = I0 + r;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int c = lane + 32 * m;
            t[r * (kMirT + 1) + c] = (i < p && (!dg || c > r)) ? S[(int64_t)i * lds + J0 + c] : 0.f;
        }
    }
    __syncthreads();
    if constexpr (MAXIMA) {
        // row maxima of the staged tile (for a diagonal pair, of its upper part)
        for (int r = warp; r < kMirT; r += 8) {
            const int i = I0 + r;
            float mx = 0.f;
            bool nan = false;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int c = lane + 32 * m;
                if (J0 + c < p && (!dg || c > r)) {
                    const float a = fabsf(t[r * (kMirT + 1) + c]);
                    nan |= !(a == a);
                    mx = fmaxf(mx, a);
                }
            }
            nanmax_warp(mx, nan);
            if (lane == 0) {
                if (dg) {
                    rmax[r] = mx;
                    rnan[r] = nan;
                } else if (i < p) {
                    m1[(int64_t)i * nbm + bj] = nan ? (uint16_t)0x7fc0 : bf16_up_f(mx);
                }
            }
        }
        __syncthreads();
    }
    // columns of the tile = rows J0 + c of the lower triangle: warp w takes c = w, w + 8, ...
    for (int c = warp; c < kMirT; c += 8) {
        const int j = J0 + c;
        if (j >= p) continue;
        float mx = 0.f;
        bool nan = false;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r = lane + 32 * m;
            const int i = I0 + r;
            if (i < p && (!dg || r < c)) {
                const float x = t[r * (kMirT + 1) + c];
                S[(int64_t)j * lds + i] = x;
                if constexpr (MAXIMA) {
                    const float a = fabsf(x);
                    nan |= !(a == a);
                    mx = fmaxf(mx, a);
                }
            }
        }
        if constexpr (MAXIMA) {
            nanmax_warp(mx, nan);
            if (lane == 0) {
                if (dg) {
                    mx = fmaxf(mx, rmax[c]);
                    nan = nan || rnan[c] != 0;
                }
                m1[(int64_t)j * nbm + bi] = nan ? (uint16_t)0x7fc0 : bf16_up_f(mx);
            }
        }
    }
}

cudaError_t launch_mirror(float* S, int64_t lds, int64_t p, uint16_t* m1, int nbm, cudaStream_t s) {
    const int nb = (int)((p + kMirT - 1) / kMirT);
    const long long pairs = (long long)nb * (nb + 1) / 2;
    if (pairs > 0x7fffffffll) return cudaErrorNotSupported;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mirror_max<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMirSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mirror_max<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMirSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // the interior blocks' float4 rows need 16-byte aligned rows: S aligned and lds a multiple of 4
    const int vec = (lds % 4 == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0) ? 1 : 0;
    if (m1) k_mirror_max<true><<<(unsigned)pairs, 256, kMirSmem, s>>>(S, lds, (int)p, nb, m1, nbm, vec);
    else k_mirror_max<false><<<(unsigned)pairs, 256, kMirSmem, s>>>(S, lds, (int)p, nb, nullptr, 0, vec);
    return cudaGetLastError();
}

// Transpose X (n x p) into K-major panels (p_pad x n_pad) of the MMA input type,
// 32 x 32 tiles: one per block, or a grid-stride loop over them when the grid is
// smaller (a staging that shares the GPU with a solve).
template <typename TX, int MODE>
__global__ void __launch_bounds__(256)
k_prep(const TX* __restrict__ X, int64_t n, int64_t p, void* __restrict__ hi, void* __restrict__ lo,
       int64_t n_pad, int64_t p_pad) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const int64_t nkt = (n_pad + 31) / 32, ntiles = nkt * ((p_pad + 31) / 32);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t k0 = (t % nkt) * 32, i0 = (t / nkt) * 32;
        __syncthreads();        // the previous tile's reads of the shared tile are done
        for (int r = ty; r < 32; r += 8) {
            const int64_t k = k0 + r, i = i0 + tx;
            float v = 0.f;
            if (k < n && i < p) {
                if constexpr (std::is_same<TX, __nv_bfloat16>::value) v = __bfloat162float(X[k * p + i]);
                else v = (float)X[k * p + i];
            }
            tile[r][tx] = v;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int64_t i = i0 + r, k = k0 + tx;
            if (i >= p_pad || k >= n_pad) continue;
            const float x = tile[tx][r];
            const int64_t o = i * n_pad + k;
            if constexpr (MODE == kModeTf32) {
                uint32_t tf;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(tf) : "f"(x));
                static_cast<float*>(hi)[o] = __uint_as_float(tf);
            } else {
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                static_cast<__nv_bfloat16*>(hi)[o] = h;
                if constexpr (MODE == kModeBf16x3)
                    static_cast<__nv_bfloat16*>(lo)[o] = __float2bfloat16_rn(x - __bfloat162float(h));
            }
        }
    }
}

// BF16 X into the BF16 panel: a transpose of 64 (k) x 128 (i) tiles with 16-byte
// global loads and stores (vec: rows of X start on 16-byte boundaries).  In the
// shared tile the 16-byte chunks of row r sit XOR-swizzled by (r / 8) % 8, so the
// column reads of the store phase -- the 8 k-groups of a warp at the same columns --
// fall on 8 different chunks, all 32 banks.  A thread reads 32-bit words (two
// adjacent i) and writes the two output rows.
__device__ __forceinline__ int prep_col(int r, int col) { return (((col >> 3) ^ ((r >> 3) & 7)) << 3) | (col & 7); }

__global__ void __launch_bounds__(256)
k_prep_bf16(const uint16_t* __restrict__ X, int64_t n, int64_t p, uint16_t* __restrict__ out, int64_t n_pad,
            int64_t p_pad, int vec) {
    __shared__ __align__(16) uint16_t t[64][128];
    const int tid = threadIdx.x;
    const int64_t nkt = n_pad / 64, ntiles = nkt * (p_pad / 128);
    // one tile per block, or a grid-stride loop when the grid is smaller (a staging
    // that shares the GPU with a solve)
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t k0 = (tile % nkt) * 64, i0 = (tile / nkt) * 128;
        __syncthreads();        // the previous tile's reads of t are done
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int r = tid / 16 + rr * 16, ch = tid % 16;
            const int64_t k = k0 + r, i = i0 + ch * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (k < n) {
                if (vec && i + 8 <= p) {
                    v = *reinterpret_cast<const uint4*>(X + k * p + i);
                } else {
                    uint16_t e[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) e[q] = (i + q < p) ? X[k * p + i + q] : (uint16_t)0;
                    v = make_uint4(e[0] | ((uint32_t)e[1] << 16), e[2] | ((uint32_t)e[3] << 16),
                                   e[4] | ((uint32_t)e[5] << 16), e[6] | ((uint32_t)e[7] << 16));
                }
            }
            *reinterpret_cast<uint4*>(&t[r][prep_col(r, ch * 8)]) = v;
        }
        __syncthreads();
        // 64 row pairs x 8 k-groups, two per thread; n_pad and p_pad are multiples of 64
        // and 128, so every output row and k-group of the tile is inside the panel
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int kg = tid % 8, il = 2 * (tid / 8 + rr * 32);
            uint32_t a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r0 = 8 * kg + 2 * q, r1 = r0 + 1;
                const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&t[r0][prep_col(r0, il)]);
                const uint32_t w1 = *reinterpret_cast<const uint32_t*>(&t[r1][prep_col(r1, il)]);
                a[q] = (w0 & 0xffffu) | (w1 << 16);               // row il:     k = r0, r1
                b[q] = (w0 >> 16) | (w1 & 0xffff0000u);           // row il + 1: k = r0, r1
            }
            const int64_t i = i0 + il, k = k0 + 8 * kg;
            *reinterpret_cast<uint4*>(out + i * n_pad + k) = make_uint4(a[0], a[1], a[2], a[3]);
            *reinterpret_cast<uint4*>(out + (i + 1) * n_pad + k) = make_uint4(b[0], b[1], b[2], b[3]);
        }
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

int mode_of(int xdt, int precision) {
    if (precision == HPC_PREC_TF32) return kModeTf32;
    return xdt == HPC_BF16 ? kModeBf16 : kModeBf16x3;
}

struct Geometry {
    int64_t p_pad, n_pad;
    size_t panel_bytes;
    int pieces;
    int64_t ntiles;
};

Geometry geometry(int xdt, int64_t n, int64_t p, int precision) {
    const int mode = mode_of(xdt, precision);
    Geometry g;
    g.p_pad = (p + kBN - 1) / kBN * kBN;
    g.n_pad = (n + 63) / 64 * 64;
    const int es = mode == kModeTf32 ? 4 : 2;
    g.panel_bytes = (size_t)g.p_pad * g.n_pad * es;
    g.panel_bytes = (g.panel_bytes + 1023) / 1024 * 1024;
    g.pieces = mode == kModeBf16x3 ? 2 : 1;
    const int64_t nbi = g.p_pad / kBM, nbj = g.p_pad / kBN;
    int64_t t = 0;
    for (int64_t bj = 0; bj < nbj; ++bj) t += std::min<int64_t>(2 * bj + 2, nbi);
    g.ntiles = t;
    return g;
}

// Upper-triangle tiles (128 bi <= 256 bj + 255) in bands of `band` row blocks;
// within a band, columns left to right, rows top to bottom.  The band sets
// which X panels the concurrently running tiles share in L2 (a tuning knob).
std::vector<int2> tile_order(int64_t p_pad, int band) {
    const int64_t nbi = p_pad / kBM, nbj = p_pad / kBN;
    std::vector<int2> t;
    for (int64_t b0 = 0; b0 < nbi; b0 += band)
        for (int64_t bj = 0; bj < nbj; ++bj)
            for (int64_t bi = b0; bi < std::min<int64_t>(b0 + band, nbi); ++bi)
                if (bi * kBM <= bj * kBN + kBN - 1) t.push_back(make_int2((int)bi, (int)bj));
    return t;
}

// The tile counter and the error word: after the tile list, in the scratch's slack.
unsigned* ctl_words(const int2* tiles, const Geometry& g) {
    return reinterpret_cast<unsigned*>((reinterpret_cast<uintptr_t>(tiles + g.ntiles) + 255) & ~uintptr_t(255));
}

bool make_map(CUtensorMap* m, void* base, int mode, const Geometry& g) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int es = mode == kModeTf32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)g.n_pad, (cuuint64_t)g.p_pad};
    cuuint64_t strides[1] = {(cuuint64_t)g.n_pad * es};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / es), (cuuint32_t)kBM};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, mode == kModeTf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// K elements per accumulation chunk when the caller gives none: the S_ii bias of a
// chunk grows with the MMAs chained into it, so 32 MMAs for one product per K step
// (BF16 X) and 48 for the three of BF16X3 keep it near 1e-6 relative (measured
// -9.5e-7 on the diagonal at n = 32768, against -1.4e-4 for one chunk over all of K).
// Shorter chunks leave the tensor core idle while the epilogue reads them out.  The
// first two chunks of a tile are twice as long (lead_k), which covers the epilogue's
// stores of the previous tile.
template <int MODE>
constexpr int default_chunk_k() { return MODE == kModeBf16 ? 512 : 256; }

// The product kernel, then the mirror pass (lower triangle and, with m1, the block
// maxima); after_kernel (nullable) is recorded between the two.
template <int MODE>
cudaError_t launch_mode(const Geometry& g, void* hi, void* lo, const int2* tiles, int64_t n, int64_t p, float* S,
                        int64_t lds, cudaStream_t s, uint16_t* m1 = nullptr, int nbm = 0, int dynamic = 1,
                        int64_t chunk_k = 0, int64_t lead_k = 0, cudaEvent_t after_kernel = nullptr) {
    using C = Cfg<MODE>;
    if (chunk_k <= 0) chunk_k = default_chunk_k<MODE>();
    if (lead_k <= 0) lead_k = std::min<int64_t>(2 * chunk_k, (int64_t)1 << 40);
    const int chunk_kt = (int)std::max<int64_t>(1, std::min<int64_t>(chunk_k / C::kBK, 1 << 30));
    const int lead_kt = (int)std::max<int64_t>(chunk_kt, std::min<int64_t>(lead_k / C::kBK, 1 << 30));
    CUtensorMap mh, ml;
    std::memset(&mh, 0, sizeof mh);
    std::memset(&ml, 0, sizeof ml);
    if (!make_map(&mh, hi, MODE, g)) return cudaErrorNotSupported;
    if (C::kPieces > 1 && !make_map(&ml, lo, MODE, g)) return cudaErrorNotSupported;
    if (C::kPieces == 1) ml = mh;
    const int k_tiles = (int)(g.n_pad / C::kBK);
    cudaError_t e =
        cudaFuncSetAttribute(k_gram_tc_persist<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    // setmaxnreg moves registers between the warpgroups of a block: the kernel must have
    // been built with enough registers per thread for both shares (else it would wait)
    static int regs = -1;
    if (regs < 0) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, k_gram_tc_persist<MODE>)) != cudaSuccess) return e;
        regs = fa.numRegs;
    }
    if (regs < kMinLaunchRegs) return cudaErrorNotSupported;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(g.ntiles, sms);
    unsigned* ctl = ctl_words(tiles, g);
    k_zero_ctl<<<1, 1, 0, s>>>(ctl);
    k_gram_tc_persist<MODE><<<grid, kPersistThreads, C::kSmem, s>>>(mh, ml, tiles, (int)g.ntiles, k_tiles, p, n, S,
                                                                   lds, ctl, reinterpret_cast<int*>(ctl + 1),
                                                                   dynamic, chunk_kt, lead_kt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (after_kernel && (e = cudaEventRecord(after_kernel, s)) != cudaSuccess) return e;
    return launch_mirror(S, lds, p, m1, nbm, s);
}

// max_blocks > 0 bounds the BF16 transpose's grid (it then loops over its tiles).
template <typename TX>
void launch_prep(const void* X, int mode, int64_t n, int64_t p, void* hi, void* lo, const Geometry& g,
                 cudaStream_t s, int max_blocks = 0) {
    const TX* x = static_cast<const TX*>(X);
    if constexpr (std::is_same<TX, __nv_bfloat16>::value) {
        if (mode == kModeBf16) {
            // n_pad is a multiple of 64 and p_pad of 256: every tile is inside the panel
            const int vec = (p % 8 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0) ? 1 : 0;
            const int64_t ntiles = (g.n_pad / 64) * (g.p_pad / 128);
            const int64_t grid = max_blocks > 0 ? std::min<int64_t>(ntiles, max_blocks) : ntiles;
            // the shared-memory configuration of the large-shared-memory kernels, so that a
            // staging transpose can share SMs with the solve's kernels
            static std::once_flag carve;
            std::call_once(carve, [] {
                cudaFuncSetAttribute(k_prep_bf16, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
            });
            k_prep_bf16<<<(unsigned)grid, 256, 0, s>>>(reinterpret_cast<const uint16_t*>(X), n, p,
                                                      static_cast<uint16_t*>(hi), g.n_pad, g.p_pad, vec);
            return;
        }
    }
    const int64_t ntiles = ((g.n_pad + 31) / 32) * ((g.p_pad + 31) / 32);
    const unsigned grid = (unsigned)(max_blocks > 0 ? std::min<int64_t>(ntiles, max_blocks) : ntiles);
    if (mode == kModeTf32) k_prep<TX, kModeTf32><<<grid, 256, 0, s>>>(x, n, p, hi, lo, g.n_pad, g.p_pad);
    else if (mode == kModeBf16x3) k_prep<TX, kModeBf16x3><<<grid, 256, 0, s>>>(x, n, p, hi, lo, g.n_pad, g.p_pad);
    else k_prep<TX, kModeBf16><<<grid, 256, 0, s>>>(x, n, p, hi, lo, g.n_pad, g.p_pad);
}

}  // namespace

size_t gram_tc_scratch_bytes(int xdt, int64_t n, int64_t p, int precision) {
    const Geometry g = geometry(xdt, n, p, precision);
    return g.pieces * g.panel_bytes + (size_t)g.ntiles * sizeof(int2) + 1024;
}

static cudaError_t check_shape(int xdt, int64_t n, int64_t p, int precision, size_t scratch_bytes) {
    if (precision != HPC_PREC_BF16X3 && precision != HPC_PREC_TF32) return cudaErrorInvalidValue;
    if (xdt == HPC_F64) return cudaErrorNotSupported;
    if (!encode_fn()) return cudaErrorNotSupported;
    const Geometry g = geometry(xdt, n, p, precision);
    if (g.ntiles > 0x7fffffff || g.n_pad / 64 > 0x7fffffff || g.p_pad > 0x7fffffff) return cudaErrorNotSupported;
    if (scratch_bytes < gram_tc_scratch_bytes(xdt, n, p, precision)) return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t gram_tc_prepare(const void* X, int xdt, int64_t n, int64_t p, int precision, void* scratch,
                            size_t scratch_bytes, cudaStream_t s, int max_blocks) {
    cudaError_t e = check_shape(xdt, n, p, precision, scratch_bytes);
    if (e != cudaSuccess) return e;
    const int mode = mode_of(xdt, precision);
    const Geometry g = geometry(xdt, n, p, precision);
    uint8_t* base = static_cast<uint8_t*>(scratch);
    void* hi = base;
    void* lo = g.pieces > 1 ? base + g.panel_bytes : nullptr;
    if (xdt == HPC_BF16) launch_prep<__nv_bfloat16>(X, mode, n, p, hi, lo, g, s, max_blocks);
    else launch_prep<float>(X, mode, n, p, hi, lo, g, s, max_blocks);
    return cudaGetLastError();
}

cudaError_t gram_tc(const void* X, int xdt, int64_t n, int64_t p, float* S, int64_t lds, int precision,
                    void* scratch, size_t scratch_bytes, cudaStream_t s, int* launches, int band,
                    cudaEvent_t before_kernel, uint16_t* m1, int nbm, int prepared, uint64_t* tiles_sig,
                    int schedule, int64_t chunk_k, int64_t lead_k, cudaEvent_t after_kernel) {
    if (band <= 0) band = kBand;
    cudaError_t e = check_shape(xdt, n, p, precision, scratch_bytes);
    if (e != cudaSuccess) return e;
    const int mode = mode_of(xdt, precision);
    const Geometry g = geometry(xdt, n, p, precision);
    uint8_t* base = static_cast<uint8_t*>(scratch);
    void* hi = base;
    void* lo = g.pieces > 1 ? base + g.panel_bytes : nullptr;
    int2* tiles = reinterpret_cast<int2*>(base + g.pieces * g.panel_bytes);
    // the tile order depends on p_pad and the band only: with tiles_sig the caller keeps
    // it on the device between calls (no copy queued behind other transfers)
    const uint64_t sig = (reinterpret_cast<uintptr_t>(tiles) * 1000003ull) ^ ((uint64_t)g.p_pad << 20) ^ (uint64_t)band;
    if (!tiles_sig || *tiles_sig != sig) {
        const std::vector<int2> order = tile_order(g.p_pad, band);
        e = cudaMemcpyAsync(tiles, order.data(), order.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        // the host vector must outlive the copy
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (tiles_sig) *tiles_sig = sig;
    }
    if (!prepared) {
        if (xdt == HPC_BF16) launch_prep<__nv_bfloat16>(X, mode, n, p, hi, lo, g, s);
        else launch_prep<float>(X, mode, n, p, hi, lo, g, s);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) *launches += 1;
    }
    if (launches) *launches += 1;
    if (before_kernel && (e = cudaEventRecord(before_kernel, s)) != cudaSuccess) return e;
    if (mode == kModeBf16)
        return launch_mode<kModeBf16>(g, hi, lo, tiles, n, p, S, lds, s, m1, nbm, schedule, chunk_k, lead_k,
                                        after_kernel);
    if (mode == kModeBf16x3)
        return launch_mode<kModeBf16x3>(g, hi, lo, tiles, n, p, S, lds, s, m1, nbm, schedule, chunk_k, lead_k,
                                        after_kernel);
    return launch_mode<kModeTf32>(g, hi, lo, tiles, n, p, S, lds, s, m1, nbm, schedule, chunk_k, lead_k,
                                        after_kernel);
}

int gram_tc_take_error(const void* scratch, int xdt, int64_t n, int64_t p, int precision, cudaStream_t s) {
    if (!scratch) return 0;                 // no Gram ran on this scratch
    const Geometry g = geometry(xdt, n, p, precision);
    const int2* tiles = reinterpret_cast<const int2*>(static_cast<const uint8_t*>(scratch) + g.pieces * g.panel_bytes);
    const int* err = reinterpret_cast<const int*>(ctl_words(tiles, g) + 1);
    int v = 0;
    if (cudaMemcpyAsync(&v, err, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return v;
}

// ------------------------------------------------------------------ allocation-free variant
//
// hpc_gram_noalloc runs the same tensor-core Gram as hpc_gram, but takes its
// scratch (the transposed operand panels and the tile list) from the fixed
// device array below instead of allocating.  It exists for callers that must
// not allocate device memory while they run: code whose device memory is owned
// by another allocator (a framework's caching allocator that has reserved the
// budget, so a raw cudaMalloc fails or fragments it), services with a fixed
// memory budget decided at start-up, and latency-critical loops where
// cudaMalloc/cudaFree would synchronise the device.
//
// The array costs kNoAllocScratchBytes of memory on every GPU that loads the
// library's device code, held until the process exits.  Under CUDA's default lazy
// module loading that happens at the first call on each device (the symbol lookup
// loads the module), so that first call reserves the 64 MiB: make it at start-up,
// or load modules eagerly (CUDA_MODULE_LOADING=EAGER).  All calls share it and it keeps the
// last call's contents: every byte a call reads is first written by that call
// (the panels, padding included, and the tile list), and calls that overlap on
// the GPU (other streams, other host threads) race on it.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;     // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_base[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

// The tile order of tile_order(), written on the device (no host staging buffer).
__global__ void k_tile_order(int2* __restrict__ out, int64_t p_pad) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t nbi = p_pad / kBM, nbj = p_pad / kBN;
    int64_t t = 0;
    for (int64_t b0 = 0; b0 < nbi; b0 += kBand)
        for (int64_t bj = 0; bj < nbj; ++bj)
            for (int64_t bi = b0; bi < (b0 + kBand < nbi ? b0 + kBand : nbi); ++bi)
                if (bi * kBM <= bj * kBN + kBN - 1) out[t++] = make_int2((int)bi, (int)bj);
}

// Device address of the scratch array for the current device; the first call on
// a device looks it up (cudaGetSymbolAddress with that device current).
cudaError_t noalloc_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace hpc

extern "C" int hpc_gram_noalloc(const void* X, hpc_dtype xdt, int64_t n, int64_t p, float* S, int64_t lds,
                                int precision, void* cuda_stream) {
    using namespace hpc;
    if (!X || !S || n < 1 || p < 1 || lds < p || (xdt != HPC_F32 && xdt != HPC_BF16)) return HPC_ERR_ARG;
    if (precision == HPC_PREC_AUTO) precision = HPC_PREC_BF16X3;
    if (precision != HPC_PREC_BF16X3 && precision != HPC_PREC_TF32) return HPC_ERR_ARG;
    const size_t need = gram_tc_scratch_bytes(xdt, n, p, precision);
    if (need > kNoAllocScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "hpc_gram_noalloc: n=%lld p=%lld needs %zu bytes of scratch; the static scratch holds %zu",
                      (long long)n, (long long)p, need, kNoAllocScratchBytes);
        set_last_error(msg);
        return HPC_ERR_ARG;
    }
    if (!encode_fn()) {
        set_last_error("hpc_gram_noalloc: the driver's TMA descriptor encoder is not available");
        return HPC_ERR_NOT_IMPLEMENTED;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    void* base_v = nullptr;
    cudaError_t e = noalloc_base(&base_v);
    if (e != cudaSuccess) {
        set_last_error("hpc_gram_noalloc: cudaGetSymbolAddress of the static scratch failed");
        return HPC_ERR_CUDA;
    }
    const int mode = mode_of(xdt, precision);
    const Geometry g = geometry(xdt, n, p, precision);
    uint8_t* base = static_cast<uint8_t*>(base_v);
    void* hi = base;
    void* lo = g.pieces > 1 ? base + g.panel_bytes : nullptr;
    int2* tiles = reinterpret_cast<int2*>(base + g.pieces * g.panel_bytes);
    k_tile_order<<<1, 1, 0, s>>>(tiles, g.p_pad);
    if (xdt == HPC_BF16) launch_prep<__nv_bfloat16>(X, mode, n, p, hi, lo, g, s);
    else launch_prep<float>(X, mode, n, p, hi, lo, g, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        if (mode == kModeBf16) e = launch_mode<kModeBf16>(g, hi, lo, tiles, n, p, S, lds, s);
        else if (mode == kModeBf16x3) e = launch_mode<kModeBf16x3>(g, hi, lo, tiles, n, p, S, lds, s);
        else e = launch_mode<kModeTf32>(g, hi, lo, tiles, n, p, S, lds, s);
    }
    if (e == cudaErrorNotSupported) {
        set_last_error("hpc_gram_noalloc: the tensor-core Gram is not available for this shape or build");
        return HPC_ERR_NOT_IMPLEMENTED;
    }
    // the launch's error word sits in the static scratch (shared by overlapping calls)
    const int w = e == cudaSuccess ? gram_tc_take_error(base_v, xdt, n, p, precision, s) : 0;
    if (e == cudaSuccess && w < 0) e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof msg, "hpc_gram_noalloc: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return HPC_ERR_CUDA;
    }
    if (w != 0) {
        char msg[128];
        std::snprintf(msg, sizeof msg, "hpc_gram_noalloc: bounded wait %d gave up", w);
        set_last_error(msg);
        return HPC_ERR_DEVICE_TIMEOUT;
    }
    return HPC_OK;
}
