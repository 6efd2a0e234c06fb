// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "hpconcord.h"

namespace hpc {

constexpr unsigned kFull = 0xffffffffu;

// Device-resident control block of one solver handle.  Kernels write it; the
// host reads it back (one small copy) at the two synchronisation points of an
// outer iteration.
struct Ctrl {
    int em_count;        // entries emitted by the gradient-screening pass
    int bucket_total;    // entries of the symmetric candidate structure (before de-dup)
    int flags;           // kFlag* bits
    int ls_accept;       // accepted number of halvings h (tau = 2^-h), -1 while searching
    int ls_base;         // first h of the next line-search window
    int nnz_next;        // entries of the accepted iterate
    int converged;       // relative change < eps
    int iter;            // outer iterations done since the last reset
    double tau;          // accepted step
    double f_cur;        // smooth part f(Omega^k)
    double pen_cur;      // lambda1 * sum_{i != j} |w_ij| at Omega^k
    double norm2_cur;    // ||Omega^k||_F^2
    double delta2;       // ||Omega^{k+1} - Omega^k||_F^2 for the accepted tau
    double rel;          // sqrt(delta2 / norm2_cur)
    long long ls_trials; // accumulated trials (the paper's t)
    int n_offrows;       // rows of the iterate with off-diagonal entries (screening pass)
    int n_mirror;        // partner entries whose W_ij the gather fill computes
    double lam1, lam2;   // regularisation of the current solve (read by the kernels)
    long long ls_windows;     // line-search launches (window evaluations) since the last reset
    long long iter_attempts;  // outer iterations started since the last reset
    long long screen_ns;      // device time of the screening passes (device-loop timing)
    long long t_stamp;        // last timestamp of k_stamp
    int nnz_cur;         // entries of the current iterate (device loop)
    int iter_limit;      // the device loop stops after this many accepted iterations
    int use_stop;        // the device loop stops at the stopping rule
    int obs_next;        // next block pair of the Obs pair kernel (shared tile counter)
    // lambda path in one launch: point index, estimate staging offset (both advanced
    // by the next point's begin kernel), and the point's start time
    int path_pt, path_pt_next;
    int path_k, path_keep;        // points; 1 = resume the current point (after a regrow)
    long long path_off, path_off_next, path_need;
    long long t_point;
    int path_full;                // 1 = the estimate staging buffer is full
    int ls_done;                  // blocks of the running line-search launch that wrote their partials
    int n_long, pad4_;            // rows of the candidate structure with more than kShortRow entries
    int n_pairs, n_row_items;     // items the bound screening keeps (pure rows; rows with neighbours)
};

// Rows with at most this many candidate entries (before de-dup) are handled one
// lane per row by the candidate, line-search and compaction kernels.
constexpr int kShortRow = 2;

enum : int {
    kFlagEmOverflow = 1,
    kFlagBucketOverflow = 2,
    kFlagNaN = 4,
    kFlagLsFail = 8,
    kFlagNnzOverflow = 16,
    kFlagBadStructure = 32,
    kFlagTimeout = 64,      // a bounded device-side wait gave up
};

// Flags on candidate entries.
enum : unsigned char { kEntSupp = 1, kEntOwn = 2, kEntMirror = 4, kEntKeep = 8 };

template <typename T>
struct Csr {
    int* rp;
    int* ci;
    T* cv;
};

// Output of the screening pass: one record per emitted (i, j).
template <typename T>
struct Emit {
    int* row;
    int* col;     // bit 31 set: (i, j) is in the support of the iterate
    T* w;         // W_ij = (Omega S)_ij
    T* om;        // w_ij (0 off the support)
    int cap;
};

// Per-row candidate structure (symmetric pattern, columns ascending after sort).
// Per-tile sums of the multi-block row-count scan: entries, long rows, their line-search units.
struct ScanPart {
    int s;
    int l;
    long long u;
};

template <typename T>
struct Buckets {
    int* cnt;     // p: entries per row before de-dup
    int* off;     // p+1: row offsets
    int* cur;     // p: scatter cursors
    int* len;     // p: entries per row after de-dup
    int* col_a; T* w_a; T* om_a; unsigned char* fl_a;    // scattered
    int* col_b; T* w_b; T* om_b; unsigned char* fl_b;    // sorted, de-duplicated
    T* g;         // G_ij of the sorted entries
    long long* uoff;  // nlong+1: prefix of line-search work units over the long rows
    int* longlist;    // p: rows with more than kShortRow entries before de-dup, ascending
    int2* mir;    // cap: (position, row) of every kept partner entry
    int cap;
};

// ---------------------------------------------------------------- launchers (iterate.cu)
template <typename T>
struct IterBufs {
    const T* S;
    int64_t ld;
    int p;
    Csr<T> cur;
    Csr<T> next;
    int csr_cap;
    Emit<T> em;
    Buckets<T> bk;
    int* cnt2;            // p: per-row entry counts of the accepted iterate
    ScanPart* scan_part;  // ceil(p / 4096): per-tile sums of the row-count scans
    double* part_obj;     // objective partials   [nblk][4]
    double* part_ls;      // line-search partials [nblk][16][4]
    int nblk;             // blocks of the warp-per-row kernels
    Ctrl* ctrl;
    T lam1, lam2;
    double eps;
    int max_halvings;
    int ls_window;
    const CUtensorMap* smap;  // TMA descriptor of S (rows p, columns ld), 64 x BJ boxes
    int4* rinfo;              // p: CSR bounds, diagonal position, pure-diagonal flag of each row
    int* offlist;             // p: rows with off-diagonal entries
    T* rdv;                   // ld (zero padded): diagonal value of each row
    unsigned* pmask;          // ld/32: pure-diagonal bit of each row
    const long long* seqoff;  // screening pass: prefix of the folded tile sequence
    int screen_grid;          // screening pass: CTAs
    int ls_blocks_per_sm;     // line-search evaluation: resident blocks per SM (0 = occupancy)
    int rows_ctas_per_sm;     // off-diagonal row kernel: CTAs per SM
    // bound screening of the pure-diagonal rows
    const unsigned short* m1; // p x nbm: max |S_ij| over column block jb, j != i, as BF16 rounded up
                              // (an upper bound; null: no bound screening)
    int nbm;                  // column blocks of width BJ
    const unsigned short* m1g;  // p x ngl (nbm % 8 == 0, else null): m1's maximum over each group of
                                // 8 blocks
    int ngl;                  // row stride of m1g: nbm / 8 rounded up to a multiple of 8
    void* colmax;             // nbm words: max |w_jj| over the pure rows j of each block (T's bits)
    int2* pairs;              // kept (row, block) items
    int pairs_cap;            // above this many items the pass streams the upper triangle instead
    int2* row_items;          // rows with neighbours: kept (8-row group, block) items of the row kernel
    int row_items_cap;
    int num_sms;
    // Obs variant: X^T (p x ldx, FP32) and n
    const float* xt;
    int64_t ldx;
    int64_t n;
    unsigned* bar;            // kBarWords: arrival counter of the fused tail's grid barriers
};

// Device-side loop control (CUDA graph conditional nodes); use = 0 outside a graph.
struct LoopCond {
    int use = 0;
    cudaGraphConditionalHandle ls = 0;    // line-search window loop
    cudaGraphConditionalHandle iter = 0;  // outer iteration loop
};

template <typename T> void launch_iter_begin(const IterBufs<T>& b, const LoopCond& lc, cudaStream_t s);
template <typename T> void launch_commit(const IterBufs<T>& b, const LoopCond& lc, cudaStream_t s);
void launch_stamp(Ctrl* ctrl, int end, cudaStream_t s);
// lambda path in one launch (device loop): per-point set-up and bookkeeping
struct PathOut {
    const double* lam1;          // k
    hpc_path_point* points;      // k
    int64_t* rp;                 // k*(p+1) or null: estimates' row offsets
    int32_t* ci;                 // cap
    float* cv;                   // cap
    long long cap;
    int k;
};
void launch_point_begin(Ctrl* ctrl, PathOut out, const LoopCond& lc, cudaStream_t s);
template <typename T> void launch_point_end(const IterBufs<T>& b, PathOut out, cudaGraphConditionalHandle path_cond,
                                            cudaStream_t s);
template <typename T> void launch_grad_screen(const IterBufs<T>& b, cudaStream_t s);
template <typename T> void launch_candidates(const IterBufs<T>& b, cudaStream_t s);
template <typename T> void launch_ls_window(const IterBufs<T>& b, const LoopCond& lc, cudaStream_t s);
template <typename T> void launch_accept(const IterBufs<T>& b, cudaStream_t s);
template <typename T> void launch_set_identity(Csr<T> c, int p, cudaStream_t s);
template <typename T> void launch_csr_export(const int* rp, const int* ci, const T* cv, int p, int nnz,
                                             int64_t* rp64, int32_t* ci_out, void* val, int vdt,
                                             cudaStream_t s);
void launch_gather_s(const void* S, int is_f64, int64_t ld, int64_t m, const int64_t* rows,
                     const int64_t* cols, double* out, cudaStream_t s);

constexpr int kLaunchesScreen = 6;
constexpr int kLaunchesBegin = 1;
constexpr int kLaunchesCandidates = 7;
constexpr int kLaunchesLsWindow = 1;     // k_ls_eval (its last block decides)
constexpr int kLaunchesAccept = 4;
constexpr int kLaunchesTail = 1;         // k_iter_tail: candidates, gradient, every window, accept
// Words of the fused tail's barrier buffer, one 128-byte line: word 0 the arrival
// counter (k_iter_begin zeroes it), word 1 the count of the one-time check that
// cooperative kernels run in graph loops.
constexpr int kBarWords = 32;

// The fused iteration tail (candidates, gradient, line-search windows with their
// decisions, compaction and stopping rule) as one cooperative launch.  obs selects
// the Obs form of the window evaluation.  Returns the launch's error code.
template <typename T> cudaError_t launch_tail(const IterBufs<T>& b, bool obs, cudaStream_t s);
// Blocks of that launch for these buffers (resident blocks per SM x SMs, at most nblk).
template <typename T> int tail_grid(const IterBufs<T>& b, bool obs);

// One cooperative launch of a one-block kernel that adds 1 to *out and sets cond to 0.
cudaError_t launch_tail_probe(int* out, cudaGraphConditionalHandle cond, cudaStream_t s);

template <typename T> void launch_row_info(int p, Csr<T> om, int4* rinfo, T* rdv, cudaStream_t s);
// max |S_ij| per (row, column block of width screen_box_cols), off the diagonal
template <typename T> void launch_rowblock_max(const T* S, int64_t ld, int p, int nbm, unsigned short* m1,
                                               cudaStream_t s);
// m1g[i][g] = max over blocks 8g .. 8g+7 of m1[i][.] (nbm % 8 == 0), once per data load.
void launch_group_max(const unsigned short* m1, int p, int nbm, unsigned short* m1g, int ngl, cudaStream_t s);
template <typename T> int screen_plan(int p, int num_sms, std::vector<long long>& seqoff);
void launch_ls_window_obs(const IterBufs<float>& b, const LoopCond& lc, cudaStream_t s);

// ---------------------------------------------------------------- Obs variant (obs_tc.cu)
size_t obs_panel_bytes(int precision, int64_t n, int64_t p);
int obs_pieces(int precision);
int64_t obs_npairs(int64_t p);
void obs_pair_list(int64_t p, std::vector<int2>& out);
void launch_obs_split(int precision, const float* in, int64_t rows, int64_t cols, int64_t ldi, void* hi, void* lo,
                      int64_t n, int64_t p, cudaStream_t s);
bool obs_make_maps(int precision, const void* y_hi, const void* y_lo, const void* x_hi, const void* x_lo, int64_t n,
                   int64_t p, CUtensorMap* maps);
cudaError_t launch_obs_pairs(int precision, const CUtensorMap* maps, const int2* pairs, int64_t npairs, int64_t n,
                             int p, const int* rp, const int* ci, const float* cv, Emit<float> em,
                             Ctrl* ctrl, cudaStream_t s, int64_t chunk_k = 0, int64_t lead_k = 0);

// ---------------------------------------------------------------- differentiation (adjoint.cu)
template <typename T>
void launch_dense_grad(int p, Csr<T> om, const int4* rinfo, const T* rdv, const T* S, int64_t lds, T* G, int64_t ldg,
                       T lam2, T scale, cudaStream_t s);
template <typename T>
void launch_spmm_dense(int p, Csr<T> om, const int4* rinfo, const T* rdv, const T* B, int64_t ldb, int64_t m, T* C,
                       int64_t ldc, cudaStream_t s);
template <typename T>
void launch_spmm_dense_t(int p, Csr<T> om, const int4* rinfo, const T* rdv, const T* B, int64_t ldb, int64_t m,
                         T* Ct, int64_t ldt, T scale, cudaStream_t s);
// launch_transpose puts rows / 32 in gridDim.y (at most 65535)
constexpr int64_t kTransposeMaxRows = 65535ll * 32;
void launch_transpose(const void* in, int in_dt, int64_t rows, int64_t cols, int64_t ldi, void* out, int out_dt,
                      int64_t ldo, double scale, cudaStream_t s);
template <typename T> void launch_transpose_index(int p, Csr<T> om, int* tr, int* row, cudaStream_t s);
template <typename T>
void launch_support_product(int p, Csr<T> om, const int4* rinfo, const double* v, const T* S, int64_t lds,
                            double* out, cudaStream_t s);
template <typename T>
void launch_support_sddmm(int p, Csr<T> om, const T* yt, const T* xt, int64_t ld, int64_t n, double* out,
                          cudaStream_t s);
template <typename T>
void launch_support_product_p(int64_t nnz, const int* row, Csr<T> om, const int4* rinfo, const double* r,
                              const double* p_old, double* p_new, const void* cg, const T* S, int64_t lds,
                              double* out, cudaStream_t s);
template <typename T>
void launch_support_combine(int64_t nnz, const int* row, Csr<T> om, const int* tr, const double* Tv, const double* v,
                            double lam2, int mode, double* out, double* part, double tol2, void* cg, cudaStream_t s);
template <typename T>
void launch_support_vectors(int p, int64_t nnz, Csr<T> om, double* omega_d, double* sign_off, cudaStream_t s);
// scale ((T_e + T_tr(e))/2 + lambda2 w_e - [i=j]/w_ii) per support entry (dL/dOmega on the support)
template <typename T>
void launch_support_grad(int64_t nnz, const int* row, Csr<T> om, const int* tr, const double* Tv, double lam2,
                         double scale, double* out, cudaStream_t s);
int cg_part_blocks(int64_t n);
void launch_dot_part(int64_t n, const double* a, const double* b, double* part, cudaStream_t s);
void launch_cg_scalar(const double* part, int nb, int stage, double tol2, void* cg, cudaStream_t s);
void launch_cg_xr(int64_t n, void* cg, const double* p, const double* Ap, double* x, double* r, double* part,
                  double tol2, cudaStream_t s);
size_t cg_state_bytes();
template <typename T>
int launch_smooth_parts(int p, Csr<T> om, const double* Tv, double* part, double* out3, cudaStream_t s);
void launch_reduce_parts(const double* part, int nb, double* out, cudaStream_t s);

// ---------------------------------------------------------------- dense products (gram*.cu)
// S = X^T X / n into S (p x lds).  Returns a CUDA error code.
cudaError_t gram_simt(const void* X, int xdt, int64_t n, int64_t p, void* S, int sdt, int64_t lds,
                      cudaStream_t s, int* launches);
// band: row blocks per band of the tile order (<= 0: the default, 16).
// before_kernel (nullable) is recorded on s between the transpose and the product kernel.
// m1 (nullable, p x nbm): also write max |S_ij| per (row, 128-column block), j != i,
// rounded up to BF16, from the product's epilogue.
// prepared: the panels in scratch already hold X's preparation (gram_tc_prepare).
// tiles_sig: the caller's record of the tile order already in scratch (null: upload it).
// chunk_k: K elements per accumulation chunk (0: the mode's default); lead_k: K elements
// of each tile's first two chunks (0: 4 chunk_k).  The product writes S_ij for i <= j; a
// pass after it writes the lower triangle (and m1); after_kernel (nullable) is recorded
// between the two.
cudaError_t gram_tc(const void* X, int xdt, int64_t n, int64_t p, float* S, int64_t lds, int precision,
                    void* scratch, size_t scratch_bytes, cudaStream_t s, int* launches, int band = 0,
                    cudaEvent_t before_kernel = nullptr, uint16_t* m1 = nullptr, int nbm = 0, int prepared = 0,
                    uint64_t* tiles_sig = nullptr, int schedule = 1, int64_t chunk_k = 0, int64_t lead_k = 0,
                    cudaEvent_t after_kernel = nullptr);
// Only the panel preparation of gram_tc (transpose / split of X into scratch);
// max_blocks > 0 bounds the BF16 transpose's grid, so that it shares the GPU with a solve.
cudaError_t gram_tc_prepare(const void* X, int xdt, int64_t n, int64_t p, int precision, void* scratch,
                            size_t scratch_bytes, cudaStream_t s, int max_blocks = 0);
// Chunk c of a tile's K loop (in stages): the first two chunks hold lead stages each,
// the rest chunk stages each (the last one ragged).  The long first chunks keep the
// MMAs of the next tile busy while the epilogue stores the previous one.
__host__ __device__ __forceinline__ int chunk_start(int c, int k_tiles, int chunk, int lead) {
    const long long st = c <= 2 ? (long long)c * lead : 2ll * lead + (long long)(c - 2) * chunk;
    return st < k_tiles ? (int)st : k_tiles;
}
__host__ __device__ __forceinline__ int num_chunks(int k_tiles, int chunk, int lead) {
    if (k_tiles <= 2 * lead) return (k_tiles + lead - 1) / lead;
    return 2 + (k_tiles - 2 * lead + chunk - 1) / chunk;
}

size_t gram_tc_scratch_bytes(int xdt, int64_t n, int64_t p, int precision);
// Error word of the tensor-core Gram's bounded waits (0 = none); reading it resets it.
// The error word of the last tensor-core Gram launched on this scratch (0: none; else the
// code of the bounded wait that gave up); synchronises s.
int gram_tc_take_error(const void* scratch, int xdt, int64_t n, int64_t p, int precision, cudaStream_t s);

// Raise a kernel's dynamic shared-memory limit once per device (the attribute call
// is a host round trip that must stay out of the iteration loop).
cudaError_t set_smem_once(const void* func, int bytes, int slot);
enum : int { kSmemSlotScreenF = 0, kSmemSlotScreenD = 1, kSmemSlotObsBf16x3 = 2, kSmemSlotObsTf32 = 3, kSmemSlots = 4 };

// Set the text returned by hpc_last_error() for this thread (api.cu).
void set_last_error(const char* msg);

// Box of the TMA descriptor of S used by the screening pass: 64 rows x BJ columns.
constexpr int kScreenBoxRows = 64;
template <typename T> constexpr int screen_box_cols() { return 32 * (16 / (int)sizeof(T)); }

}  // namespace hpc
