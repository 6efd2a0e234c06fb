// C ABI of the solver: handle life cycle, data loading (the Gram of Alg. 2
// step 2), and the host driver of Alg. 1 that enqueues each outer iteration's
// kernels and reads back a small control block twice per iteration.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "ptx.cuh"

namespace {

thread_local char g_last_error[512] = "";

void set_cuda_error(cudaError_t e, const char* what, int line) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s (api.cu:%d)", what, cudaGetErrorString(e), line);
}

#define CUDA_TRY(expr)                                     \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) {                           \
            set_cuda_error(e_, #expr, __LINE__);           \
            return e_ == cudaErrorMemoryAllocation ? HPC_ERR_OOM : HPC_ERR_CUDA; \
        }                                                  \
    } while (0)

#define STATUS_TRY(expr)             \
    do {                             \
        int st_ = (expr);            \
        if (st_ < 0) return st_;     \
    } while (0)

size_t dtype_size(int dt) { return dt == HPC_F64 ? 8 : dt == HPC_F32 ? 4 : 2; }

template <typename T>
T* as(void* p) { return static_cast<T*>(p); }

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

namespace hpc {
void set_last_error(const char* msg) { std::snprintf(g_last_error, sizeof g_last_error, "%s", msg); }
}  // namespace hpc

struct hpc_ctx {
    int64_t n = 0, p = 0, ld = 0;
    int variant = HPC_COV;
    int vdt = HPC_F32;      // value dtype of S / Omega / G
    int precision = HPC_PREC_AUTO;
    double lam1 = 0, lam2 = 0;
    hpc_options opt{};
    cudaStream_t stream = nullptr;
    bool loaded = false;

    // dense data
    void* S = nullptr;              // p x ld, vdt
    // iterate (double-buffered CSR)
    int* rp[2] = {nullptr, nullptr};
    int* ci[2] = {nullptr, nullptr};
    void* cv[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t csr_cap = 0;
    int64_t nnz = 0;
    // screening output and candidate structure
    int64_t cap = 0;                // emission capacity
    int* em_row = nullptr;
    int* em_col = nullptr;
    void* em_w = nullptr;
    void* em_om = nullptr;
    int* bk_cnt = nullptr; int* bk_off = nullptr; int* bk_cur = nullptr; int* bk_len = nullptr;
    long long* bk_uoff = nullptr;
    int* bk_long = nullptr;
    unsigned* bar = nullptr;      // arrival counters of the cooperative tail kernels' grid barriers
    int2* bk_mir = nullptr;
    int* col_a = nullptr; void* w_a = nullptr; void* om_a = nullptr; unsigned char* fl_a = nullptr;
    int* col_b = nullptr; void* w_b = nullptr; void* om_b = nullptr; unsigned char* fl_b = nullptr;
    void* g_b = nullptr;
    int* cnt2 = nullptr;
    hpc::ScanPart* scan_part = nullptr;
    double* part_obj = nullptr;
    double* part_ls = nullptr;
    int nblk = 0;
    hpc::Ctrl* d_ctrl = nullptr;
    hpc::Ctrl* h_ctrl = nullptr;    // pinned
    // screening pass: TMA descriptor of S, per-row set-up, persistent grid size
    CUtensorMap smap;
    int4* rinfo = nullptr;
    int* offlist = nullptr;
    void* rdv = nullptr;            // ld entries, zero padded
    unsigned* pmask = nullptr;      // ld / 32 words
    long long* seqoff = nullptr;    // folded tile sequence of the screening pass
    int screen_grid = 1;
    // bound screening: max |S_ij| per (row, column block), the column maxima of the
    // pure diagonals, and the kept (row, block) items
    void* m1 = nullptr;
    void* m1g = nullptr;
    int ngl = 0;
    int nbm = 0;
    void* colmax = nullptr;
    int2* pairs_list = nullptr;
    int pairs_cap = 0;
    int2* row_items = nullptr;
    int row_items_cap = 0;
    int num_sms = 0;
    // scratch for the tensor-core Gram
    void* gram_scratch = nullptr;
    size_t gram_scratch_bytes = 0;
    // events
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_scr0 = nullptr, ev_scr1 = nullptr;
    int64_t regrows = 0;
    double ms_gram = 0.0;
    double ms_gram_kernel = 0.0;
    cudaEvent_t ev_gk = nullptr;     // between the transpose and the tensor-core product
    cudaEvent_t ev_ge = nullptr;     // end of the Gram (before the block-maxima pass)
    cudaEvent_t ev_gp = nullptr;     // end of the tensor-core product (before its mirror pass)
    // device staging buffer for X passed from the host (kept between loads)
    void* x_stage = nullptr;
    size_t x_stage_bytes = 0;
    // staging of the next data set (hpc_prefetch_x), all on pf_stream: a copy of X into
    // x_stage (or X itself when it is device memory), then, after the handle's next
    // Gram has read the panels, that X's panel preparation
    cudaStream_t pf_stream = nullptr;
    cudaEvent_t ev_pf = nullptr;          // end of the work queued on pf_stream so far
    cudaEvent_t ev_copy = nullptr;        // end of the last staging copy
    cudaEvent_t ev_prep = nullptr;        // end of the last staged panel preparation
    cudaEvent_t ev_gdone = nullptr;       // a Gram's end on the handle's stream
    uint64_t tiles_sig = 0;               // the tile order in the Gram scratch (gram_tc)
    bool pf_issued = false;               // ev_pf has been recorded at least once
    bool st_valid = false;                // st_dev holds st_ptr's data (copy queued)
    const void* st_ptr = nullptr;
    const void* st_dev = nullptr;
    int st_xdt = -1;
    bool pf_valid = false;                // the Gram panels hold pf_ptr's preparation (queued)
    const void* pf_ptr = nullptr;
    int pf_xdt = -1;
    // launch shapes (hpc_set_tuning / hpc_autotune); ls_window starts from the options
    hpc_tuning tune{16, 8, 0, 2, 1, 1, 1, 0, 0, 0};
    // device loop: one CUDA graph (outer iteration WHILE node, inner line-search
    // WHILE node) captured on a private stream; rebuilt when a buffer it captured
    // is reallocated (epoch), when the current CSR buffer changes, or with timing
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t epoch = 0;
    int64_t g_epoch = -1;
    int g_cur = -1, g_timing = -1;
    int g_fused = 0;              // tail form of the device-loop graph (tuning fused_tail)
    // differentiation scratch (grown on demand)
    void* adj_buf = nullptr;
    size_t adj_bytes = 0;
    // Obs variant (Alg. 3): X^T and Y^T in FP32 (p x ldx), their MMA panels, tile pairs
    float* xt = nullptr;
    float* yt = nullptr;
    int64_t ldx = 0;
    void* xp[2] = {nullptr, nullptr};
    void* yp[2] = {nullptr, nullptr};
    int2* pairs = nullptr;
    int64_t npairs = 0;
    CUtensorMap obs_maps[4];
    // device buffers the handle holds (address -> bytes), for hpc_get_info
    std::unordered_map<void*, size_t> held;
    size_t held_bytes = 0;
};

namespace {

// cudaMalloc of a buffer the handle keeps, recorded in its ledger.
template <typename T>
cudaError_t hold(hpc_ctx* h, T** q, size_t bytes) {
    void* v = nullptr;
    const cudaError_t e = cudaMalloc(&v, bytes);
    if (e == cudaSuccess) {
        *q = static_cast<T*>(v);
        h->held[v] = bytes;
        h->held_bytes += bytes;
    }
    return e;
}

void release(hpc_ctx* h, void* q) {
    if (!q) return;
    auto it = h->held.find(q);
    if (it != h->held.end()) {
        h->held_bytes -= it->second;
        h->held.erase(it);
    }
    cudaFree(q);
}

void free_candidates(hpc_ctx* h) {
    void* ptrs[] = {h->em_row, h->em_col, h->em_w, h->em_om, h->col_a, h->w_a, h->om_a, h->fl_a,
                    h->col_b, h->w_b, h->om_b, h->fl_b, h->g_b, h->bk_mir};
    for (void* q : ptrs) release(h, q);
    h->em_row = h->em_col = nullptr; h->em_w = h->em_om = nullptr;
    h->col_a = h->col_b = nullptr; h->w_a = h->om_a = h->w_b = h->om_b = h->g_b = nullptr;
    h->fl_a = h->fl_b = nullptr;
    h->bk_mir = nullptr;
}

int alloc_candidates(hpc_ctx* h, int64_t cap) {
    const size_t vs = dtype_size(h->vdt);
    const int64_t bcap = 2 * cap;
    free_candidates(h);
    CUDA_TRY(hold(h, &h->em_row, cap * sizeof(int)));
    CUDA_TRY(hold(h, &h->em_col, cap * sizeof(int)));
    CUDA_TRY(hold(h, &h->em_w, cap * vs));
    CUDA_TRY(hold(h, &h->em_om, cap * vs));
    CUDA_TRY(hold(h, &h->col_a, bcap * sizeof(int)));
    CUDA_TRY(hold(h, &h->w_a, bcap * vs));
    CUDA_TRY(hold(h, &h->om_a, bcap * vs));
    CUDA_TRY(hold(h, &h->fl_a, bcap));
    CUDA_TRY(hold(h, &h->col_b, bcap * sizeof(int)));
    CUDA_TRY(hold(h, &h->w_b, bcap * vs));
    CUDA_TRY(hold(h, &h->om_b, bcap * vs));
    CUDA_TRY(hold(h, &h->fl_b, bcap));
    CUDA_TRY(hold(h, &h->g_b, bcap * vs));
    CUDA_TRY(hold(h, &h->bk_mir, bcap * sizeof(int2)));
    h->cap = cap;
    h->epoch += 1;
    return HPC_OK;
}

// (Re)allocate the double-buffered CSR with capacity newcap, keeping the current iterate.
int grow_csr(hpc_ctx* h, int64_t newcap) {
    const size_t vs = dtype_size(h->vdt);
    for (int b = 0; b < 2; ++b) {
        int* ci = nullptr;
        void* cv = nullptr;
        CUDA_TRY(hold(h, &ci, newcap * sizeof(int)));
        CUDA_TRY(hold(h, &cv, newcap * vs));
        if (b == h->cur && h->ci[b] && h->nnz > 0) {
            CUDA_TRY(cudaMemcpyAsync(ci, h->ci[b], h->nnz * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
            CUDA_TRY(cudaMemcpyAsync(cv, h->cv[b], h->nnz * vs, cudaMemcpyDeviceToDevice, h->stream));
            CUDA_TRY(cudaStreamSynchronize(h->stream));
        }
        if (h->ci[b]) release(h, h->ci[b]);
        if (h->cv[b]) release(h, h->cv[b]);
        h->ci[b] = ci;
        h->cv[b] = cv;
    }
    h->csr_cap = newcap;
    h->epoch += 1;
    return HPC_OK;
}

int set_identity(hpc_ctx* h) {
    if (h->vdt == HPC_F64)
        hpc::launch_set_identity<double>({h->rp[h->cur], h->ci[h->cur], as<double>(h->cv[h->cur])}, (int)h->p, h->stream);
    else
        hpc::launch_set_identity<float>({h->rp[h->cur], h->ci[h->cur], as<float>(h->cv[h->cur])}, (int)h->p, h->stream);
    CUDA_TRY(cudaGetLastError());
    h->nnz = h->p;
    return HPC_OK;
}

template <typename T>
hpc::IterBufs<T> bufs(hpc_ctx* h) {
    hpc::IterBufs<T> b{};
    b.S = static_cast<const T*>(h->S);
    b.ld = h->ld;
    b.p = (int)h->p;
    b.cur = {h->rp[h->cur], h->ci[h->cur], as<T>(h->cv[h->cur])};
    b.next = {h->rp[1 - h->cur], h->ci[1 - h->cur], as<T>(h->cv[1 - h->cur])};
    b.csr_cap = (int)std::min<int64_t>(h->csr_cap, 0x7fffffff);
    b.em = {h->em_row, h->em_col, as<T>(h->em_w), as<T>(h->em_om), (int)h->cap};
    b.bk.cnt = h->bk_cnt; b.bk.off = h->bk_off; b.bk.cur = h->bk_cur; b.bk.len = h->bk_len;
    b.bk.col_a = h->col_a; b.bk.w_a = as<T>(h->w_a); b.bk.om_a = as<T>(h->om_a); b.bk.fl_a = h->fl_a;
    b.bk.col_b = h->col_b; b.bk.w_b = as<T>(h->w_b); b.bk.om_b = as<T>(h->om_b); b.bk.fl_b = h->fl_b;
    b.bk.g = as<T>(h->g_b);
    b.bk.uoff = h->bk_uoff;
    b.bk.longlist = h->bk_long;
    b.bk.mir = h->bk_mir;
    b.bk.cap = (int)std::min<int64_t>(2 * h->cap, 0x7fffffff);
    b.cnt2 = h->cnt2;
    b.scan_part = h->scan_part;
    b.bar = h->bar;
    b.part_obj = h->part_obj;
    b.part_ls = h->part_ls;
    b.nblk = h->nblk;
    b.ctrl = h->d_ctrl;
    b.lam1 = (T)h->lam1;
    b.lam2 = (T)h->lam2;
    b.eps = h->opt.eps;
    b.max_halvings = h->opt.max_halvings;
    b.ls_window = h->tune.ls_window;
    b.ls_blocks_per_sm = h->tune.ls_blocks_per_sm;
    b.rows_ctas_per_sm = h->tune.rows_ctas_per_sm;
    b.smap = &h->smap;
    b.rinfo = h->rinfo;
    b.offlist = h->offlist;
    b.rdv = as<T>(h->rdv);
    b.pmask = h->pmask;
    b.seqoff = h->seqoff;
    b.screen_grid = h->screen_grid;
    const bool bounds = h->tune.screen_bounds != 0;
    b.m1 = bounds ? static_cast<const unsigned short*>(h->m1) : nullptr;
    b.m1g = bounds ? static_cast<const unsigned short*>(h->m1g) : nullptr;
    b.ngl = h->ngl;
    b.nbm = h->nbm;
    b.colmax = h->colmax;
    b.pairs = h->pairs_list;
    b.pairs_cap = h->pairs_cap;
    b.row_items = h->row_items;
    b.row_items_cap = h->row_items_cap;
    b.num_sms = h->num_sms;
    b.xt = h->xt;
    b.ldx = h->ldx;
    b.n = h->n;
    return b;
}

int read_ctrl(hpc_ctx* h) {
    CUDA_TRY(cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(hpc::Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return HPC_OK;
}

int flags_to_status(int flags) {
    if (flags & hpc::kFlagNaN) return HPC_ERR_NAN;
    if (flags & hpc::kFlagLsFail) return HPC_ERR_LS_FAIL;
    if (flags & hpc::kFlagTimeout) return HPC_ERR_DEVICE_TIMEOUT;
    if (flags & hpc::kFlagBadStructure) return HPC_ERR_CUDA;
    return HPC_OK;
}

// Grow the candidate (and iterate) capacity after an overflow.  Returns HPC_OK or
// HPC_ERR_CAPACITY when max_capacity is reached.
int regrow(hpc_ctx* h, int64_t need) {
    const int64_t limit = h->opt.max_capacity > 0 ? h->opt.max_capacity : h->p * h->p;
    int64_t nc = std::max<int64_t>(2 * h->cap, need);
    nc = std::min<int64_t>(nc, std::min<int64_t>(limit, 0x3fffffff));
    if (nc <= h->cap) {
        std::snprintf(g_last_error, sizeof g_last_error, "candidate capacity %lld exhausted",
                      (long long)h->cap);
        return HPC_ERR_CAPACITY;
    }
    STATUS_TRY(alloc_candidates(h, nc));
    if (2 * nc > h->csr_cap) STATUS_TRY(grow_csr(h, 2 * nc));
    h->regrows += 1;
    return HPC_OK;
}

// Obs (Alg. 3 steps 2, 4-6): Y^T = Omega X^T, its MMA panels, and the paired-tile
// Z GEMM with the screening emission.
int obs_screen(hpc_ctx* h, const hpc::IterBufs<float>& b, cudaStream_t s) {
    const int p = (int)h->p;
    hpc::launch_row_info<float>(p, b.cur, h->rinfo, as<float>(h->rdv), s);
    hpc::launch_spmm_dense<float>(p, b.cur, h->rinfo, as<float>(h->rdv), h->xt, h->ldx, h->ldx, h->yt, h->ldx, s);
    hpc::launch_obs_split(h->precision, h->yt, p, h->ldx, h->ldx, h->yp[0], h->yp[1], h->n, h->p, s);
    cudaError_t e = hpc::launch_obs_pairs(h->precision, h->obs_maps, h->pairs, h->npairs, h->n, p, b.cur.rp, b.cur.ci,
                                          b.cur.cv, b.em, h->d_ctrl, s, h->tune.gram_chunk, h->tune.gram_lead);
    if (e != cudaSuccess) { set_cuda_error(e, "obs pair GEMM", __LINE__); return HPC_ERR_CUDA; }
    return HPC_OK;
}

int tail_mode(const hpc_ctx* h);

// One outer iteration.  *done is set when the stopping rule holds.
template <typename T>
int one_iteration(hpc_ctx* h, hpc_stats* st, bool use_stop, bool* done) {
    for (int attempt = 0; attempt < 64; ++attempt) {
        hpc::IterBufs<T> b = bufs<T>(h);
        const hpc::LoopCond host_loop{};
        hpc::launch_iter_begin<T>(b, host_loop, h->stream);
        if (h->opt.timing) CUDA_TRY(cudaEventRecord(h->ev_scr0, h->stream));
        if constexpr (std::is_same<T, float>::value) {
            if (h->variant == HPC_OBS) STATUS_TRY(obs_screen(h, b, h->stream));
            else hpc::launch_grad_screen<T>(b, h->stream);
        } else {
            hpc::launch_grad_screen<T>(b, h->stream);
        }
        if (h->opt.timing) CUDA_TRY(cudaEventRecord(h->ev_scr1, h->stream));
        const bool fused = tail_mode(h) == 1;
        int launches = hpc::kLaunchesBegin + hpc::kLaunchesScreen;
        bool accepted = false, overflow = false;
        if (fused) {
            // candidates, gradient, every window and the accept in one launch
            const cudaError_t e = hpc::launch_tail<T>(b, h->variant == HPC_OBS, h->stream);
            if (e != cudaSuccess) {
                set_cuda_error(e, "fused iteration tail", __LINE__);
                return HPC_ERR_CUDA;
            }
            launches += hpc::kLaunchesTail;
            STATUS_TRY(read_ctrl(h));
            const hpc::Ctrl& c = *h->h_ctrl;
            if (c.flags & (hpc::kFlagEmOverflow | hpc::kFlagBucketOverflow)) overflow = true;
            else if (c.ls_accept >= 0 && (c.flags & ~hpc::kFlagNnzOverflow) == 0) accepted = true;
        } else {
            hpc::launch_candidates<T>(b, h->stream);
            CUDA_TRY(cudaGetLastError());
            launches += hpc::kLaunchesCandidates;
        }
        for (int hb = 0; !fused && hb <= h->opt.max_halvings; hb += h->tune.ls_window) {
            if constexpr (std::is_same<T, float>::value) {
                if (h->variant == HPC_OBS) hpc::launch_ls_window_obs(b, host_loop, h->stream);
                else hpc::launch_ls_window<T>(b, host_loop, h->stream);
            } else {
                hpc::launch_ls_window<T>(b, host_loop, h->stream);
            }
            CUDA_TRY(cudaGetLastError());
            launches += hpc::kLaunchesLsWindow;
            STATUS_TRY(read_ctrl(h));
            const hpc::Ctrl& c = *h->h_ctrl;
            if (c.flags & (hpc::kFlagEmOverflow | hpc::kFlagBucketOverflow)) { overflow = true; break; }
            if (c.flags) break;
            if (c.ls_accept >= 0) { accepted = true; break; }
        }
        if (h->opt.timing && st) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, h->ev_scr0, h->ev_scr1));
            st->ms_grad_pass += ms;
            st->grad_pass_launches += 1;
        }
        if (st) st->kernel_launches += launches;
        const hpc::Ctrl c = *h->h_ctrl;
        if (st) {
            st->f = c.f_cur;
            st->F = c.f_cur + c.pen_cur;
            st->candidates = c.em_count;
        }
        if (overflow) {
            const int64_t need = (int64_t)c.em_count + 1;
            STATUS_TRY(regrow(h, need));
            continue;
        }
        if (!accepted) {
            const int s = flags_to_status(c.flags);
            return s != HPC_OK ? s : HPC_ERR_LS_FAIL;
        }
        if (!fused) {
            hpc::launch_accept<T>(b, h->stream);
            CUDA_TRY(cudaGetLastError());
            if (st) st->kernel_launches += hpc::kLaunchesAccept;
            STATUS_TRY(read_ctrl(h));
        }
        const hpc::Ctrl& c2 = *h->h_ctrl;
        if (c2.flags & hpc::kFlagNnzOverflow) {
            STATUS_TRY(grow_csr(h, std::max<int64_t>(2 * h->csr_cap, (int64_t)c2.nnz_next + 1)));
            h->regrows += 1;
            continue;
        }
        if (c2.flags) return flags_to_status(c2.flags);
        h->cur = 1 - h->cur;
        h->nnz = c2.nnz_next;
        if (st) {
            st->iterations += 1;
            st->rel_change = c2.rel;
            st->accepted_halvings = c2.ls_accept;
            st->nnz = h->nnz;
        }
        *done = use_stop && c2.converged;
        return HPC_OK;
    }
    return HPC_ERR_CAPACITY;
}

// Reset the counters of the control block and load the solve's parameters
// (lambda, iteration limit, stopping rule) into it.
int load_ctrl(hpc_ctx* h, int64_t k, bool use_stop) {
    hpc::Ctrl& c = *h->h_ctrl;
    c.iter = 0;
    c.ls_trials = 0;
    c.ls_windows = 0;
    c.iter_attempts = 0;
    c.screen_ns = 0;
    c.t_stamp = 0;
    c.flags = 0;
    c.converged = 0;
    c.lam1 = h->lam1;
    c.lam2 = h->lam2;
    c.nnz_cur = (int)h->nnz;
    c.iter_limit = (int)std::min<int64_t>(k, 0x7fffffff);
    c.use_stop = use_stop ? 1 : 0;
    CUDA_TRY(cudaMemcpyAsync(h->d_ctrl, h->h_ctrl, sizeof(hpc::Ctrl), cudaMemcpyHostToDevice, h->stream));
    return HPC_OK;
}

void destroy_graph(hpc_ctx* h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->g_epoch = -1;
}

// The last node captured on stream cs (captures here are linear chains).
int capture_leaf(cudaStream_t cs, cudaGraphNode_t* leaf) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &nd));
    if (st != cudaStreamCaptureStatusActive || nd != 1) {
        std::snprintf(g_last_error, sizeof g_last_error, "device loop capture: unexpected capture state");
        return HPC_ERR_CUDA;
    }
    *leaf = deps[0];
    return HPC_OK;
}

// End a capture into an existing graph, keeping the first error.
int end_capture(cudaStream_t cs, cudaGraph_t g, int status) {
    cudaGraph_t out = g;
    const cudaError_t e = cudaStreamEndCapture(cs, &out);
    if (status != HPC_OK) return status;
    CUDA_TRY(e);
    CUDA_TRY(cudaGetLastError());
    return HPC_OK;
}

// A WHILE node of graph g on condition handle hnd (created for g), after dep if any.
int add_while(cudaGraph_t g, const cudaGraphNode_t* dep, cudaGraphConditionalHandle hnd, cudaGraphNode_t* node,
              cudaGraph_t* body) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    CUDA_TRY(cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &np));
    *body = np.conditional.phGraph_out[0];
    return HPC_OK;
}

// Whether a cooperative kernel runs inside a conditional WHILE node's body on the
// current device: checked once per device, before any capture, by a graph whose
// loop body is one cooperative launch of a one-block kernel that ends the loop.
// The kernel counts its runs in word 1 of the handle's barrier buffer (word 0 is
// the fused tail's arrival counter), so the check allocates no device memory.
bool tail_in_graph_supported(const hpc_ctx* h) {
    static std::mutex mu;
    static int state[64] = {};     // 0 unknown, 1 supported, 2 not
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (state[dev]) return state[dev] == 1;
    bool ok = false;
    int* d = h && h->bar ? reinterpret_cast<int*>(h->bar + 1) : nullptr;
    cudaStream_t s = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int coop = 0;
    if (d && cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
        cudaMemsetAsync(d, 0, sizeof(int), s) == cudaSuccess && cudaGraphCreate(&g, 0) == cudaSuccess) {
        cudaGraphConditionalHandle hnd;
        cudaGraphNode_t node;
        cudaGraph_t body;
        if (cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault) == cudaSuccess &&
            add_while(g, nullptr, hnd, &node, &body) == HPC_OK &&
            cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
            const cudaError_t le = hpc::launch_tail_probe(d, hnd, s);
            cudaGraph_t out = body;
            const cudaError_t ce = cudaStreamEndCapture(s, &out);
            int ran = 0;
            if (le == cudaSuccess && ce == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess &&
                cudaGraphLaunch(ge, s) == cudaSuccess &&
                cudaMemcpyAsync(&ran, d, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                cudaStreamSynchronize(s) == cudaSuccess)
                ok = ran == 1;
        }
    }
    (void)cudaGetLastError();   // a refused capture leaves its error here
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (s) cudaStreamDestroy(s);
    if (!d) return false;       // no handle buffer to check with: decide at the next call
    state[dev] = ok ? 1 : 2;
    return ok;
}

// Form of the iteration tail: the tuning's fused_tail (0 the chain of kernels, 1
// the one cooperative kernel) where the device runs cooperative kernels in graph
// loops, else the chain (the host-driven loop needs only the cooperative launch
// itself, which the same check covers).
int tail_mode(const hpc_ctx* h) { return h->tune.fused_tail != 0 && tail_in_graph_supported(h) ? h->tune.fused_tail : 0; }

template <typename T>
int capture_screen(hpc_ctx* h, const hpc::IterBufs<T>& b, cudaStream_t cs) {
    if constexpr (std::is_same<T, float>::value) {
        if (h->variant == HPC_OBS) return obs_screen(h, b, cs);
    }
    hpc::launch_grad_screen<T>(b, cs);
    return HPC_OK;
}

template <typename T>
void capture_window(hpc_ctx* h, const hpc::IterBufs<T>& b, const hpc::LoopCond& lc, cudaStream_t cs) {
    if constexpr (std::is_same<T, float>::value) {
        if (h->variant == HPC_OBS) { hpc::launch_ls_window_obs(b, lc, cs); return; }
    }
    hpc::launch_ls_window<T>(b, lc, cs);
}

// Capture the iteration loop as a WHILE node of graph g (after dep, if any) on
// the handle lc.iter, which the caller created for g:
//   WHILE (iteration condition) {
//       begin, [stamp], screening pass, [stamp], candidates, gradient
//       WHILE (line-search condition) { window evaluation, decision }
//       compaction, stopping rule, commit of the accepted iterate
//   }
// k_iter_begin arms the line-search loop, the last block of k_ls_eval ends it, and the commit
// kernel continues or ends the iteration loop.
//
// With the fused tail (mode 1) the body is
//       begin, [stamp], screening pass, [stamp], k_iter_tail, commit
// with no inner loop: the tail runs the windows itself.
template <typename T>
int capture_iteration_loop(hpc_ctx* h, cudaGraph_t g, const cudaGraphNode_t* dep, hpc::LoopCond& lc,
                           cudaGraphNode_t* node, int mode) {
    cudaStream_t cs = h->cap_stream;
    const hpc::IterBufs<T> b = bufs<T>(h);
    const bool fused = mode == 1;
    const bool timing = h->opt.timing != 0;
    lc.use = 1;
    cudaGraphNode_t inner, leaf;
    cudaGraph_t body, ls_body;
    STATUS_TRY(add_while(g, dep, lc.iter, node, &body));
    if (fused) {
        CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        int st = HPC_OK;
        hpc::launch_iter_begin<T>(b, hpc::LoopCond{}, cs);
        if (timing) hpc::launch_stamp(h->d_ctrl, 0, cs);
        st = capture_screen<T>(h, b, cs);
        if (st == HPC_OK) {
            if (timing) hpc::launch_stamp(h->d_ctrl, 1, cs);
            const cudaError_t e = hpc::launch_tail<T>(b, h->variant == HPC_OBS, cs);
            if (e != cudaSuccess) {
                set_cuda_error(e, "fused iteration tail", __LINE__);
                st = HPC_ERR_CUDA;
            }
        }
        if (st == HPC_OK) hpc::launch_commit<T>(b, lc, cs);
        return end_capture(cs, body, st);
    }
    // the line-search handle lives in the body that holds its node
    CUDA_TRY(cudaGraphConditionalHandleCreate(&lc.ls, body, 1, cudaGraphCondAssignDefault));
    {
        CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        int st = HPC_OK;
        hpc::launch_iter_begin<T>(b, lc, cs);
        if (timing) hpc::launch_stamp(h->d_ctrl, 0, cs);
        st = capture_screen<T>(h, b, cs);
        if (st == HPC_OK) {
            if (timing) hpc::launch_stamp(h->d_ctrl, 1, cs);
            hpc::launch_candidates<T>(b, cs);
            st = capture_leaf(cs, &leaf);
        }
        STATUS_TRY(end_capture(cs, body, st));
    }
    STATUS_TRY(add_while(body, &leaf, lc.ls, &inner, &ls_body));
    {
        CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, ls_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        capture_window<T>(h, b, lc, cs);
        STATUS_TRY(end_capture(cs, ls_body, HPC_OK));
    }
    {
        CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, &inner, nullptr, 1, cudaStreamCaptureModeRelaxed));
        hpc::launch_accept<T>(b, cs);
        hpc::launch_commit<T>(b, lc, cs);
        STATUS_TRY(end_capture(cs, body, HPC_OK));
    }
    return HPC_OK;
}

int ensure_cap_stream(hpc_ctx* h) {
    if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    return HPC_OK;
}

// The solve graph: the iteration loop alone (its condition is 1 at every launch).
template <typename T>
int build_graph(hpc_ctx* h) {
    destroy_graph(h);
    STATUS_TRY(ensure_cap_stream(h));
    CUDA_TRY(cudaGraphCreate(&h->graph, 0));
    hpc::LoopCond lc;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&lc.iter, h->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t loop;
    const int mode = tail_mode(h);
    STATUS_TRY(capture_iteration_loop<T>(h, h->graph, nullptr, lc, &loop, mode));
    CUDA_TRY(cudaGraphInstantiate(&h->gexec, h->graph, 0));
    h->g_fused = mode;
    h->g_epoch = h->epoch;
    h->g_cur = h->cur;
    h->g_timing = h->opt.timing ? 1 : 0;
    return HPC_OK;
}

// The path graph: WHILE (points) { k_point_begin, iteration loop, k_point_end }.
template <typename T>
int build_path_graph(hpc_ctx* h, const hpc::PathOut& out, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    STATUS_TRY(ensure_cap_stream(h));
    cudaStream_t cs = h->cap_stream;
    const int mode = tail_mode(h);
    CUDA_TRY(cudaGraphCreate(graph, 0));
    cudaGraphConditionalHandle path_cond;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&path_cond, *graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t outer, begin_leaf, loop;
    cudaGraph_t body;
    STATUS_TRY(add_while(*graph, nullptr, path_cond, &outer, &body));
    hpc::LoopCond lc;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&lc.iter, body, 1, cudaGraphCondAssignDefault));
    {
        CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        hpc::launch_point_begin(h->d_ctrl, out, lc, cs);
        const int st = capture_leaf(cs, &begin_leaf);
        STATUS_TRY(end_capture(cs, body, st));
    }
    STATUS_TRY(capture_iteration_loop<T>(h, body, &begin_leaf, lc, &loop, mode));
    {
        const hpc::IterBufs<T> b = bufs<T>(h);
        CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, &loop, nullptr, 1, cudaStreamCaptureModeRelaxed));
        hpc::launch_point_end<T>(b, out, path_cond, cs);
        STATUS_TRY(end_capture(cs, body, HPC_OK));
    }
    CUDA_TRY(cudaGraphInstantiate(exec, *graph, 0));
    return HPC_OK;
}

// Launches of one outer iteration of the device loop besides its line-search
// windows (two each).
int loop_launches(const hpc_ctx* h, int mode) {
    if (mode == 1) return hpc::kLaunchesBegin + hpc::kLaunchesScreen + hpc::kLaunchesTail + 1 + (h->opt.timing ? 2 : 0);
    return hpc::kLaunchesBegin + hpc::kLaunchesScreen + hpc::kLaunchesCandidates + hpc::kLaunchesAccept + 1 +
           (h->opt.timing ? 2 : 0);
}

// Window launches of the device loop (none with the fused tail: it runs them).
int64_t window_launches(int mode, long long windows) {
    return mode == 1 ? 0 : (int64_t)hpc::kLaunchesLsWindow * windows;
}

// The device loop: one graph launch runs iterations until the stopping rule, the
// iteration limit or a raised flag; the host only grows buffers after an
// overflow (the failed iteration is repeated) and reads the control block.
template <typename T>
int run_device_loop(hpc_ctx* h, int64_t k, bool use_stop, hpc_stats* s, bool fresh = true) {
    const int64_t regrows0 = h->regrows;
    if (fresh) STATUS_TRY(load_ctrl(h, k, use_stop));
    if (h->opt.timing) CUDA_TRY(cudaEventRecord(h->ev[0], h->stream));
    int status = HPC_OK;
    bool ran = false;
    for (int attempt = 0; attempt < 64 && k > 0; ++attempt) {
        if (!h->gexec || h->g_epoch != h->epoch || h->g_cur != h->cur || h->g_timing != (h->opt.timing ? 1 : 0))
            STATUS_TRY(build_graph<T>(h));
        CUDA_TRY(cudaGraphLaunch(h->gexec, h->stream));
        STATUS_TRY(read_ctrl(h));
        const hpc::Ctrl& c = *h->h_ctrl;
        h->nnz = c.nnz_cur;
        ran = true;
        if (c.flags & (hpc::kFlagEmOverflow | hpc::kFlagBucketOverflow)) {
            STATUS_TRY(regrow(h, (int64_t)c.em_count + 1));
            ran = false;
            continue;
        }
        if (c.flags & hpc::kFlagNnzOverflow) {
            STATUS_TRY(grow_csr(h, std::max<int64_t>(2 * h->csr_cap, (int64_t)c.nnz_next + 1)));
            h->regrows += 1;
            ran = false;
            continue;
        }
        break;
    }
    if (k > 0 && !ran) return HPC_ERR_CAPACITY;
    const hpc::Ctrl& c = *h->h_ctrl;
    if (c.flags) {
        status = flags_to_status(c.flags);
        if (status == HPC_OK) status = HPC_ERR_CUDA;
    } else if (use_stop) {
        status = c.converged ? HPC_OK : HPC_NOT_CONVERGED;
    }
    if (h->opt.timing) {
        CUDA_TRY(cudaEventRecord(h->ev[1], h->stream));
        CUDA_TRY(cudaEventSynchronize(h->ev[1]));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
        s->ms_total = ms;
        s->ms_grad_pass = (double)c.screen_ns * 1e-6;
    }
    s->iterations = c.iter;
    s->ls_trials = c.ls_trials;
    s->nnz = h->nnz;
    s->accepted_halvings = c.ls_accept;
    s->f = c.f_cur;
    s->F = c.f_cur + c.pen_cur;
    s->rel_change = c.rel;
    s->candidates = c.em_count;
    s->grad_pass_launches = c.iter_attempts;
    s->kernel_launches = c.iter_attempts * loop_launches(h, h->g_fused) + window_launches(h->g_fused, c.ls_windows);
    s->ms_gram = h->ms_gram;
    s->ms_gram_kernel = h->ms_gram_kernel;
    s->capacity_regrows = h->regrows - regrows0;
    s->status = status;
    return status;
}

// Independent handles (device loop, same device) solved by one graph launch:
// each handle's iteration loop is a WHILE branch of the same graph, with no
// edges between branches.  The graph runs on the first handle's stream after it
// waits for the others.  A handle whose buffers overflowed grows them and
// finishes alone with its own graph, its counters continuing.
int solve_batch_device(const std::vector<hpc_ctx*>& hs, std::vector<int>& status, std::vector<hpc_stats>& st) {
    const size_t m = hs.size();
    cudaStream_t s0 = hs[0]->stream;
    std::vector<int64_t> regrows0(m);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    auto cleanup = [&]() {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
    };
    int r = HPC_OK;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return HPC_ERR_CUDA;
    for (size_t t = 0; t < m && r == HPC_OK; ++t) {
        hpc_ctx* h = hs[t];
        regrows0[t] = h->regrows;
        r = load_ctrl(h, h->opt.max_iter, true);
        if (r == HPC_OK) r = ensure_cap_stream(h);
        if (r != HPC_OK) break;
        if (h->opt.max_iter <= 0) continue;          // nothing to run: reported as not converged
        hpc::LoopCond lc;
        if (cudaGraphConditionalHandleCreate(&lc.iter, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            r = HPC_ERR_CUDA;
            break;
        }
        cudaGraphNode_t node;
        // the problems' loops run concurrently: the chain of separate kernels, whose
        // blocks never wait on one another
        r = h->vdt == HPC_F64 ? capture_iteration_loop<double>(h, g, nullptr, lc, &node, 0)
                              : capture_iteration_loop<float>(h, g, nullptr, lc, &node, 0);
    }
    if (r == HPC_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) r = HPC_ERR_CUDA;
    // order the launch after every handle's pending work (its control-block upload)
    for (size_t t = 1; t < m && r == HPC_OK; ++t) {
        if (hs[t]->stream == s0) continue;
        if (cudaEventRecord(hs[t]->ev[2], hs[t]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(s0, hs[t]->ev[2], 0) != cudaSuccess)
            r = HPC_ERR_CUDA;
    }
    float batch_ms = 0.f;
    if (r == HPC_OK) {
        cudaEventRecord(hs[0]->ev[0], s0);
        if (cudaGraphLaunch(ge, s0) != cudaSuccess) r = HPC_ERR_CUDA;
        cudaEventRecord(hs[0]->ev[1], s0);
        if (r == HPC_OK && cudaEventSynchronize(hs[0]->ev[1]) != cudaSuccess) r = HPC_ERR_CUDA;
        if (r == HPC_OK) cudaEventElapsedTime(&batch_ms, hs[0]->ev[0], hs[0]->ev[1]);
    }
    cleanup();
    if (r != HPC_OK) return r;
    for (size_t t = 0; t < m; ++t) {
        hpc_ctx* h = hs[t];
        hpc_stats& s = st[t];
        std::memset(&s, 0, sizeof s);
        int rr = read_ctrl(h);
        if (rr != HPC_OK) { status[t] = rr; continue; }
        const hpc::Ctrl c = *h->h_ctrl;
        h->nnz = c.nnz_cur;
        if (c.flags & (hpc::kFlagEmOverflow | hpc::kFlagBucketOverflow | hpc::kFlagNnzOverflow)) {
            if (c.flags & hpc::kFlagNnzOverflow) {
                rr = grow_csr(h, std::max<int64_t>(2 * h->csr_cap, (int64_t)c.nnz_next + 1));
                h->regrows += 1;
            } else {
                rr = regrow(h, (int64_t)c.em_count + 1);
            }
            if (rr == HPC_OK)
                rr = h->vdt == HPC_F64 ? run_device_loop<double>(h, h->opt.max_iter, true, &s, false)
                                       : run_device_loop<float>(h, h->opt.max_iter, true, &s, false);
            s.ms_total += batch_ms;
            s.capacity_regrows = h->regrows - regrows0[t];
            status[t] = rr;
            continue;
        }
        int stt = HPC_OK;
        if (c.flags) {
            stt = flags_to_status(c.flags);
            if (stt == HPC_OK) stt = HPC_ERR_CUDA;
        } else {
            stt = c.converged ? HPC_OK : HPC_NOT_CONVERGED;
        }
        s.iterations = c.iter;
        s.ls_trials = c.ls_trials;
        s.nnz = h->nnz;
        s.accepted_halvings = c.ls_accept;
        s.f = c.f_cur;
        s.F = c.f_cur + c.pen_cur;
        s.rel_change = c.rel;
        s.candidates = c.em_count;
        s.ms_total = batch_ms;
        s.ms_grad_pass = h->opt.timing ? (double)c.screen_ns * 1e-6 : 0.0;
        s.grad_pass_launches = c.iter_attempts;
        s.kernel_launches = c.iter_attempts * loop_launches(h, 0) + window_launches(0, c.ls_windows);
        s.ms_gram = h->ms_gram;
        s.ms_gram_kernel = h->ms_gram_kernel;
        s.capacity_regrows = h->regrows - regrows0[t];
        s.status = stt;
        status[t] = stt;
    }
    return HPC_OK;
}

template <typename T>
int run_iterations(hpc_ctx* h, int64_t k, bool use_stop, hpc_stats* st) {
    hpc_stats local{};
    hpc_stats* s = st ? st : &local;
    std::memset(s, 0, sizeof *s);
    if (h->opt.device_loop) return run_device_loop<T>(h, k, use_stop, s);
    const int64_t regrows0 = h->regrows;
    STATUS_TRY(load_ctrl(h, k, use_stop));
    if (h->opt.timing) CUDA_TRY(cudaEventRecord(h->ev[0], h->stream));
    int status = use_stop ? HPC_NOT_CONVERGED : HPC_OK;
    for (int64_t it = 0; it < k; ++it) {
        bool done = false;
        const int r = one_iteration<T>(h, s, use_stop, &done);
        if (r != HPC_OK) { status = r; break; }
        if (done) { status = HPC_OK; break; }
    }
    if (h->opt.timing) {
        CUDA_TRY(cudaEventRecord(h->ev[1], h->stream));
        CUDA_TRY(cudaEventSynchronize(h->ev[1]));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
        s->ms_total = ms;
    }
    STATUS_TRY(read_ctrl(h));
    s->ls_trials = h->h_ctrl->ls_trials;
    s->nnz = h->nnz;
    s->ms_gram = h->ms_gram;
    s->ms_gram_kernel = h->ms_gram_kernel;
    s->capacity_regrows = h->regrows - regrows0;
    s->status = status;
    return status;
}

int load_x_obs(hpc_ctx* h, const void* Xd) {
    // X^T (p x ldx, FP32, zero padded) and its MMA panels
    CUDA_TRY(cudaMemsetAsync(h->xt, 0, (size_t)h->p * h->ldx * sizeof(float), h->stream));
    return HPC_OK;
}

// Order the handle's stream after everything queued for staging (which writes the
// Gram panels and the staging buffer) and forget it; every other user of those
// buffers calls this first.
int drop_prefetch(hpc_ctx* h) {
    if (h->pf_issued) CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_pf, 0));
    h->pf_valid = false;
    h->st_valid = false;
    return HPC_OK;
}

int load_x(hpc_ctx* h, const void* X, int xdt, int on_host) {
    const void* Xd = X;
    const size_t xbytes = (size_t)h->n * h->p * dtype_size(xdt);
    const bool tc_cov = h->variant == HPC_COV && (h->precision == HPC_PREC_BF16X3 || h->precision == HPC_PREC_TF32);
    // a staged X (same pointer and type): its prepared panels, else its device copy
    const bool prepared = tc_cov && h->pf_valid && h->pf_ptr == X && h->pf_xdt == xdt;
    const bool staged = tc_cov && !prepared && h->st_valid && h->st_ptr == X && h->st_xdt == xdt;
    if (prepared || staged) {
        // the panels, or the copy: not a later copy queued for the data after this one
        CUDA_TRY(cudaStreamWaitEvent(h->stream, prepared ? h->ev_prep : h->ev_copy, 0));
        h->pf_valid = false;
        on_host = 0;
        if (staged) {
            Xd = h->st_dev;
            h->st_valid = false;
        }
    } else if (h->pf_issued) {
        // this load rewrites the panels: after a staged preparation, which it discards;
        // a staged copy of another X stays (its panels follow this Gram)
        CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_prep, 0));
        h->pf_valid = false;
        if (!tc_cov) h->st_valid = false;
    }
    if (on_host && tc_cov) {
        // Page-locked host memory is mapped into the device's address space: the
        // tensor-core Gram's panel preparation, which reads X once, then reads it
        // there directly (the host-to-device transfer and the transpose in one pass).
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, X) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer) {
            Xd = a.devicePointer;
            on_host = 0;
        } else {
            cudaGetLastError();     // pageable memory: the query's error is not sticky; stage it
        }
    }
    if (on_host) {
        // the staging buffer is kept for the next load of the same size or smaller; a
        // staged copy in it is discarded (after its copy has landed)
        if (h->pf_issued) {
            CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_pf, 0));
            h->st_valid = false;
        }
        if (xbytes > h->x_stage_bytes) {
            if (h->pf_issued) CUDA_TRY(cudaEventSynchronize(h->ev_pf));
            if (h->x_stage) release(h, h->x_stage);
            h->x_stage = nullptr;
            h->x_stage_bytes = 0;
            CUDA_TRY(hold(h, &h->x_stage, xbytes));
            h->x_stage_bytes = xbytes;
        }
        CUDA_TRY(cudaMemcpyAsync(h->x_stage, X, xbytes, cudaMemcpyHostToDevice, h->stream));
        Xd = h->x_stage;
    }
    int launches = 0;
    if (h->opt.timing) CUDA_TRY(cudaEventRecord(h->ev[2], h->stream));
    cudaError_t e;
    int prec = h->precision;
    if (h->variant == HPC_OBS) {
        STATUS_TRY(load_x_obs(h, Xd));
        hpc::launch_transpose(Xd, xdt, h->n, h->p, h->p, h->xt, HPC_F32, h->ldx, 1.0, h->stream);
        hpc::launch_obs_split(prec, h->xt, h->p, h->ldx, h->ldx, h->xp[0], h->xp[1], h->n, h->p, h->stream);
        e = cudaGetLastError();
    } else if (prec == HPC_PREC_FP64 || prec == HPC_PREC_FP32) {
        e = hpc::gram_simt(Xd, xdt, h->n, h->p, h->S, h->vdt, h->ld, h->stream, &launches);
    } else {
        const size_t need = hpc::gram_tc_scratch_bytes(xdt, h->n, h->p, prec);
        if (need > h->gram_scratch_bytes) {
            if (h->pf_issued) CUDA_TRY(cudaEventSynchronize(h->ev_pf));
            if (h->gram_scratch) release(h, h->gram_scratch);
            h->gram_scratch = nullptr;
            h->tiles_sig = 0;     // a new buffer may reuse the old address
            h->gram_scratch_bytes = 0;
            CUDA_TRY(hold(h, &h->gram_scratch, need));
            h->gram_scratch_bytes = need;
        }
        e = hpc::gram_tc(Xd, xdt, h->n, h->p, static_cast<float*>(h->S), h->ld, prec, h->gram_scratch,
                         h->gram_scratch_bytes, h->stream, &launches, h->tune.gram_band,
                         h->opt.timing ? h->ev_gk : nullptr,
                         h->tune.gram_maxima ? static_cast<uint16_t*>(h->m1) : nullptr, h->nbm, prepared ? 1 : 0,
                         &h->tiles_sig, h->tune.gram_schedule, h->tune.gram_chunk, h->tune.gram_lead,
                         h->opt.timing ? h->ev_gp : nullptr);
        if (e == cudaErrorNotSupported) {
            std::snprintf(g_last_error, sizeof g_last_error, "tensor-core Gram not available for this shape");
            return HPC_ERR_NOT_IMPLEMENTED;
        }
        if (e == cudaSuccess && h->st_valid) {
            // a staged next X: its panels once this Gram has read them, on the staging
            // stream (one block per SM), so that the preparation overlaps the solve
            CUDA_TRY(cudaEventRecord(h->ev_gdone, h->stream));
            CUDA_TRY(cudaStreamWaitEvent(h->pf_stream, h->ev_gdone, 0));
            e = hpc::gram_tc_prepare(h->st_dev, h->st_xdt, h->n, h->p, prec, h->gram_scratch, h->gram_scratch_bytes,
                                     h->pf_stream, h->num_sms);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_prep, h->pf_stream);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_pf, h->pf_stream);
            h->pf_valid = e == cudaSuccess;
            h->pf_ptr = h->st_ptr;
            h->pf_xdt = h->st_xdt;
            h->st_valid = false;
        }
    }
    if (e != cudaSuccess) {
        set_cuda_error(e, "gram", __LINE__);
        return HPC_ERR_CUDA;
    }
    // block maxima of the bound screening: from the Gram's epilogue, or a pass over S
    const bool maxima_from_gram =
        h->variant == HPC_COV && (prec == HPC_PREC_BF16X3 || prec == HPC_PREC_TF32) && h->tune.gram_maxima;
    if (h->opt.timing) CUDA_TRY(cudaEventRecord(h->ev_ge, h->stream));
    if (h->m1 && !maxima_from_gram) {
        if (h->vdt == HPC_F64)
            hpc::launch_rowblock_max<double>(static_cast<const double*>(h->S), h->ld, (int)h->p, h->nbm,
                                             static_cast<unsigned short*>(h->m1), h->stream);
        else
            hpc::launch_rowblock_max<float>(static_cast<const float*>(h->S), h->ld, (int)h->p, h->nbm,
                                            static_cast<unsigned short*>(h->m1), h->stream);
        CUDA_TRY(cudaGetLastError());
    }
    if (h->m1g) {
        hpc::launch_group_max(static_cast<const unsigned short*>(h->m1), (int)h->p, h->nbm,
                              static_cast<unsigned short*>(h->m1g), h->ngl, h->stream);
        CUDA_TRY(cudaGetLastError());
    }
    if (h->opt.timing) {
        CUDA_TRY(cudaEventRecord(h->ev[3], h->stream));
        CUDA_TRY(cudaEventSynchronize(h->ev[3]));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
        h->ms_gram = ms;
        const bool tc = h->variant == HPC_COV && (prec == HPC_PREC_BF16X3 || prec == HPC_PREC_TF32);
        float mk = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&mk, tc ? h->ev_gk : h->ev[2], tc ? h->ev_gp : h->ev_ge));
        h->ms_gram_kernel = mk;
    }

    if (h->variant == HPC_COV && (prec == HPC_PREC_BF16X3 || prec == HPC_PREC_TF32)) {
        // the tensor-core Gram's error word, in the scratch it ran on (the Obs variant has no Gram)
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        const int w = hpc::gram_tc_take_error(h->gram_scratch, xdt, h->n, h->p, prec, h->stream);
        if (w != 0) {
            std::snprintf(g_last_error, sizeof g_last_error, "tensor-core Gram: bounded wait %d gave up", w);
            return HPC_ERR_DEVICE_TIMEOUT;
        }
    }
    h->cur = 0;
    STATUS_TRY(set_identity(h));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->loaded = true;
    return HPC_OK;
}

void destroy(hpc_ctx* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->pf_stream) {
        cudaStreamSynchronize(h->pf_stream);
        cudaStreamDestroy(h->pf_stream);
    }
    if (h->ev_pf) cudaEventDestroy(h->ev_pf);
    if (h->ev_gdone) cudaEventDestroy(h->ev_gdone);
    if (h->ev_copy) cudaEventDestroy(h->ev_copy);
    if (h->ev_prep) cudaEventDestroy(h->ev_prep);
    destroy_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    free_candidates(h);
    void* ptrs[] = {h->S, h->rp[0], h->rp[1], h->ci[0], h->ci[1], h->cv[0], h->cv[1], h->bk_cnt, h->bk_off,
                    h->bk_cur, h->bk_len, h->cnt2, h->scan_part, h->part_obj, h->part_ls, h->d_ctrl, h->gram_scratch,
                    h->rinfo, h->rdv, h->adj_buf, h->offlist, h->xt, h->yt, h->xp[0], h->xp[1],
                    h->yp[0], h->yp[1], h->pairs, h->bk_uoff, h->pmask, h->seqoff, h->bk_long,
                    h->m1, h->m1g, h->colmax, h->pairs_list, h->row_items, h->x_stage, h->bar};
    for (void* q : ptrs) release(h, q);
    if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
    for (auto& e : h->ev) if (e) cudaEventDestroy(e);
    if (h->ev_scr0) cudaEventDestroy(h->ev_scr0);
    if (h->ev_gk) cudaEventDestroy(h->ev_gk);
    if (h->ev_ge) cudaEventDestroy(h->ev_ge);
    if (h->ev_gp) cudaEventDestroy(h->ev_gp);
    if (h->ev_scr1) cudaEventDestroy(h->ev_scr1);
    delete h;
}

bool valid_dtype(int d) { return d == HPC_F32 || d == HPC_F64 || d == HPC_BF16; }

}  // namespace

extern "C" {

void hpc_default_options(hpc_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->eps = 1e-6;
    opt->max_iter = 1000;
    opt->max_halvings = 60;
    opt->precision = HPC_PREC_AUTO;
    opt->value_dtype = HPC_F32;
    opt->ls_window = 8;
    opt->capacity = 0;
    opt->max_capacity = 0;
    opt->x_on_host = 0;
    opt->timing = 1;
    opt->device_loop = 1;
}

const char* hpc_status_string(int s) {
    switch (s) {
        case HPC_OK: return "ok";
        case HPC_NOT_CONVERGED: return "not converged (max_iter reached)";
        case HPC_ERR_ARG: return "invalid argument";
        case HPC_ERR_OOM: return "device out of memory";
        case HPC_ERR_CAPACITY: return "candidate capacity exceeded";
        case HPC_ERR_NONPOS_DIAG: return "non-positive or missing diagonal entry";
        case HPC_ERR_NAN: return "NaN or Inf in gradient or objective";
        case HPC_ERR_LS_FAIL: return "line search failed within max_halvings";
        case HPC_ERR_CUDA: return "CUDA error";
        case HPC_ERR_NOT_IMPLEMENTED: return "not implemented";
        case HPC_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

const char* hpc_last_error(void) { return g_last_error; }

int hpc_choose_variant(int64_t n, int64_t p, double s, double t, double d, double gamma_ratio, double* cost_cov,
                       double* cost_obs) {
    if (n < 1 || p < 1) return HPC_ERR_ARG;
    if (!(s > 0.0)) s = 40.0;
    if (!(t > 0.0)) t = 3.0;
    if (!(d > 0.0)) d = 2.0;
    if (!(gamma_ratio > 0.0)) gamma_ratio = HPC_GAMMA_RATIO;
    const double N = (double)n, P = (double)p;
    // Lemma 3.1's flop counts, the sparse-dense terms weighted by gamma_sparse / gamma_dense
    const double cov = 2.0 * N * P * P + gamma_ratio * 2.0 * d * P * P * (s * t + 1.0);
    const double obs = 2.0 * N * P * P * s + gamma_ratio * 2.0 * d * N * P * (s * t + 1.0);
    if (cost_cov) *cost_cov = cov;
    if (cost_obs) *cost_obs = obs;
    return cov < obs ? HPC_COV : HPC_OBS;
}

int hpc_create(hpc_handle* out, const void* X, hpc_dtype xdt, int64_t n, int64_t p, double lambda1,
               double lambda2, hpc_variant variant, const hpc_options* opt, void* cuda_stream) {
    if (!out) return HPC_ERR_ARG;
    if (variant == HPC_OBS && n > hpc::kTransposeMaxRows) {
        std::snprintf(g_last_error, sizeof g_last_error, "the Obs variant transposes X: n <= %lld",
                      (long long)hpc::kTransposeMaxRows);
        return HPC_ERR_ARG;
    }
    *out = nullptr;
    hpc_options o;
    if (opt) o = *opt; else hpc_default_options(&o);
    if (n < 1 || p < 1 || p > (1ll << 30) || !(lambda1 >= 0.0) || !(lambda2 >= 0.0) || !(o.eps > 0.0) ||
        o.max_iter < 0 || o.max_halvings < 0 || o.max_halvings > 1000 || !valid_dtype(xdt) ||
        (o.value_dtype != HPC_F32 && o.value_dtype != HPC_F64) ||
        !(o.ls_window == 1 || o.ls_window == 2 || o.ls_window == 4 || o.ls_window == 8 || o.ls_window == 16) ||
        o.precision < HPC_PREC_AUTO || o.precision > HPC_PREC_TF32)
        return HPC_ERR_ARG;
    if (variant == HPC_AUTO)
        variant = (hpc_variant)hpc_choose_variant(n, p, 0.0, 0.0, 0.0, 0.0, nullptr, nullptr);
    if (variant != HPC_COV && variant != HPC_OBS) return HPC_ERR_ARG;
    int prec = o.precision;
    if (prec == HPC_PREC_AUTO) prec = (o.value_dtype == HPC_F64) ? HPC_PREC_FP64 : HPC_PREC_BF16X3;
    // the Obs variant's FP32-class Z product is the chunked BF16X3 split (the SIMT FP32
    // product would repeat a 2 n p^2 flop GEMM every iteration)
    if (variant == HPC_OBS && prec == HPC_PREC_FP32 && o.value_dtype == HPC_F32) prec = HPC_PREC_BF16X3;
    if (variant == HPC_OBS && (o.value_dtype != HPC_F32 || (prec != HPC_PREC_BF16X3 && prec != HPC_PREC_TF32))) {
        std::snprintf(g_last_error, sizeof g_last_error,
                      "the Obs variant runs its Z product on tensor cores: FP32 values with BF16X3 or TF32");
        return HPC_ERR_NOT_IMPLEMENTED;
    }
    if (prec == HPC_PREC_FP64 && o.value_dtype != HPC_F64) return HPC_ERR_ARG;
    if (o.value_dtype == HPC_F64 && prec != HPC_PREC_FP64) return HPC_ERR_ARG;

    hpc_ctx* h = new (std::nothrow) hpc_ctx();
    if (!h) return HPC_ERR_OOM;
    h->n = n; h->p = p; h->variant = variant; h->vdt = o.value_dtype; h->precision = prec;
    h->lam1 = lambda1; h->lam2 = lambda2; h->opt = o;
    h->tune.ls_window = o.ls_window;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->ld = (p + 127) / 128 * 128;

    auto fail = [&](int st) { destroy(h); return st; };
    auto cu = [&](cudaError_t e, const char* what, int line) -> int {
        if (e == cudaSuccess) return HPC_OK;
        set_cuda_error(e, what, line);
        return e == cudaErrorMemoryAllocation ? HPC_ERR_OOM : HPC_ERR_CUDA;
    };
#define CK(expr) do { int s_ = cu((expr), #expr, __LINE__); if (s_ != HPC_OK) return fail(s_); } while (0)
    const size_t vs = dtype_size(h->vdt);
    {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    if (variant == HPC_OBS) {
        h->ldx = (n + 63) / 64 * 64;
        CK(hold(h, &h->xt, (size_t)p * h->ldx * sizeof(float)));
        CK(hold(h, &h->yt, (size_t)p * h->ldx * sizeof(float)));
        const size_t pb = hpc::obs_panel_bytes(prec, n, p);
        for (int t = 0; t < hpc::obs_pieces(prec); ++t) {
            CK(hold(h, &h->xp[t], pb));
            CK(hold(h, &h->yp[t], pb));
        }
        std::vector<int2> pl;
        hpc::obs_pair_list(p, pl);
        h->npairs = (int64_t)pl.size();
        CK(hold(h, &h->pairs, pl.size() * sizeof(int2)));
        CK(cudaMemcpy(h->pairs, pl.data(), pl.size() * sizeof(int2), cudaMemcpyHostToDevice));
        if (!hpc::obs_make_maps(prec, h->yp[0], h->yp[1], h->xp[0], h->xp[1], n, p, h->obs_maps)) {
            std::snprintf(g_last_error, sizeof g_last_error, "TMA descriptors of the Obs panels could not be encoded");
            return fail(HPC_ERR_NOT_IMPLEMENTED);
        }
    }
    if (variant == HPC_COV) {
    CK(hold(h, &h->S, (size_t)p * h->ld * vs));
    CK(cudaMemsetAsync(h->S, 0, (size_t)p * h->ld * vs, h->stream));
    }
    if (variant == HPC_COV) {
        const int box_cols = h->vdt == HPC_F64 ? hpc::screen_box_cols<double>() : hpc::screen_box_cols<float>();
        std::memset(&h->smap, 0, sizeof h->smap);
        if (!hpc::encode_tensor_map_2d(&h->smap, h->S, (int)vs, (uint64_t)h->ld, (uint64_t)p, (uint64_t)h->ld * vs,
                                       (uint32_t)box_cols, (uint32_t)hpc::kScreenBoxRows)) {
            std::snprintf(g_last_error, sizeof g_last_error, "TMA descriptor of S could not be encoded");
            return fail(HPC_ERR_NOT_IMPLEMENTED);
        }
    }
    CK(hold(h, &h->rinfo, p * sizeof(int4)));
    CK(hold(h, &h->offlist, p * sizeof(int)));
    CK(hold(h, &h->rdv, h->ld * vs));
    CK(cudaMemsetAsync(h->rdv, 0, h->ld * vs, h->stream));
    CK(hold(h, &h->pmask, (h->ld / 32) * sizeof(unsigned)));
    CK(cudaMemsetAsync(h->pmask, 0, (h->ld / 32) * sizeof(unsigned), h->stream));
    if (variant == HPC_COV) {
        std::vector<long long> so;
        h->screen_grid = h->vdt == HPC_F64 ? hpc::screen_plan<double>((int)p, h->num_sms, so)
                                           : hpc::screen_plan<float>((int)p, h->num_sms, so);
        CK(hold(h, &h->seqoff, so.size() * sizeof(long long)));
        CK(cudaMemcpy(h->seqoff, so.data(), so.size() * sizeof(long long), cudaMemcpyHostToDevice));
        // bound screening (the grid is filled after each Gram)
        const int bj = h->vdt == HPC_F64 ? hpc::screen_box_cols<double>() : hpc::screen_box_cols<float>();
        h->nbm = (int)((p + bj - 1) / bj);
        const int64_t items = p * (int64_t)h->nbm / 2 + p;
        h->pairs_cap = (int)std::min<int64_t>(std::max<int64_t>(items / 4, 1024), 0x7ffffff0);
        CK(hold(h, &h->m1, (size_t)p * h->nbm * sizeof(unsigned short)));
        if (h->nbm % 8 == 0) {
            h->ngl = (h->nbm / 8 + 7) / 8 * 8;
            CK(hold(h, &h->m1g, (size_t)p * h->ngl * sizeof(unsigned short)));
        }
        CK(hold(h, &h->colmax, (size_t)h->nbm * vs));
        CK(hold(h, &h->pairs_list, (size_t)h->pairs_cap * sizeof(int2)));
        h->row_items_cap = (int)std::min<int64_t>((p + 7) / 8 * (int64_t)h->nbm, 0x7ffffff0);
        CK(hold(h, &h->row_items, (size_t)h->row_items_cap * sizeof(int2)));
    }
    for (int b = 0; b < 2; ++b) CK(hold(h, &h->rp[b], (p + 1) * sizeof(int)));
    const int64_t cap0 = o.capacity > 0 ? o.capacity : std::max<int64_t>(32 * p, 1024);
    {
        const int s = alloc_candidates(h, cap0);
        if (s != HPC_OK) return fail(s);
        const int s2 = grow_csr(h, 2 * cap0);
        if (s2 != HPC_OK) return fail(s2);
    }
    CK(hold(h, &h->bk_cnt, p * sizeof(int)));
    CK(hold(h, &h->bk_off, (p + 1) * sizeof(int)));
    CK(hold(h, &h->bk_cur, p * sizeof(int)));
    CK(hold(h, &h->bk_len, p * sizeof(int)));
    CK(hold(h, &h->bk_uoff, (p + 1) * sizeof(long long)));
    CK(hold(h, &h->bk_long, p * sizeof(int)));
    CK(hold(h, &h->cnt2, p * sizeof(int)));
    CK(hold(h, &h->scan_part, std::max<int64_t>(1, (p + 4095) / 4096) * sizeof(hpc::ScanPart)));
    h->nblk = (int)std::min<int64_t>((p + 7) / 8, 152 * 16);
    CK(hold(h, &h->part_obj, (size_t)h->nblk * 4 * sizeof(double)));
    CK(hold(h, &h->part_ls, (size_t)h->nblk * 16 * 4 * sizeof(double)));
    CK(hold(h, &h->d_ctrl, sizeof(hpc::Ctrl)));
    CK(cudaMemsetAsync(h->d_ctrl, 0, sizeof(hpc::Ctrl), h->stream));
    CK(hold(h, &h->bar, hpc::kBarWords * sizeof(unsigned)));
    CK(cudaMemsetAsync(h->bar, 0, hpc::kBarWords * sizeof(unsigned), h->stream));
    CK(cudaMallocHost(&h->h_ctrl, sizeof(hpc::Ctrl)));
    std::memset(h->h_ctrl, 0, sizeof(hpc::Ctrl));
    for (auto& e : h->ev) CK(cudaEventCreate(&e));
    CK(cudaEventCreate(&h->ev_scr0));
    CK(cudaEventCreate(&h->ev_gk));
    CK(cudaEventCreate(&h->ev_ge));
    CK(cudaEventCreate(&h->ev_gp));
    CK(cudaEventCreate(&h->ev_scr1));
#undef CK
    if (X) {
        const int s = load_x(h, X, xdt, o.x_on_host);
        if (s != HPC_OK) return fail(s);
    }
    *out = h;
    return HPC_OK;
}

int hpc_load_x(hpc_handle h, const void* X, hpc_dtype xdt, int x_on_host) {
    if (!h || !X || !valid_dtype(xdt)) return HPC_ERR_ARG;
    return load_x(h, X, xdt, x_on_host);
}

int hpc_prefetch_x(hpc_handle h, const void* X, hpc_dtype xdt, int x_on_host) {
    if (!h || !X || !valid_dtype(xdt)) return HPC_ERR_ARG;
    const bool tc_cov = h->variant == HPC_COV && (h->precision == HPC_PREC_BF16X3 || h->precision == HPC_PREC_TF32);
    if (!tc_cov || xdt == HPC_F64) return HPC_OK;       // nothing is staged ahead on the other paths
    const size_t need = hpc::gram_tc_scratch_bytes(xdt, h->n, h->p, h->precision);
    if (need > h->gram_scratch_bytes) return HPC_OK;     // the first hpc_load_x sizes the scratch
    if (!h->pf_stream) {
        CUDA_TRY(cudaStreamCreateWithFlags(&h->pf_stream, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&h->ev_pf, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&h->ev_prep, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&h->ev_gdone, cudaEventDisableTiming));
    }
    const void* dev = X;
    if (x_on_host) {
        // the copy engine moves X into the staging buffer: it needs no SM, so it runs
        // alongside the handle's next Gram.  The buffer's earlier readers on the staging
        // stream come first (in order); a load that staged through it has finished.
        const size_t xbytes = (size_t)h->n * h->p * dtype_size(xdt);
        if (xbytes > h->x_stage_bytes) {
            if (h->pf_issued) CUDA_TRY(cudaEventSynchronize(h->ev_pf));
            if (h->x_stage) release(h, h->x_stage);
            h->x_stage = nullptr;
            h->x_stage_bytes = 0;
            CUDA_TRY(hold(h, &h->x_stage, xbytes));
            h->x_stage_bytes = xbytes;
        }
        CUDA_TRY(cudaMemcpyAsync(h->x_stage, X, xbytes, cudaMemcpyHostToDevice, h->pf_stream));
        dev = h->x_stage;
    }
    CUDA_TRY(cudaEventRecord(h->ev_copy, h->pf_stream));
    CUDA_TRY(cudaEventRecord(h->ev_pf, h->pf_stream));
    h->pf_issued = true;
    h->st_valid = true;
    h->st_ptr = X;
    h->st_dev = dev;
    h->st_xdt = xdt;
    return HPC_OK;
}

int hpc_solve(hpc_handle h, hpc_stats* stats) {
    if (!h || !h->loaded) return HPC_ERR_ARG;
    return h->vdt == HPC_F64 ? run_iterations<double>(h, h->opt.max_iter, true, stats)
                             : run_iterations<float>(h, h->opt.max_iter, true, stats);
}

int hpc_iterate(hpc_handle h, int64_t k, hpc_stats* stats) {
    if (!h || !h->loaded || k < 0) return HPC_ERR_ARG;
    return h->vdt == HPC_F64 ? run_iterations<double>(h, k, false, stats)
                             : run_iterations<float>(h, k, false, stats);
}

int hpc_get_omega(hpc_handle h, int64_t* nnz_inout, int64_t* row_ptr, int32_t* col, void* val, hpc_dtype vdt,
                  int on_device) {
    if (!h || !nnz_inout) return HPC_ERR_ARG;
    if (!row_ptr) { *nnz_inout = h->nnz; return HPC_OK; }
    if (!col || !val || (vdt != HPC_F32 && vdt != HPC_F64)) return HPC_ERR_ARG;
    if (*nnz_inout < h->nnz) { *nnz_inout = h->nnz; return HPC_ERR_CAPACITY; }
    const int64_t p = h->p, nnz = h->nnz;
    const size_t ovs = dtype_size(vdt);
    int64_t* d_rp = row_ptr;
    int32_t* d_ci = col;
    void* d_v = val;
    if (!on_device) {
        CUDA_TRY(cudaMalloc(&d_rp, (p + 1) * sizeof(int64_t)));
        CUDA_TRY(cudaMalloc(&d_ci, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
        CUDA_TRY(cudaMalloc(&d_v, std::max<int64_t>(nnz, 1) * ovs));
    }
    if (h->vdt == HPC_F64)
        hpc::launch_csr_export<double>(h->rp[h->cur], h->ci[h->cur], as<double>(h->cv[h->cur]), (int)p, (int)nnz,
                                       d_rp, d_ci, d_v, vdt, h->stream);
    else
        hpc::launch_csr_export<float>(h->rp[h->cur], h->ci[h->cur], as<float>(h->cv[h->cur]), (int)p, (int)nnz,
                                      d_rp, d_ci, d_v, vdt, h->stream);
    CUDA_TRY(cudaGetLastError());
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(row_ptr, d_rp, (p + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(col, d_ci, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(val, d_v, nnz * ovs, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        cudaFree(d_rp); cudaFree(d_ci); cudaFree(d_v);
    } else {
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    *nnz_inout = nnz;
    return HPC_OK;
}

int hpc_set_omega(hpc_handle h, int64_t nnz, const int64_t* row_ptr, const int32_t* col, const void* val,
                  hpc_dtype vdt, int on_device) {
    if (!h || !row_ptr || !col || !val || nnz < h->p || (vdt != HPC_F32 && vdt != HPC_F64)) return HPC_ERR_ARG;
    const int64_t p = h->p;
    std::vector<int64_t> rp(p + 1);
    std::vector<int32_t> ci(nnz);
    std::vector<double> v(nnz);
    if (on_device) {
        CUDA_TRY(cudaMemcpy(rp.data(), row_ptr, (p + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(ci.data(), col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (vdt == HPC_F64) {
            CUDA_TRY(cudaMemcpy(v.data(), val, nnz * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(nnz);
            CUDA_TRY(cudaMemcpy(f.data(), val, nnz * sizeof(float), cudaMemcpyDeviceToHost));
            for (int64_t t = 0; t < nnz; ++t) v[t] = f[t];
        }
    } else {
        std::memcpy(rp.data(), row_ptr, (p + 1) * sizeof(int64_t));
        std::memcpy(ci.data(), col, nnz * sizeof(int32_t));
        if (vdt == HPC_F64) std::memcpy(v.data(), val, nnz * sizeof(double));
        else for (int64_t t = 0; t < nnz; ++t) v[t] = static_cast<const float*>(val)[t];
    }
    // validate: row_ptr monotone, columns sorted and in range, positive diagonal present
    if (rp[0] != 0 || rp[p] != nnz) return HPC_ERR_ARG;
    for (int64_t i = 0; i < p; ++i) {
        if (rp[i + 1] < rp[i]) return HPC_ERR_ARG;
        bool diag = false;
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
            if (ci[t] < 0 || ci[t] >= p) return HPC_ERR_ARG;
            if (t > rp[i] && ci[t] <= ci[t - 1]) return HPC_ERR_ARG;
            if (ci[t] == i) {
                if (!(v[t] > 0.0)) return HPC_ERR_NONPOS_DIAG;
                diag = true;
            }
            if (!std::isfinite(v[t])) return HPC_ERR_NAN;
        }
        if (!diag) return HPC_ERR_NONPOS_DIAG;
    }
    if (nnz > h->csr_cap) STATUS_TRY(grow_csr(h, 2 * nnz));
    std::vector<int> rp32(p + 1);
    for (int64_t i = 0; i <= p; ++i) rp32[i] = (int)rp[i];
    const int c = h->cur;
    CUDA_TRY(cudaMemcpyAsync(h->rp[c], rp32.data(), (p + 1) * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->ci[c], ci.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (h->vdt == HPC_F64) {
        CUDA_TRY(cudaMemcpyAsync(h->cv[c], v.data(), nnz * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    } else {
        std::vector<float> f(nnz);
        for (int64_t t = 0; t < nnz; ++t) f[t] = (float)v[t];
        CUDA_TRY(cudaMemcpyAsync(h->cv[c], f.data(), nnz * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    h->nnz = nnz;
    return HPC_OK;
}

}  // extern "C"

namespace {

// The lambda path as one graph launch (device loop): WHILE (points) { begin,
// iteration loop, end }.  Per-point statistics and, if asked for, the estimates
// are written to device buffers and copied back once.  An overflow ends the
// launch; the buffers grow, the graph is rebuilt and the point resumes.
template <typename T>
int solve_path_device(hpc_ctx* h, const double* lambda1, int64_t k, double lambda2, hpc_path_point* points,
                      int64_t* row_ptr, int32_t* col, float* val, int64_t* cap_inout) {
    const int64_t p = h->p;
    const int64_t cap = row_ptr ? *cap_inout : 0;
    struct Bufs {
        void* q[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        ~Bufs() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
            for (void* x : q) if (x) cudaFree(x);
        }
    } bf;
    hpc::PathOut out{};
    CUDA_TRY(cudaMalloc(&bf.q[0], k * sizeof(double)));
    CUDA_TRY(cudaMalloc(&bf.q[1], k * sizeof(hpc_path_point)));
    out.lam1 = static_cast<const double*>(bf.q[0]);
    out.points = static_cast<hpc_path_point*>(bf.q[1]);
    if (row_ptr) {
        CUDA_TRY(cudaMalloc(&bf.q[2], (size_t)k * (p + 1) * sizeof(int64_t)));
        CUDA_TRY(cudaMalloc(&bf.q[3], std::max<int64_t>(cap, 1) * sizeof(int32_t)));
        CUDA_TRY(cudaMalloc(&bf.q[4], std::max<int64_t>(cap, 1) * sizeof(float)));
        out.rp = static_cast<int64_t*>(bf.q[2]);
        out.ci = static_cast<int32_t*>(bf.q[3]);
        out.cv = static_cast<float*>(bf.q[4]);
    }
    out.cap = cap;
    out.k = (int)k;
    CUDA_TRY(cudaMemcpyAsync(bf.q[0], lambda1, k * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemsetAsync(bf.q[1], 0, k * sizeof(hpc_path_point), h->stream));
    h->lam1 = lambda1[0];
    h->lam2 = lambda2;
    hpc::Ctrl& c0 = *h->h_ctrl;
    c0.path_pt = c0.path_pt_next = 0;
    c0.path_k = (int)k;
    c0.path_keep = 0;
    c0.path_off = c0.path_off_next = c0.path_need = 0;
    c0.path_full = 0;
    STATUS_TRY(load_ctrl(h, h->opt.max_iter, true));
    int64_t epoch = -1;
    bool ran = false;
    for (int attempt = 0; attempt < 64; ++attempt) {
        if (!bf.e || epoch != h->epoch) {
            if (bf.e) { cudaGraphExecDestroy(bf.e); bf.e = nullptr; }
            if (bf.g) { cudaGraphDestroy(bf.g); bf.g = nullptr; }
            STATUS_TRY(build_path_graph<T>(h, out, &bf.g, &bf.e));
            epoch = h->epoch;
        }
        CUDA_TRY(cudaGraphLaunch(bf.e, h->stream));
        STATUS_TRY(read_ctrl(h));
        const hpc::Ctrl& c = *h->h_ctrl;
        h->nnz = c.nnz_cur;
        ran = true;
        int grow = 0;
        if (c.flags & (hpc::kFlagEmOverflow | hpc::kFlagBucketOverflow)) {
            STATUS_TRY(regrow(h, (int64_t)c.em_count + 1));
            grow = 1;
        } else if (c.flags & hpc::kFlagNnzOverflow) {
            STATUS_TRY(grow_csr(h, std::max<int64_t>(2 * h->csr_cap, (int64_t)c.nnz_next + 1)));
            h->regrows += 1;
            grow = 1;
        }
        if (!grow) break;
        ran = false;
        // resume the interrupted point with its counters
        const int one = 1;
        CUDA_TRY(cudaMemcpyAsync(&h->d_ctrl->path_keep, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    if (!ran) return HPC_ERR_CAPACITY;
    const hpc::Ctrl c = *h->h_ctrl;
    const int64_t reached = std::min<int64_t>(c.path_pt_next, k);
    std::vector<hpc_path_point> pts(k);
    CUDA_TRY(cudaMemcpy(pts.data(), bf.q[1], k * sizeof(hpc_path_point), cudaMemcpyDeviceToHost));
    int status = HPC_OK;
    for (int64_t t = 0; t < reached; ++t) {
        points[t] = pts[t];
        if (pts[t].status < 0 && status == HPC_OK) status = pts[t].status;
    }
    if (reached > 0) h->lam1 = lambda1[reached - 1];
    if (row_ptr) {
        CUDA_TRY(cudaMemcpy(row_ptr, bf.q[2], (size_t)reached * (p + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        const int64_t used = c.path_off_next;
        if (used > 0) {
            CUDA_TRY(cudaMemcpy(col, bf.q[3], used * sizeof(int32_t), cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemcpy(val, bf.q[4], used * sizeof(float), cudaMemcpyDeviceToHost));
        }
        if (c.path_full) {
            *cap_inout = c.path_need;
            return HPC_ERR_CAPACITY;
        }
        *cap_inout = used;
    }
    return status;
}

}  // namespace

extern "C" {

static int solve_path_host(hpc_handle h, const double* lambda1, int64_t k, double lambda2, hpc_path_point* points,
                           int64_t* row_ptr, int32_t* col, float* val, int64_t* cap_inout) {
    const int64_t cap = row_ptr ? *cap_inout : 0;
    int64_t used = 0;
    int status = HPC_OK;
    for (int64_t t = 0; t < k; ++t) {
        h->lam1 = lambda1[t];
        h->lam2 = lambda2;
        hpc_stats st{};
        const int r = h->vdt == HPC_F64 ? run_iterations<double>(h, h->opt.max_iter, true, &st)
                                        : run_iterations<float>(h, h->opt.max_iter, true, &st);
        hpc_path_point& pt = points[t];
        std::memset(&pt, 0, sizeof pt);
        pt.lambda1 = lambda1[t];
        pt.iterations = st.iterations;
        pt.ls_trials = st.ls_trials;
        pt.nnz = h->nnz;
        pt.status = r;
        pt.f = st.f;
        pt.F = st.F;
        pt.rel_change = st.rel_change;
        pt.ms = st.ms_total;
        if (r < 0) { status = r; break; }
        if (row_ptr) {
            if (used + h->nnz > cap) { *cap_inout = used + h->nnz; return HPC_ERR_CAPACITY; }
            int64_t m = cap - used;
            const int e = hpc_get_omega(h, &m, row_ptr + t * (h->p + 1), col + used, val + used, HPC_F32, 0);
            if (e != HPC_OK) return e;
            used += m;
        }
    }
    if (row_ptr) *cap_inout = used;
    return status;
}

int hpc_solve_path(hpc_handle h, const double* lambda1, int64_t k, double lambda2, hpc_path_point* points,
                   int64_t* row_ptr, int32_t* col, float* val, int64_t* cap_inout) {
    if (!h || !h->loaded || k < 0 || (k > 0 && (!lambda1 || !points)) || !(lambda2 >= 0.0)) return HPC_ERR_ARG;
    if (row_ptr && (!col || !val || !cap_inout)) return HPC_ERR_ARG;
    for (int64_t t = 0; t < k; ++t)
        if (!(lambda1[t] >= 0.0)) return HPC_ERR_ARG;
    if (k == 0 || !h->opt.device_loop || k > 0x7fffffff)
        return solve_path_host(h, lambda1, k, lambda2, points, row_ptr, col, val, cap_inout);
    return h->vdt == HPC_F64 ? solve_path_device<double>(h, lambda1, k, lambda2, points, row_ptr, col, val, cap_inout)
                             : solve_path_device<float>(h, lambda1, k, lambda2, points, row_ptr, col, val, cap_inout);
}

int hpc_solve_batch(hpc_handle* handles, int count, int threads, hpc_stats* stats) {
    if (count < 0 || (count > 0 && !handles)) return HPC_ERR_ARG;
    for (int t = 0; t < count; ++t)
        if (!handles[t] || !handles[t]->loaded) return HPC_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HPC_ERR_CUDA;
    std::vector<int> status(count, HPC_OK);
    std::vector<hpc_stats> st(count);
    bool all_device = count > 0;
    for (int t = 0; t < count; ++t) all_device = all_device && handles[t]->opt.device_loop;
    if (all_device) {
        // one graph launch for the whole batch
        std::vector<hpc_ctx*> hs(handles, handles + count);
        const int r = solve_batch_device(hs, status, st);
        if (r != HPC_OK) return r;
        int ret = HPC_OK;
        for (int t = 0; t < count; ++t) {
            if (stats) stats[t] = st[t];
            if (status[t] < 0 && ret >= 0) ret = status[t];
            else if (status[t] == HPC_NOT_CONVERGED && ret == HPC_OK) ret = HPC_NOT_CONVERGED;
        }
        return ret;
    }
    // handles that share a stream go to the same worker, in index order
    std::vector<std::vector<int>> groups;
    {
        std::vector<cudaStream_t> keys;
        for (int t = 0; t < count; ++t) {
            size_t g = 0;
            while (g < keys.size() && keys[g] != handles[t]->stream) ++g;
            if (g == keys.size()) { keys.push_back(handles[t]->stream); groups.emplace_back(); }
            groups[g].push_back(t);
        }
    }
    const int nw = threads > 0 ? std::min<int>(threads, (int)groups.size()) : (int)groups.size();
    std::atomic<int> next{0};
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (int g = next.fetch_add(1); g < (int)groups.size(); g = next.fetch_add(1))
            for (int t : groups[g]) status[t] = hpc_solve(handles[t], &st[t]);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    int ret = HPC_OK;
    for (int t = 0; t < count; ++t) {
        if (stats) stats[t] = st[t];
        if (status[t] < 0 && ret >= 0) ret = status[t];
        else if (status[t] == HPC_NOT_CONVERGED && ret == HPC_OK) ret = HPC_NOT_CONVERGED;
    }
    return ret;
}

int hpc_set_lambda(hpc_handle h, double lambda1, double lambda2) {
    if (!h || !(lambda1 >= 0.0) || !(lambda2 >= 0.0)) return HPC_ERR_ARG;
    h->lam1 = lambda1;
    h->lam2 = lambda2;
    return HPC_OK;
}

int hpc_get_s_entries(hpc_handle h, int64_t m, const int64_t* rows, const int64_t* cols, double* out) {
    if (!h || m < 0 || (m > 0 && (!rows || !cols || !out))) return HPC_ERR_ARG;
    if (!h->S || h->variant != HPC_COV) return HPC_ERR_ARG;
    for (int64_t t = 0; t < m; ++t)
        if (rows[t] < 0 || rows[t] >= h->p || cols[t] < 0 || cols[t] >= h->p) return HPC_ERR_ARG;
    if (m == 0) return HPC_OK;
    int64_t* d_idx = nullptr;
    double* d_out = nullptr;
    CUDA_TRY(cudaMalloc(&d_idx, 2 * m * sizeof(int64_t)));
    CUDA_TRY(cudaMalloc(&d_out, m * sizeof(double)));
    CUDA_TRY(cudaMemcpyAsync(d_idx, rows, m * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(d_idx + m, cols, m * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    hpc::launch_gather_s(h->S, h->vdt == HPC_F64, h->ld, m, d_idx, d_idx + m, d_out, h->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out, d_out, m * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaFree(d_idx);
    cudaFree(d_out);
    return HPC_OK;
}

int hpc_get_candidates(hpc_handle h, int64_t* m_inout, int64_t* rows, int64_t* cols, double* omega, double* grad) {
    if (!h || !m_inout) return HPC_ERR_ARG;
    const int64_t p = h->p;
    std::vector<int> off(p + 1), len(p);
    CUDA_TRY(cudaMemcpyAsync(off.data(), h->bk_off, (p + 1) * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(len.data(), h->bk_len, p * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    const int64_t tot = off[p];
    std::vector<int> col(std::max<int64_t>(tot, 1));
    std::vector<unsigned char> fl(std::max<int64_t>(tot, 1));
    const size_t vs = dtype_size(h->vdt);
    std::vector<char> om(std::max<int64_t>(tot, 1) * vs), g(std::max<int64_t>(tot, 1) * vs);
    if (tot > 0) {
        CUDA_TRY(cudaMemcpyAsync(col.data(), h->col_b, tot * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(fl.data(), h->fl_b, tot, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(om.data(), h->om_b, tot * vs, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(g.data(), h->g_b, tot * vs, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    auto val = [&](const std::vector<char>& a, int64_t t) {
        return h->vdt == HPC_F64 ? reinterpret_cast<const double*>(a.data())[t]
                                 : (double)reinterpret_cast<const float*>(a.data())[t];
    };
    int64_t m = 0;
    for (int64_t i = 0; i < p; ++i)
        for (int64_t t = off[i]; t < off[i] + len[i]; ++t)
            if (fl[t] & hpc::kEntKeep) {
                if (rows) {
                    if (m >= *m_inout) return HPC_ERR_CAPACITY;
                    rows[m] = i; cols[m] = col[t];
                    if (omega) omega[m] = val(om, t);
                    if (grad) grad[m] = val(g, t);
                }
                ++m;
            }
    *m_inout = m;
    return HPC_OK;
}

}  // extern "C"

namespace {

int adj_reserve(hpc_ctx* h, size_t bytes) {
    if (bytes <= h->adj_bytes) return HPC_OK;
    if (h->adj_buf) release(h, h->adj_buf);
    h->adj_buf = nullptr;
    h->adj_bytes = 0;
    CUDA_TRY(hold(h, &h->adj_buf, bytes));
    h->adj_bytes = bytes;
    return HPC_OK;
}

template <typename T>
hpc::Csr<T> cur_csr(hpc_ctx* h) { return {h->rp[h->cur], h->ci[h->cur], as<T>(h->cv[h->cur])}; }

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

template <typename T>
int smooth_value_t(hpc_ctx* h, double* f) {
    const int p = (int)h->p;
    const int64_t nnz = h->nnz;
    const size_t b_v = align256(nnz * sizeof(double));
    STATUS_TRY(adj_reserve(h, 2 * b_v + align256(1024 * 3 * sizeof(double)) + 256));
    uint8_t* base = static_cast<uint8_t*>(h->adj_buf);
    double* om_d = reinterpret_cast<double*>(base);
    double* Tv = reinterpret_cast<double*>(base + b_v);
    double* part = reinterpret_cast<double*>(base + 2 * b_v);
    double* out3 = reinterpret_cast<double*>(base + 2 * b_v + align256(1024 * 3 * sizeof(double)));
    hpc::Csr<T> om = cur_csr<T>(h);
    hpc::launch_row_info<T>(p, om, h->rinfo, as<T>(h->rdv), h->stream);
    hpc::launch_support_vectors<T>(p, nnz, om, om_d, Tv, h->stream);     // Tv used as scratch for signs
    hpc::launch_support_product<T>(p, om, h->rinfo, om_d, static_cast<const T*>(h->S), h->ld, Tv, h->stream);
    hpc::launch_smooth_parts<T>(p, om, Tv, part, out3, h->stream);
    CUDA_TRY(cudaGetLastError());
    double o[3];
    CUDA_TRY(cudaMemcpyAsync(o, out3, sizeof o, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *f = -o[2] + 0.5 * o[0] + 0.5 * h->lam2 * o[1];
    return HPC_OK;
}

template <typename T>
int backward_t(hpc_ctx* h, const void* X, int xdt, double grad_loss, void* dOmega, int64_t ld_domega, void* dX) {
    const int p = (int)h->p;
    const int64_t n = h->n;
    hpc::Csr<T> om = cur_csr<T>(h);
    hpc::launch_row_info<T>(p, om, h->rinfo, as<T>(h->rdv), h->stream);
    if (dOmega)
        hpc::launch_dense_grad<T>(p, om, h->rinfo, as<T>(h->rdv), static_cast<const T*>(h->S), h->ld,
                                  static_cast<T*>(dOmega), ld_domega, (T)h->lam2, (T)grad_loss, h->stream);
    if (dX) {
        const size_t plane = align256((size_t)p * n * sizeof(T));
        STATUS_TRY(adj_reserve(h, 2 * plane));
        T* xt = static_cast<T*>(h->adj_buf);
        T* yt = reinterpret_cast<T*>(static_cast<uint8_t*>(h->adj_buf) + plane);
        const int tdt = sizeof(T) == 8 ? HPC_F64 : HPC_F32;
        hpc::launch_transpose(X, xdt, n, p, p, xt, tdt, n, 1.0, h->stream);                  // X^T (p x n)
        hpc::launch_spmm_dense<T>(p, om, h->rinfo, as<T>(h->rdv), xt, n, n, yt, n, h->stream);  // Y^T = Omega X^T
        // dX = (Omega Y^T)^T grad_loss / n, transposed as it is written
        hpc::launch_spmm_dense_t<T>(p, om, h->rinfo, as<T>(h->rdv), yt, n, n, static_cast<T*>(dX), p,
                                    (T)(grad_loss / (double)n), h->stream);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return HPC_OK;
}

// dL/dOmega at the support entries (FP64, CSR order) and optionally dL/dX, at the current
// iterate.  Cov: (Omega S)_ij by gathers of S; Obs: from Y^T = Omega X^T and the resident X^T.
template <typename T>
int backward_support_t(hpc_ctx* h, const void* X, int xdt, double grad_loss, double* dvals, void* dX) {
    const int p = (int)h->p;
    const int64_t nnz = h->nnz;
    if (dvals) {
        const size_t b_v = align256(nnz * sizeof(double));
        const size_t b_i = align256(nnz * sizeof(int));
        const size_t b_y = h->S ? 0 : align256((size_t)p * h->ldx * sizeof(T));
        STATUS_TRY(adj_reserve(h, 2 * b_v + 2 * b_i + b_y));
        uint8_t* q = static_cast<uint8_t*>(h->adj_buf);
        double* om_d = reinterpret_cast<double*>(q); q += b_v;
        double* Tv = reinterpret_cast<double*>(q); q += b_v;
        int* tr = reinterpret_cast<int*>(q); q += b_i;
        int* rowid = reinterpret_cast<int*>(q); q += b_i;
        hpc::Csr<T> om = cur_csr<T>(h);
        hpc::launch_row_info<T>(p, om, h->rinfo, as<T>(h->rdv), h->stream);
        hpc::launch_transpose_index<T>(p, om, tr, rowid, h->stream);
        hpc::launch_support_vectors<T>(p, nnz, om, om_d, Tv, h->stream);      // Tv: scratch for the signs
        if (h->S) {
            hpc::launch_support_product<T>(p, om, h->rinfo, om_d, static_cast<const T*>(h->S), h->ld, Tv, h->stream);
        } else {
            T* yt = reinterpret_cast<T*>(q);
            const T* xt = reinterpret_cast<const T*>(h->xt);
            hpc::launch_spmm_dense<T>(p, om, h->rinfo, as<T>(h->rdv), xt, h->ldx, h->ldx, yt, h->ldx, h->stream);
            hpc::launch_support_sddmm<T>(p, om, yt, xt, h->ldx, h->n, Tv, h->stream);
        }
        hpc::launch_support_grad<T>(nnz, rowid, om, tr, Tv, h->lam2, grad_loss, dvals, h->stream);
        CUDA_TRY(cudaGetLastError());
    }
    if (dX) return backward_t<T>(h, X, xdt, grad_loss, nullptr, h->p, dX);
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return HPC_OK;
}

// L_val(Omega) = -sum log w_ii + tr(Omega S_val Omega) / 2 at the current iterate, with
// tr(Omega S_val Omega) = sum_e w_e (Omega S_val)_e over the support and (Omega S_val)_ij =
// <(X_val Omega)_{:,i}, X_val_{:,j}> / n_val (S_val is never formed).
template <typename T>
int heldout_t(hpc_ctx* h, const void* Xval, int xdt, int64_t nval, double* loss) {
    const int p = (int)h->p;
    const int64_t nnz = h->nnz;
    const size_t b_x = align256((size_t)p * nval * sizeof(T));
    const size_t b_v = align256(nnz * sizeof(double));
    const size_t b_p = align256(1024 * 3 * sizeof(double));
    STATUS_TRY(adj_reserve(h, 2 * b_x + b_v + b_p + 256));
    uint8_t* q = static_cast<uint8_t*>(h->adj_buf);
    T* xtv = reinterpret_cast<T*>(q); q += b_x;
    T* ytv = reinterpret_cast<T*>(q); q += b_x;
    double* Tv = reinterpret_cast<double*>(q); q += b_v;
    double* part = reinterpret_cast<double*>(q); q += b_p;
    double* out3 = reinterpret_cast<double*>(q);
    cudaStream_t s = h->stream;
    hpc::Csr<T> om = cur_csr<T>(h);
    hpc::launch_row_info<T>(p, om, h->rinfo, as<T>(h->rdv), s);
    const int tdt = sizeof(T) == 8 ? HPC_F64 : HPC_F32;
    hpc::launch_transpose(Xval, xdt, nval, p, p, xtv, tdt, nval, 1.0, s);
    hpc::launch_spmm_dense<T>(p, om, h->rinfo, as<T>(h->rdv), xtv, nval, nval, ytv, nval, s);
    hpc::launch_support_sddmm<T>(p, om, ytv, xtv, nval, nval, Tv, s);
    hpc::launch_smooth_parts<T>(p, om, Tv, part, out3, s);
    CUDA_TRY(cudaGetLastError());
    double o[3];
    CUDA_TRY(cudaMemcpyAsync(o, out3, sizeof o, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *loss = -o[2] + 0.5 * o[0];
    return HPC_OK;
}

template <typename T>
int hypergrad_t(hpc_ctx* h, const void* Xval, int xdt, int64_t nval, double cg_tol, int64_t cg_max, double* dl1,
                double* dl2, hpc_hypergrad_info* info) {
    const int p = (int)h->p;
    const int64_t nnz = h->nnz;
    const size_t vs = sizeof(T);
    const size_t b_x = align256((size_t)p * nval * vs);
    const size_t b_v = align256(nnz * sizeof(double));
    const size_t b_i = align256(nnz * sizeof(int));
    const size_t b_p = align256(1024 * sizeof(double));
    STATUS_TRY(adj_reserve(h, 2 * b_x + 9 * b_v + 2 * b_i + b_p + 4 * 256));
    uint8_t* q = static_cast<uint8_t*>(h->adj_buf);
    T* xtv = reinterpret_cast<T*>(q); q += b_x;
    T* ytv = reinterpret_cast<T*>(q); q += b_x;
    double* om_d = reinterpret_cast<double*>(q); q += b_v;
    double* sgn = reinterpret_cast<double*>(q); q += b_v;
    double* Tv = reinterpret_cast<double*>(q); q += b_v;
    double* bvec = reinterpret_cast<double*>(q); q += b_v;
    double* x = reinterpret_cast<double*>(q); q += b_v;
    double* r = reinterpret_cast<double*>(q); q += b_v;
    double* pbuf[2];
    pbuf[0] = reinterpret_cast<double*>(q); q += b_v;
    pbuf[1] = reinterpret_cast<double*>(q); q += b_v;
    double* Ap = reinterpret_cast<double*>(q); q += b_v;
    int* tr = reinterpret_cast<int*>(q); q += b_i;
    int* rowid = reinterpret_cast<int*>(q); q += b_i;
    double* part = reinterpret_cast<double*>(q); q += b_p;
    void* cg = q; q += 256;
    double* out = reinterpret_cast<double*>(q);
    cudaStream_t s = h->stream;
    hpc::Csr<T> om = cur_csr<T>(h);

    hpc::launch_row_info<T>(p, om, h->rinfo, as<T>(h->rdv), s);
    hpc::launch_transpose_index<T>(p, om, tr, rowid, s);
    hpc::launch_support_vectors<T>(p, nnz, om, om_d, sgn, s);
    // b = gradient of the held-out loss on the support.  Its term (Omega S_val)_ij is
    // (1/n_val) <(X_val Omega)_{:,i}, X_val_{:,j}>: Y^T = Omega X_val^T, then one row
    // pair per support entry; S_val itself is never formed.
    const int tdt = sizeof(T) == 8 ? HPC_F64 : HPC_F32;
    hpc::launch_transpose(Xval, xdt, nval, p, p, xtv, tdt, nval, 1.0, s);
    hpc::launch_spmm_dense<T>(p, om, h->rinfo, as<T>(h->rdv), xtv, nval, nval, ytv, nval, s);
    hpc::launch_support_sddmm<T>(p, om, ytv, xtv, nval, nval, Tv, s);
    hpc::launch_support_combine<T>(nnz, rowid, om, tr, Tv, om_d, h->lam2, 1, bvec, nullptr, 0.0, cg, s);
    // CG on H_A v = b
    CUDA_TRY(cudaMemsetAsync(x, 0, nnz * sizeof(double), s));
    CUDA_TRY(cudaMemcpyAsync(r, bvec, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(pbuf[0], bvec, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const int nb = hpc::cg_part_blocks(nnz);
    const double tol2 = cg_tol * cg_tol;
    CUDA_TRY(cudaMemsetAsync(cg, 0, hpc::cg_state_bytes(), s));      // the fused reductions' ticket starts at 0
    hpc::launch_dot_part(nnz, r, r, part, s);
    hpc::launch_cg_scalar(part, nb, 0, tol2, cg, s);
    // One CG iteration k is three kernels: the direction p = r + beta p_old (beta = 0 at
    // first, so p = r = b) with its S gathers, Ap = H_A p with alpha, then x, r, beta and
    // the stopping test.  Directions alternate between two buffers.
    const hpc::Csr<T> omc = om;
    auto iteration = [&](int64_t k, cudaStream_t st) {
        double* p_old = pbuf[k & 1];
        double* p_new = pbuf[(k + 1) & 1];
        hpc::launch_support_product_p<T>(nnz, rowid, omc, h->rinfo, r, p_old, p_new, cg, static_cast<const T*>(h->S),
                                         h->ld, Tv, st);
        hpc::launch_support_combine<T>(nnz, rowid, omc, tr, Tv, p_new, h->lam2, 0, Ap, part, tol2, cg, st);
        hpc::launch_cg_xr(nnz, cg, p_new, Ap, x, r, part, tol2, st);
    };
    // Chunks of kChunk iterations run as one captured graph (an even count, so every
    // chunk starts on buffer 0); the host reads the stop flag between chunks.
    constexpr int kChunk = 8;
    cudaGraphExec_t chunk = nullptr;
    if (cg_max >= kChunk) {
        STATUS_TRY(ensure_cap_stream(h));
        cudaStream_t cs = h->cap_stream;
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kChunk; ++k) iteration(k, cs);
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        if (ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            set_cuda_error(ec != cudaSuccess ? ec : cudaErrorUnknown, "CG chunk capture", __LINE__);
            return HPC_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&chunk, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) { set_cuda_error(ei, "CG chunk instantiate", __LINE__); return HPC_ERR_CUDA; }
    }
    int64_t it = 0;
    int done = 0;
    int status = HPC_OK;
    while (it < cg_max && status == HPC_OK) {
        cudaError_t e2 = cudaSuccess;
        if (chunk && it + kChunk <= cg_max) {
            e2 = cudaGraphLaunch(chunk, s);
            it += kChunk;
        } else {
            for (; it < cg_max; ++it) iteration(it, s);     // the tail (it is even here)
            e2 = cudaGetLastError();
        }
        int dd = 0;
        if (e2 == cudaSuccess)
            e2 = cudaMemcpyAsync(&dd, reinterpret_cast<uint8_t*>(cg) + 5 * sizeof(double), sizeof(int),
                                 cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        if (e2 != cudaSuccess) { set_cuda_error(e2, "CG", __LINE__); status = HPC_ERR_CUDA; }
        if (dd) { done = dd; break; }
    }
    if (chunk) cudaGraphExecDestroy(chunk);
    if (status != HPC_OK) return status;
    // dL_val/dlambda1 = -<v, sgn_off>, dL_val/dlambda2 = -<v, Omega_A>
    hpc::launch_dot_part(nnz, x, sgn, part, s);
    hpc::launch_reduce_parts(part, nb, out, s);
    hpc::launch_dot_part(nnz, x, om_d, part, s);
    hpc::launch_reduce_parts(part, nb, out + 1, s);
    CUDA_TRY(cudaGetLastError());
    double o[2], st[2];
    CUDA_TRY(cudaMemcpyAsync(o, out, sizeof o, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(st, cg, sizeof st, cudaMemcpyDeviceToHost, s));   // rr, rr0
    CUDA_TRY(cudaStreamSynchronize(s));
    *dl1 = -o[0];
    *dl2 = -o[1];
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->cg_iterations = it;
        info->rel_residual = st[1] > 0.0 ? std::sqrt(st[0] / st[1]) : 0.0;
        info->support = nnz;
        info->converged = done == 1 ? 1 : 0;
    }
    if (done == 2) {
        std::snprintf(g_last_error, sizeof g_last_error, "CG met a non-positive curvature on the support");
        return HPC_ERR_NAN;
    }
    return done == 1 ? HPC_OK : HPC_NOT_CONVERGED;
}

// ---------------------------------------------------------------- autotuner
bool tuning_ok(const hpc_tuning& t) {
    const int w = t.ls_window;
    return t.gram_band >= 1 && t.gram_band <= 256 && (w == 1 || w == 2 || w == 4 || w == 8 || w == 16) &&
           t.ls_blocks_per_sm >= 0 && t.ls_blocks_per_sm <= 8 && t.rows_ctas_per_sm >= 1 && t.rows_ctas_per_sm <= 4 &&
           (t.gram_maxima == 0 || t.gram_maxima == 1) && (t.screen_bounds == 0 || t.screen_bounds == 1) &&
           (t.gram_schedule == 0 || t.gram_schedule == 1) && t.gram_chunk >= 0 &&
           t.gram_lead >= 0 && (t.fused_tail == 0 || t.fused_tail == 1);
}

void apply_tuning(hpc_ctx* h, const hpc_tuning& t) {
    h->tune = t;
    h->epoch += 1;          // the device-loop graph captured the old launch shapes
}

// A copy of the current iterate (CSR) that trials restore before they run.
struct IterateCopy {
    int* rp = nullptr;
    int* ci = nullptr;
    void* cv = nullptr;
    int64_t nnz = 0;
    ~IterateCopy() {
        if (rp) cudaFree(rp);
        if (ci) cudaFree(ci);
        if (cv) cudaFree(cv);
    }
};

int save_iterate(hpc_ctx* h, IterateCopy& c) {
    const size_t vs = dtype_size(h->vdt);
    c.nnz = h->nnz;
    CUDA_TRY(cudaMalloc(&c.rp, (h->p + 1) * sizeof(int)));
    CUDA_TRY(cudaMalloc(&c.ci, std::max<int64_t>(c.nnz, 1) * sizeof(int)));
    CUDA_TRY(cudaMalloc(&c.cv, std::max<int64_t>(c.nnz, 1) * vs));
    CUDA_TRY(cudaMemcpyAsync(c.rp, h->rp[h->cur], (h->p + 1) * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(c.ci, h->ci[h->cur], c.nnz * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(c.cv, h->cv[h->cur], c.nnz * vs, cudaMemcpyDeviceToDevice, h->stream));
    return HPC_OK;
}

int restore_iterate(hpc_ctx* h, const IterateCopy& c) {
    const size_t vs = dtype_size(h->vdt);
    if (c.nnz > h->csr_cap) STATUS_TRY(grow_csr(h, c.nnz));
    CUDA_TRY(cudaMemcpyAsync(h->rp[h->cur], c.rp, (h->p + 1) * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->ci[h->cur], c.ci, c.nnz * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->cv[h->cur], c.cv, c.nnz * vs, cudaMemcpyDeviceToDevice, h->stream));
    h->nnz = c.nnz;
    return HPC_OK;
}

void add_trial(hpc_tune_report* r, int knob, int value, double ms) {
    if (!r || r->ntrials >= HPC_TUNE_MAX_TRIALS) return;
    r->trials[r->ntrials].knob = knob;
    r->trials[r->ntrials].value = value;
    r->trials[r->ntrials].ms = ms;
    r->ntrials += 1;
}

// Milliseconds per iteration of `iters` iterations from the saved iterate under
// tuning t (one untimed iteration first, which also captures the graph).
template <typename T>
int time_iterations(hpc_ctx* h, const IterateCopy& c, const hpc_tuning& t, int64_t iters, double* ms) {
    apply_tuning(h, t);
    hpc_stats st{};
    STATUS_TRY(restore_iterate(h, c));
    int r = run_iterations<T>(h, 1, false, &st);
    if (r != HPC_OK) return r;
    STATUS_TRY(restore_iterate(h, c));
    r = run_iterations<T>(h, iters, false, &st);
    if (r != HPC_OK) return r;
    *ms = st.ms_total / (double)std::max<int64_t>(st.iterations, 1);
    return HPC_OK;
}

template <typename T>
int autotune_t(hpc_ctx* h, const void* X, int xdt, int on_host, int64_t iters, hpc_tuning* best,
               hpc_tune_report* rep) {
    const int timing0 = h->opt.timing;
    h->opt.timing = 1;
    hpc_tuning t = h->tune;
    int status = HPC_OK;
    // 1. the Gram's tile-order band (tensor-core Gram only).  Under the power cap the
    // SM clock drifts over seconds, so the candidates are timed round-robin, three
    // rounds, and each keeps its fastest load.
    const bool tc_gram = h->variant == HPC_COV && (h->precision == HPC_PREC_BF16X3 || h->precision == HPC_PREC_TF32);
    if (X && tc_gram) {
        constexpr int kRounds = 3;
        const int nbi = (int)((h->p + 255) / 256 * 256 / 128);
        std::vector<int> bands;
        for (int b : {2, 4, 8, 16, 32, 64})
            if (b <= nbi || bands.empty()) bands.push_back(b);
        std::vector<double> band_ms(bands.size(), 1e300);
        for (int r = 0; r < kRounds && status == HPC_OK; ++r)
            for (size_t q = 0; q < bands.size() && status == HPC_OK; ++q) {
                hpc_tuning u = t;
                u.gram_band = bands[q];
                apply_tuning(h, u);
                status = load_x(h, X, xdt, on_host);
                band_ms[q] = std::min(band_ms[q], h->ms_gram);
            }
        if (status == HPC_OK) {
            size_t best = 0;
            for (size_t q = 0; q < bands.size(); ++q) {
                add_trial(rep, 0, bands[q], band_ms[q]);
                if (band_ms[q] < band_ms[best]) best = q;
            }
            t.gram_band = bands[best];
        }
        // the tile schedule at that band: shared counter or static round-robin
        const int sched[2] = {1, 0};
        double sc_ms[2] = {1e300, 1e300};
        for (int r = 0; r < kRounds && status == HPC_OK; ++r)
            for (int q = 0; q < 2 && status == HPC_OK; ++q) {
                hpc_tuning u = t;
                u.gram_schedule = sched[q];
                apply_tuning(h, u);
                status = load_x(h, X, xdt, on_host);
                sc_ms[q] = std::min(sc_ms[q], h->ms_gram);
            }
        if (status == HPC_OK) {
            for (int q = 0; q < 2; ++q) add_trial(rep, 5, sched[q], sc_ms[q]);
            t.gram_schedule = sc_ms[1] < sc_ms[0] ? sched[1] : sched[0];
        }
        // block maxima from the Gram's epilogue or from a pass over S, whole loads timed
        const int fused[2] = {1, 0};
        double mx_ms[2] = {1e300, 1e300};
        for (int r = 0; r < kRounds && status == HPC_OK; ++r)
            for (int q = 0; q < 2 && status == HPC_OK; ++q) {
                hpc_tuning u = t;
                u.gram_maxima = fused[q];
                apply_tuning(h, u);
                status = load_x(h, X, xdt, on_host);
                mx_ms[q] = std::min(mx_ms[q], h->ms_gram);
            }
        if (status == HPC_OK) {
            for (int q = 0; q < 2; ++q) add_trial(rep, 4, fused[q], mx_ms[q]);
            // the separate pass re-reads S (17 GB at p = 65536), the fused form costs the
            // epilogue a little: it has to win by more than the clock noise (2%)
            t.gram_maxima = mx_ms[1] < 0.98 * mx_ms[0] ? fused[1] : fused[0];
        }
        apply_tuning(h, t);     // S and the maxima of the last trial are the same either way
    } else if (X) {
        status = load_x(h, X, xdt, on_host);
    }
    // 2. iteration knobs, one after another, from the current iterate
    if (status == HPC_OK && iters > 0) {
        IterateCopy c;
        status = save_iterate(h, c);
        struct Knob { int id; std::vector<int> vals; };
        // (the tail's form is not tuned here: the one-launch tail is a cooperative kernel,
        // which waits for the whole grid to be resident, so it queues behind work on
        // other streams, such as hpc_prefetch_x's transpose, that an iteration-only
        // timing does not see)
        const Knob knobs[] = {{1, {2, 4, 8, 16}}, {3, {1, 2, 3, 4}}, {2, {1, 2, 3}}};
        for (const Knob& k : knobs) {
            if (status != HPC_OK) break;
            if (k.id == 3 && h->variant == HPC_OBS) continue;       // Obs has no row kernel
            double best_ms = 1e300;
            int best_v = 0;
            for (int v : k.vals) {
                hpc_tuning u = t;
                if (k.id == 1) u.ls_window = v; else if (k.id == 2) u.ls_blocks_per_sm = v; else u.rows_ctas_per_sm = v;
                double ms = 0;
                status = time_iterations<T>(h, c, u, iters, &ms);
                if (status != HPC_OK) break;
                add_trial(rep, k.id, v, ms);
                if (ms < best_ms) { best_ms = ms; best_v = v; }
            }
            if (status != HPC_OK) break;
            if (k.id == 1) t.ls_window = best_v; else if (k.id == 2) t.ls_blocks_per_sm = best_v; else t.rows_ctas_per_sm = best_v;
        }
        if (status == HPC_OK) status = restore_iterate(h, c);
        if (status == HPC_OK) status = cudaStreamSynchronize(h->stream) == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
    }
    apply_tuning(h, t);
    h->opt.timing = timing0;
    if (best) *best = t;
    return status;
}

}  // namespace

extern "C" {

int hpc_get_block_maxima(hpc_handle h, int64_t* count_inout, uint16_t* out) {
    if (!h || !count_inout) return HPC_ERR_ARG;
    if (!h->m1 || !h->loaded) return HPC_ERR_NOT_IMPLEMENTED;
    const int64_t total = h->p * (int64_t)h->nbm;
    if (!out) { *count_inout = total; return HPC_OK; }
    if (*count_inout < total) { *count_inout = total; return HPC_ERR_CAPACITY; }
    CUDA_TRY(cudaMemcpyAsync(out, h->m1, total * sizeof(uint16_t), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *count_inout = total;
    return HPC_OK;
}

int hpc_get_tuning(hpc_handle h, hpc_tuning* t) {
    if (!h || !t) return HPC_ERR_ARG;
    *t = h->tune;
    return HPC_OK;
}

int hpc_set_tuning(hpc_handle h, const hpc_tuning* t) {
    if (!h || !t || !tuning_ok(*t)) return HPC_ERR_ARG;
    apply_tuning(h, *t);
    return HPC_OK;
}

int hpc_autotune(hpc_handle h, const void* X, hpc_dtype xdt, int x_on_host, int64_t iters, hpc_tuning* best,
                 hpc_tune_report* report) {
    if (!h || iters < 0 || (X && !valid_dtype(xdt))) return HPC_ERR_ARG;
    if (!X && !h->loaded) return HPC_ERR_ARG;
    if (report) std::memset(report, 0, sizeof *report);
    return h->vdt == HPC_F64 ? autotune_t<double>(h, X, xdt, x_on_host, iters, best, report)
                             : autotune_t<float>(h, X, xdt, x_on_host, iters, best, report);
}

int hpc_smooth_value(hpc_handle h, double* f) {
    if (!h || !h->loaded || !f) return HPC_ERR_ARG;
    if (!h->S) return HPC_ERR_NOT_IMPLEMENTED;      // needs S (Cov variant)
    return h->vdt == HPC_F64 ? smooth_value_t<double>(h, f) : smooth_value_t<float>(h, f);
}

int hpc_backward(hpc_handle h, const void* X, hpc_dtype xdt, double grad_loss, void* dOmega, int64_t ld_domega,
                 void* dX) {
    if (!h || !h->loaded || (dX && !X) || (dOmega && ld_domega < h->p) || !valid_dtype(xdt) ||
        !std::isfinite(grad_loss))
        return HPC_ERR_ARG;
    if (!h->S) return HPC_ERR_NOT_IMPLEMENTED;      // needs S (Cov variant)
    if (dX && h->n > hpc::kTransposeMaxRows) {
        std::snprintf(g_last_error, sizeof g_last_error, "dL/dX transposes X: n <= %lld",
                      (long long)hpc::kTransposeMaxRows);
        return HPC_ERR_ARG;
    }
    return h->vdt == HPC_F64 ? backward_t<double>(h, X, xdt, grad_loss, dOmega, ld_domega, dX)
                             : backward_t<float>(h, X, xdt, grad_loss, dOmega, ld_domega, dX);
}

int hpc_backward_support(hpc_handle h, const void* X, hpc_dtype xdt, double grad_loss, double* dOmega_vals,
                         void* dX) {
    if (!h || !h->loaded || (dX && !X) || !valid_dtype(xdt) || !std::isfinite(grad_loss)) return HPC_ERR_ARG;
    if (dX && !h->S) return HPC_ERR_NOT_IMPLEMENTED;     // dL/dX: Cov variant (as hpc_backward)
    if (dX && h->n > hpc::kTransposeMaxRows) {
        std::snprintf(g_last_error, sizeof g_last_error, "dL/dX transposes X: n <= %lld",
                      (long long)hpc::kTransposeMaxRows);
        return HPC_ERR_ARG;
    }
    return h->vdt == HPC_F64 ? backward_support_t<double>(h, X, xdt, grad_loss, dOmega_vals, dX)
                             : backward_support_t<float>(h, X, xdt, grad_loss, dOmega_vals, dX);
}

int hpc_heldout_loss(hpc_handle h, const void* Xval, hpc_dtype xdt, int64_t nval, double* loss) {
    if (!h || !h->loaded || !Xval || nval < 1 || !valid_dtype(xdt) || !loss) return HPC_ERR_ARG;
    if (nval > hpc::kTransposeMaxRows) {
        std::snprintf(g_last_error, sizeof g_last_error, "hpc_heldout_loss transposes X_val: nval <= %lld",
                      (long long)hpc::kTransposeMaxRows);
        return HPC_ERR_ARG;
    }
    return h->vdt == HPC_F64 ? heldout_t<double>(h, Xval, xdt, nval, loss) : heldout_t<float>(h, Xval, xdt, nval, loss);
}

int hpc_hypergrad(hpc_handle h, const void* Xval, hpc_dtype xdt, int64_t nval, double cg_tol, int64_t cg_max_iter,
                  double* dlambda1, double* dlambda2, hpc_hypergrad_info* info) {
    if (!h || !h->loaded || !Xval || nval < 1 || !valid_dtype(xdt) || !(cg_tol > 0.0) || cg_max_iter < 1 ||
        !dlambda1 || !dlambda2)
        return HPC_ERR_ARG;
    if (!h->S) return HPC_ERR_NOT_IMPLEMENTED;      // needs S (Cov variant)
    if (nval > hpc::kTransposeMaxRows) {
        std::snprintf(g_last_error, sizeof g_last_error, "hpc_hypergrad transposes X_val: nval <= %lld",
                      (long long)hpc::kTransposeMaxRows);
        return HPC_ERR_ARG;
    }
    return h->vdt == HPC_F64 ? hypergrad_t<double>(h, Xval, xdt, nval, cg_tol, cg_max_iter, dlambda1, dlambda2, info)
                             : hypergrad_t<float>(h, Xval, xdt, nval, cg_tol, cg_max_iter, dlambda1, dlambda2, info);
}

int hpc_get_info(hpc_handle h, hpc_info* info) {
    if (!h || !info) return HPC_ERR_ARG;
    std::memset(info, 0, sizeof *info);
    info->n = h->n;
    info->p = h->p;
    info->ld = h->ld;
    info->variant = h->variant;
    info->precision = h->precision;
    info->value_dtype = h->vdt;
    info->capacity = h->cap;
    info->device_bytes = (int64_t)h->held_bytes;
    info->lambda1 = h->lam1;
    info->lambda2 = h->lam2;
    return HPC_OK;
}

int hpc_destroy(hpc_handle h) {
    destroy(h);
    return HPC_OK;
}

int hpc_gram(const void* X, hpc_dtype xdt, int64_t n, int64_t p, void* S, hpc_dtype sdt, int64_t lds,
             int precision, void* cuda_stream) {
    if (!X || !S || n < 1 || p < 1 || lds < p || !valid_dtype(xdt) || (sdt != HPC_F32 && sdt != HPC_F64))
        return HPC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (precision == HPC_PREC_AUTO) precision = sdt == HPC_F64 ? HPC_PREC_FP64 : HPC_PREC_BF16X3;
    if (precision == HPC_PREC_FP64 || precision == HPC_PREC_FP32) {
        if ((precision == HPC_PREC_FP64) != (sdt == HPC_F64)) return HPC_ERR_ARG;
        cudaError_t e = hpc::gram_simt(X, xdt, n, p, S, sdt, lds, s, nullptr);
        if (e != cudaSuccess) { set_cuda_error(e, "gram_simt", __LINE__); return HPC_ERR_CUDA; }
        return HPC_OK;
    }
    if (sdt != HPC_F32 || (precision != HPC_PREC_BF16X3 && precision != HPC_PREC_TF32)) return HPC_ERR_ARG;
    const size_t need = hpc::gram_tc_scratch_bytes(xdt, n, p, precision);
    void* scratch = nullptr;
    if (need) CUDA_TRY(cudaMallocAsync(&scratch, need, s));
    cudaError_t e = hpc::gram_tc(X, xdt, n, p, static_cast<float*>(S), lds, precision, scratch, need, s, nullptr);
    // the launch's error word sits in this call's scratch: read it before the scratch is freed
    const int w = e == cudaSuccess ? hpc::gram_tc_take_error(scratch, xdt, n, p, precision, s) : 0;
    if (scratch) cudaFreeAsync(scratch, s);
    if (e == cudaErrorNotSupported) {
        std::snprintf(g_last_error, sizeof g_last_error, "tensor-core Gram not available for this shape");
        return HPC_ERR_NOT_IMPLEMENTED;
    }
    if (e != cudaSuccess) { set_cuda_error(e, "gram_tc", __LINE__); return HPC_ERR_CUDA; }
    if (w < 0) { set_cuda_error(cudaGetLastError(), "gram_tc error word", __LINE__); return HPC_ERR_CUDA; }
    if (w != 0) {
        std::snprintf(g_last_error, sizeof g_last_error, "tensor-core Gram: bounded wait %d gave up", w);
        return HPC_ERR_DEVICE_TIMEOUT;
    }
    return HPC_OK;
}

}  // extern "C"
