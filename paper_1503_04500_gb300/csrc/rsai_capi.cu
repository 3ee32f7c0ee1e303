// rsai_capi.cu -- host side of the C ABI declared in include/rsai.h.
//
// A handle owns: a device copy of A (CSR + CSC + the CSC->CSR position map),
// the per-column outputs, the result pool, the overflow queues of the size
// bins, M in CSC and CSR, and the CUDA graph of the build sequence.  All device
// memory is taken on the caller's stream, from the allocator installed with
// rsai_set_allocator when the handle was created, else from the library's own
// stream-ordered pool; nothing is allocated by the build sequence itself, so
// rsai_rebuild can replay it as one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace rsai;

namespace {
// A named range on the host timeline of a profiler (NVTX; nothing happens
// unless a tool is attached): the phases of the entry points below.
struct Nvtx {
    explicit Nvtx(const char *name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
    Nvtx(const Nvtx &) = delete;
    Nvtx &operator=(const Nvtx &) = delete;
};
}  // namespace

namespace {
// device memory source: a caller's allocator, or the CUDA stream-ordered one
struct Allocator {
    rsai_alloc_fn alloc = nullptr;
    rsai_free_fn release = nullptr;
    void *ctx = nullptr;
};
Allocator g_allocator;  // process-wide; a handle keeps the one in effect when it was created
}  // namespace

struct rsai_handle {
    int device = 0;
    int sms = 0;
    int64_t n = 0, nnz = 0;
    rsai_params params{};
    // A on the device
    int64_t *row_ptr = nullptr, *col_ptr = nullptr, *csc_to_csr = nullptr;
    int32_t *col_idx = nullptr, *row_idx = nullptr;
    double *val = nullptr, *cval = nullptr;
    float *cval32 = nullptr;  // FP32 copy of cval (FP32_REFINE builds), refreshed by every build
    // 8-byte words: (unused), (unused), frob2, counters, column counts, partial sums
    unsigned long long *dscal = nullptr;
    // blocks (a batch of independent matrices as one block-diagonal matrix)
    int32_t nblocks = 1;
    std::vector<int64_t> cstart_h{0};
    int64_t *d_cstart = nullptr;
    int32_t *col_block = nullptr;     // NULL for one block
    double *norm1_arr = nullptr;      // ||A_b||_1 per block
    double *tau_arr = nullptr;        // tol / ||A_b||_1 per block
    double *bfrob2 = nullptr;         // per-block statistics
    long long *bnc = nullptr, *bnnz = nullptr;
    int32_t *err = nullptr;
    // [0..3] queue counters of bins W, W2, C, G; [4..6] overflow counts W->W2,
    // W2->C, C->G; [7] columns of a pool-overflow rerun; [8] queue counter of
    // bin H, [9] overflow count H->W
    uint32_t *qnext = nullptr;
    int32_t *ovf0 = nullptr, *ovf1 = nullptr, *ovf2 = nullptr, *ovf3 = nullptr;
    int32_t *ovf3_sorted = nullptr;  // the global bin's queue, largest column first
    uint8_t *cost_bucket = nullptr;
    uint32_t *cost_hist = nullptr;   // [kCostBuckets]
    int64_t ovf_cap = 0;
    // per column
    int64_t *col_off = nullptr;
    int32_t *col_len = nullptr, *col_q = nullptr, *loops = nullptr, *flags = nullptr;
    double *rho = nullptr;
    // pool
    int32_t *pool_rows = nullptr;
    double *pool_vals = nullptr;
    int64_t pool_cap = 0;
    unsigned long long *pool_top = nullptr;
    // M
    int64_t *Mcolptr = nullptr, *Mrowptr = nullptr, *Mcsc_to_csr = nullptr, *tsrc = nullptr;
    int32_t *Mrows = nullptr, *Mcols = nullptr, *row_count = nullptr, *cursor = nullptr, *tcols = nullptr;
    double *Mvals_csc = nullptr, *Mvals = nullptr, *tvals = nullptr;
    int64_t *scan_tmp = nullptr;
    int64_t scan_tmp_len = 0;
    // bin G slab
    char *gwork = nullptr;
    size_t gstride = 0;
    int grid_g = 0;
    // bins
    Caps capH{}, capW{}, capW2{}, capC{}, capG{};
    int grid_h = 0, grid_w = 0, grid_w2 = 0, warps_w2 = 0, grid_c = 0;
    rsai_tuning tuning{8, 0, kSmallP, 0, 0};
    // refit / backward scratch (allocated on first use)
    double *fval = nullptr, *fcval = nullptr;
    int64_t *qoff = nullptr, *Mcsr_to_csc = nullptr;
    int32_t *poolI = nullptr;
    double *poolR = nullptr, *poolW = nullptr, *alphaM = nullptr, *xM = nullptr;
    int64_t pool_q_cap = 0, adj_m_cap = 0;
    unsigned long long *fctr = nullptr;  // work counters of refit / backward passes
    // graph
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    // host copy of the last statistics
    std::vector<std::pair<void *, size_t>> allocs;
    Allocator allocator;
    cudaStream_t alloc_stream = nullptr;
};

namespace {

// layout of the scalar block (8-byte words); words 0 and 1 are unused since
// ||A||_1 and the drop threshold moved to per-block arrays
constexpr int kFrob2 = 2, kCtr = 3;
constexpr int kCounts = kCtr + CTR_COUNT + kBinSlots;
constexpr int kPartial = kCounts + 2;
constexpr int kScalars = kPartial + kStatBlocks;

double *dword(const rsai_handle *h, int at) { return reinterpret_cast<double *>(h->dscal + at); }

// a failed allocation inside a launch sequence (the global bin's slab) comes
// back as cudaErrorMemoryAllocation: it is an OOM, not a CUDA fault
int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RSAI_OK;
    return e == cudaErrorMemoryAllocation ? RSAI_ERR_OOM : RSAI_ERR_CUDA;
}

// The library's own stream-ordered pool on the current device.  Up to
// kPoolKeep bytes that handles give back stay mapped in it, so that building
// and freeing handles repeatedly does not map and unmap device memory each
// time; the application's default pool is left as it is.
constexpr uint64_t kPoolKeep = 2ull << 30;

cudaMemPool_t library_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = kPoolKeep;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

void *raw_alloc(const Allocator &a, size_t bytes, cudaStream_t st) {
    void *p = nullptr;
    if (a.alloc) return a.alloc(bytes, (void *)st, a.ctx);
    cudaMemPool_t pool = library_pool();
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void raw_free(const Allocator &a, void *p, size_t bytes, cudaStream_t st) {
    if (!p) return;
    if (a.release) a.release(p, bytes, (void *)st, a.ctx);
    else cudaFreeAsync(p, st);
}

template <typename P> int dalloc(rsai_handle *h, P **ptr, size_t count, cudaStream_t st) {
    size_t bytes = sizeof(P) * (count ? count : 1);
    void *p = raw_alloc(h->allocator, bytes, st);
    if (!p) return RSAI_ERR_OOM;
    h->allocs.push_back({p, bytes});
    *ptr = (P *)p;
    return RSAI_OK;
}

// frees one buffer taken by dalloc (stream-ordered on st)
void dfree(rsai_handle *h, void *p, cudaStream_t st) {
    for (size_t i = 0; i < h->allocs.size(); ++i) {
        if (h->allocs[i].first == p) {
            raw_free(h->allocator, p, h->allocs[i].second, st);
            h->allocs.erase(h->allocs.begin() + i);
            return;
        }
    }
}

// copy host or device memory into a device buffer
cudaError_t to_device(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
}

DevA dev_a(const rsai_handle *h) {
    return DevA{h->n, h->row_ptr, h->col_idx, h->val, h->col_ptr, h->row_idx, h->cval, h->cval32};
}

DevParams dev_params(const rsai_handle *h) {
    DevParams P;
    P.c = h->params.c;
    P.l_max = h->params.l_max;
    P.drop_mode = h->params.drop_mode;
    P.precision = h->params.precision;
    P.init_a = (h->params.flags & RSAI_FLAG_INIT_PATTERN_A) ? 1 : 0;
    P.spai = (h->params.flags & RSAI_FLAG_SELECT_SPAI) ? 1 : 0;
    P.eps = h->params.eps;
    P.tol = h->params.tol;
    P.tie_band = h->params.tie_band;
    P.norm1 = h->norm1_arr;
    P.tau_fixed = h->tau_arr;
    P.col_block = h->col_block;
    return P;
}

unsigned blocks(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

cudaError_t scan_counts(rsai_handle *h, const int32_t *in, int64_t *out, cudaStream_t st) {
    int64_t nb = (h->n + 1023) / 1024;
    if (nb < 1) nb = 1;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, st>>>(in, h->n, out, h->scan_tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(h->scan_tmp, nb, h->scan_tmp + h->scan_tmp_len - 1);
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, h->n, h->scan_tmp, h->scan_tmp + h->scan_tmp_len - 1);
    return cudaGetLastError();
}

// The three bins over all columns (mode: build, refit or backward); queue
// counters are reset first.  `ev` (optional) brackets the bins (ev[1..4]).
// `before_global` (optional, host side): called between bins C and G, e.g. to
// size the global-bin slab from the number of columns that reached it.
typedef int (*BinHook)(rsai_handle *h, cudaStream_t st);

cudaError_t enqueue_bins(rsai_handle *h, int mode, const DevA &A, const Frozen &F, unsigned long long *gctr,
                         cudaStream_t st, cudaEvent_t *ev = nullptr, BinHook before_global = nullptr,
                         const int32_t *wlist = nullptr, const uint32_t *wcount = nullptr) {
    const int64_t n = h->n;
    cudaMemsetAsync(h->qnext, 0, sizeof(uint32_t) * 7, st);  // queue and overflow counters; [7] = retry count
    cudaMemsetAsync(h->qnext + 8, 0, sizeof(uint32_t) * 2, st);
    const DevParams P = dev_params(h);
    const bool fp32 = h->params.precision == RSAI_FP32_REFINE;
    ColOut O{h->col_off, h->col_len, h->col_q, h->rho, h->loops, h->flags, h->pool_rows, h->pool_vals,
             h->pool_cap, h->pool_top, h->err};
    // the first bin (H or W) takes the given list (or every column)
    const bool use_h = h->tuning.half_bin != 0;
    ColQueue QH{wlist, wcount, n, h->qnext + 8, h->ovf0, h->qnext + 9, h->ovf_cap};
    ColQueue QW = use_h ? ColQueue{h->ovf0, h->qnext + 9, n, h->qnext + 0, h->ovf1, h->qnext + 4, h->ovf_cap}
                        : ColQueue{wlist, wcount, n, h->qnext + 0, h->ovf1, h->qnext + 4, h->ovf_cap};
    ColQueue QW2{h->ovf1, h->qnext + 4, n, h->qnext + 1, h->ovf2, h->qnext + 5, h->ovf_cap};
    ColQueue QC{h->ovf2, h->qnext + 5, n, h->qnext + 2, h->ovf3, h->qnext + 6, h->ovf_cap};
    ColQueue QG{h->ovf3_sorted, h->qnext + 6, n, h->qnext + 3, nullptr, nullptr, 0};
    if (ev) cudaEventRecord(ev[1], st);
    cudaError_t e = cudaSuccess;
    if (use_h) {
        e = launch_bin_half(mode, fp32, h->grid_h, h->tuning.warp_bin_warps, A, P, h->capH, QH, O, F, gctr, false, st);
        if (e != cudaSuccess) return e;
    }
    e = launch_bin_warp(mode, fp32, h->grid_w, h->tuning.warp_bin_warps, A, P, h->capW, QW, O, F, gctr, false, st);
    if (e != cudaSuccess) return e;
    e = launch_bin_warp(mode, fp32, h->grid_w2, h->warps_w2, A, P, h->capW2, QW2, O, F, gctr, false, st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], st);
    e = launch_bin_block(mode, fp32, h->grid_c, A, P, h->capC, QC, O, F, gctr, false, nullptr, 0, 1, st);
    if (e != cudaSuccess) return e;
    if (before_global) {
        const int hr = before_global(h, st);
        if (hr != RSAI_OK) return hr == RSAI_ERR_OOM ? cudaErrorMemoryAllocation : cudaErrorUnknown;
    }
    // the columns that reached the global bin, largest first (grids cover n;
    // the device-side count bounds the work)
    cudaMemsetAsync(h->cost_hist, 0, sizeof(uint32_t) * kCostBuckets, st);
    k_cost_buckets<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(h->ovf3, h->qnext + 6, A.col_ptr, A.row_idx,
                                                                 A.row_ptr, h->cost_bucket, h->cost_hist);
    k_cost_offsets<<<1, 32, 0, st>>>(h->cost_hist);
    k_cost_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(h->ovf3, h->qnext + 6, h->cost_bucket, h->cost_hist,
                                                                 h->ovf3_sorted);
    if (ev) cudaEventRecord(ev[3], st);
    e = launch_bin_block(mode, fp32, h->grid_g, A, P, h->capG, QG, O, F, gctr, true, h->gwork, h->gstride, 2, st);
    return e;
}

// The build sequence: no allocation, no host synchronisation (capturable).
// `ev` (optional, RSAI_PHASE_COUNT + 1 events) are recorded between phases.
cudaError_t enqueue_build_tail(rsai_handle *h, cudaStream_t st, cudaEvent_t *ev);

cudaError_t enqueue_build(rsai_handle *h, cudaStream_t st, cudaEvent_t *ev = nullptr, BinHook hook = nullptr) {
    const int64_t n = h->n;
    if (ev) cudaEventRecord(ev[0], st);
    cudaMemsetAsync(h->dscal, 0, sizeof(unsigned long long) * kScalars, st);
    cudaMemsetAsync(h->err, 0, sizeof(int32_t), st);
    cudaMemsetAsync(h->qnext, 0, sizeof(uint32_t) * 10, st);
    cudaMemsetAsync(h->pool_top, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(h->row_count, 0, sizeof(int32_t) * (size_t)n, st);
    cudaMemsetAsync(h->cursor, 0, sizeof(int32_t) * (size_t)n, st);
    cudaMemsetAsync(h->norm1_arr, 0, sizeof(double) * (size_t)h->nblocks, st);
    k_norm1<<<blocks(n, 256), 256, 0, st>>>(h->col_ptr, h->cval, n, h->col_block, h->norm1_arr);
    if (h->cval32) k_to_f32<<<blocks(h->nnz, 256), 256, 0, st>>>(h->cval, h->cval32, h->nnz);
    k_tau_fixed<<<blocks(h->nblocks, 256), 256, 0, st>>>(h->norm1_arr, h->params.tol, h->tau_arr, h->nblocks);

    cudaError_t e = enqueue_bins(h, MODE_BUILD, dev_a(h), Frozen{}, h->dscal + kCtr, st, ev, hook);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[4], st);
    return enqueue_build_tail(h, st, ev);
}

// statistics and the assembly of M (the end of the build sequence)
cudaError_t enqueue_build_tail(rsai_handle *h, cudaStream_t st, cudaEvent_t *ev) {
    const int64_t n = h->n;
    cudaError_t e;
    cudaMemsetAsync(h->dscal + kCounts, 0, sizeof(unsigned long long) * 2, st);  // n_c, nnz(M): accumulated
    k_column_stats<<<kStatBlocks, 256, 0, st>>>(h->rho, h->flags, h->col_len, n, h->params.eps,
                                                dword(h, kPartial), h->dscal + kCounts);
    k_column_stats_final<<<1, kStatBlocks, 0, st>>>(dword(h, kPartial), dword(h, kFrob2));
    // M in CSC, then CSR with rows sorted by column index
    e = scan_counts(h, h->col_len, h->Mcolptr, st);
    if (e != cudaSuccess) return e;
    k_pool_to_csc<<<blocks(n * 32, 256), 256, 0, st>>>(h->col_off, h->col_len, h->pool_rows, h->pool_vals,
                                                       h->Mcolptr, h->Mrows, h->Mvals_csc, h->row_count, n);
    e = scan_counts(h, h->row_count, h->Mrowptr, st);
    if (e != cudaSuccess) return e;
    k_csc_to_rows<<<blocks(n * 32, 256), 256, 0, st>>>(h->Mcolptr, h->Mrows, h->Mvals_csc, h->Mrowptr, h->cursor,
                                                       h->tcols, h->tvals, h->tsrc, n);
    k_sort_rows<<<blocks(n * 32, 256), 256, 0, st>>>(h->Mrowptr, h->tcols, h->tvals, h->tsrc, h->Mcols, h->Mvals,
                                                     h->Mcsc_to_csr, n);
    if (ev) cudaEventRecord(ev[5], st);
    return cudaGetLastError();
}

void free_all(rsai_handle *h) {
    if (!h) return;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    // the caller's stream may be gone by now: wait for the handle's device,
    // then free there (the current device is restored)
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto &a : h->allocs) {
        if (h->allocator.release) h->allocator.release(a.first, a.second, nullptr, h->allocator.ctx);
        else cudaFreeAsync(a.first, nullptr);  // the device is idle: returned to the pool at once
    }
    h->allocs.clear();
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
}

int check_csr_host(const rsai_csr *A) {
    if (!A || !A->row_ptr || !A->col_idx || !A->val) return RSAI_ERR_INVALID_ARG;
    if (A->n <= 0 || A->nnz < 0 || A->n > INT32_MAX) return RSAI_ERR_SHAPE;
    return RSAI_OK;
}

// launch shape of bin W2: the warps per CTA of the warp bin, halved until its
// larger workspace fits
int plan_w2(rsai_handle *h, bool fp32) {
    int w = h->tuning.warp_bin_warps, occ = 0;
    while ((occ = occupancy_bin_warp(fp32, w, h->capW2)) < 1 && w > 1) w /= 2;
    if (occ < 1) return RSAI_ERR_CUDA;
    h->warps_w2 = w;
    h->grid_w2 = h->sms * occ;
    return RSAI_OK;
}

// launch shape of bin H: the warps per CTA of the warp bin (two columns per
// warp), as many CTAs per SM as fit
int plan_h(rsai_handle *h, bool fp32) {
    const int occ0 = occupancy_bin_half(fp32, h->tuning.warp_bin_warps, h->capH);
    if (occ0 < 1) return RSAI_ERR_CUDA;
    const int occ = h->tuning.warp_bin_ctas_per_sm > 0 ? std::min(occ0, h->tuning.warp_bin_ctas_per_sm) : occ0;
    h->grid_h = h->sms * occ;
    return RSAI_OK;
}

#define TRY_PLAN(x)                        \
    do {                                   \
        const int rc_ = (x);               \
        if (rc_ != RSAI_OK) return rc_;    \
    } while (0)

// choose the capacities of the five bins from the device limits
int plan_bins(rsai_handle *h) {
    const bool fp32 = h->params.precision == RSAI_FP32_REFINE;
    int dev = h->device, max_optin = 0;
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int rneed = std::max(64, h->params.c * std::max(1, h->params.l_max));
    // bin H: half a warp per column, |I| <= 48, |J| <= 16 (the register QR's
    // three rows per lane), sort buffers of 128 entries
    const int spai = (h->params.flags & RSAI_FLAG_SELECT_SPAI) ? 1 : 0;
    h->capH = Caps{48, 16, 128, 32, 48 * 16, 32, h->tuning.small_qr_max_p, 0, 0, 32, spai};
    int occ = 0;
    TRY_PLAN(plan_h(h, fp32));
    h->capW = Caps{64, 32, 256, 64, 64 * 32, 64, h->tuning.small_qr_max_p, 0, 0, 64, spai};
    occ = occupancy_bin_warp(fp32, h->tuning.warp_bin_warps, h->capW);
    if (occ < 1) return RSAI_ERR_CUDA;
    if (h->tuning.warp_bin_ctas_per_sm > 0) occ = std::min(occ, h->tuning.warp_bin_ctas_per_sm);
    h->grid_w = h->sms * occ;
    // bin W2: the warp bin's algorithm for |I| <= 128 (B 128 x 32), fewer warps per SM
    h->capW2 = Caps{128, 32, 512, 64, 128 * 32, 64, h->tuning.small_qr_max_p, 0, 0, 128, spai};
    if (plan_w2(h, fp32) != RSAI_OK) return RSAI_ERR_CUDA;
    // bin C: shared-memory workspace as large as the opt-in limit allows
    Caps c{1024, 256, 4096, std::min(rneed * 2, 2048), 0, 0, 0, 0, 1, 1024, spai};
    size_t base = fp32 ? work_bytes<float>(c) : work_bytes<double>(c);
    size_t avail = (size_t)max_optin - 2048;
    if (base >= avail) return RSAI_ERR_CUDA;
    c.bcap = (int64_t)((avail - base) / (fp32 ? sizeof(float) : sizeof(double))) - 64;
    h->capC = c;
    occ = occupancy_bin_block(fp32, h->capC, false);
    if (occ < 1) return RSAI_ERR_CUDA;
    h->grid_c = h->sms * occ;
    // bin G: a global-memory slab per CTA, one CTA per SM
    h->capG = Caps{32768, 4096, 131072, 8192, (int64_t)1 << 24, 0, 0, max_optin - 2048, 1, 32768, spai};
    h->gstride = ((fp32 ? work_bytes<float>(h->capG) : work_bytes<double>(h->capG)) + 255) & ~size_t(255);
    h->grid_g = 1;  // sized by the first build (size_global_slab)
    return RSAI_OK;
}

}  // namespace

extern "C" {

int32_t rsai_abi_version(void) { return RSAI_ABI_VERSION; }

const char *rsai_status_string(rsai_status s) {
    switch (s) {
        case RSAI_OK: return "ok";
        case RSAI_ERR_INVALID_ARG: return "invalid argument";
        case RSAI_ERR_SHAPE: return "inconsistent shape (n, nnz, or CSR/CSC mismatch)";
        case RSAI_ERR_UNSORTED: return "indices not strictly ascending within a row/column";
        case RSAI_ERR_INDEX_RANGE: return "index or pointer out of range";
        case RSAI_ERR_EMPTY_COLUMN: return "a column of A has no nonzeros (A is singular)";
        case RSAI_ERR_OOM: return "device allocation failed";
        case RSAI_ERR_CUDA: return "CUDA runtime error";
        case RSAI_ERR_TIMEOUT: return "a bounded device wait ran out";
        case RSAI_ERR_WORKSPACE: return "a column outgrew every size bin or the result pool";
        case RSAI_ERR_BREAKDOWN: return "BiCGStab breakdown";
        case RSAI_ERR_NOT_CONVERGED: return "BiCGStab did not converge within maxit";
        case RSAI_ERR_NO_DEVICE: return "no CUDA device";
        case RSAI_ERR_TOO_LARGE: return "problem larger than the fixed-size workspace of this entry point";
    }
    return "unknown status";
}

rsai_status rsai_params_default(rsai_params *p) {
    if (!p) return RSAI_ERR_INVALID_ARG;
    p->c = 3;
    p->l_max = 10;
    p->eps = 0.3;
    p->drop_mode = RSAI_DROP_FIXED;
    p->tol = 1e-3;
    p->precision = RSAI_FP64;
    p->tie_band = 1e-12;
    p->flags = 0;
    return RSAI_OK;
}

rsai_status rsai_params_check(const rsai_params *p) {
    if (!p) return RSAI_ERR_INVALID_ARG;
    if (p->c < 1 || p->c > 32) return RSAI_ERR_INVALID_ARG;
    if (p->l_max < 0 || p->l_max > 100000) return RSAI_ERR_INVALID_ARG;
    if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return RSAI_ERR_INVALID_ARG;
    if (p->drop_mode < RSAI_DROP_NONE || p->drop_mode > RSAI_DROP_FIXED) return RSAI_ERR_INVALID_ARG;
    if (!(p->tol >= 0.0) || !std::isfinite(p->tol)) return RSAI_ERR_INVALID_ARG;
    if (p->precision != RSAI_FP64 && p->precision != RSAI_FP32_REFINE) return RSAI_ERR_INVALID_ARG;
    if (!(p->tie_band >= 0.0) || !(p->tie_band < 1.0)) return RSAI_ERR_INVALID_ARG;
    if (p->flags & ~(uint32_t)(RSAI_FLAG_INIT_PATTERN_A | RSAI_FLAG_SELECT_SPAI)) return RSAI_ERR_INVALID_ARG;
    return RSAI_OK;
}

void rsai_handle_free(rsai_handle *h) {
    if (!h) return;
    free_all(h);
    delete h;
}

}  // extern "C"

namespace {

// One CTA of the global bin per column that reached it, up to one per SM: the
// slab (a few tens of MB per CTA) is sized by the first build only.
int size_global_slab(rsai_handle *h, cudaStream_t st) {
    uint32_t cnt = 0;
    if (cudaMemcpyAsync(&cnt, h->qnext + 6, sizeof(cnt), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RSAI_ERR_CUDA;
    int want = std::max(1, std::min(h->sms, (int)cnt));
    if (h->tuning.global_bin_ctas > 0) want = std::min(h->tuning.global_bin_ctas, h->sms);
    if (want <= h->grid_g) return RSAI_OK;
    // the larger slab first, so that a failed allocation leaves the old one in place
    char *slab = nullptr;
    const int rc = dalloc(h, &slab, h->gstride * (size_t)want, st);
    if (rc != RSAI_OK) return rc;
    if (h->gwork) dfree(h, h->gwork, st);
    h->gwork = slab;
    h->grid_g = want;
    return RSAI_OK;
}

// Everything after A (CSR, CSC, csc_to_csr space) and the block arrays are in
// the handle: input checks, bins, buffers, the first build.  Returns OK or
// WORKSPACE with a usable handle; any other status means failure.
int build_common(rsai_handle *h, cudaStream_t st) {
    const int64_t n = h->n, nnz = h->nnz;
    int rc = RSAI_OK;
#define TRY(x)                        \
    do {                              \
        rc = (x);                     \
        if (rc != RSAI_OK) return rc; \
    } while (0)
    TRY(dalloc(h, &h->dscal, kScalars, st));
    TRY(dalloc(h, &h->err, 1, st));
    TRY(dalloc(h, &h->norm1_arr, h->nblocks, st));
    TRY(dalloc(h, &h->tau_arr, h->nblocks, st));
    // ---- validation of A (device kernels, error codes) ----
    // One pass on the stream, one read of the first error: each check after
    // the pointer checks returns at once if an earlier one set the error word,
    // so it never follows an index that was not checked.
    {
        Nvtx range("rsai: check A");
        int32_t herr = 0;
        cudaMemsetAsync(h->err, 0, sizeof(int32_t), st);
        k_check_ptr<<<blocks(n + 1, 256), 256, 0, st>>>(h->row_ptr, n, nnz, h->err);
        k_check_ptr<<<blocks(n + 1, 256), 256, 0, st>>>(h->col_ptr, n, nnz, h->err);
        k_check_idx<<<blocks(n, 256), 256, 0, st>>>(h->row_ptr, h->col_idx, n, h->err, 0);
        k_check_idx<<<blocks(n, 256), 256, 0, st>>>(h->col_ptr, h->row_idx, n, h->err, 1);
        k_csc_map<<<blocks(n, 256), 256, 0, st>>>(dev_a(h), h->csc_to_csr, h->err);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&herr, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RSAI_ERR_CUDA;
        TRY(herr);
    }
    {
        Nvtx range("rsai: plan bins");
        TRY(plan_bins(h));
    }
    if (h->params.precision == RSAI_FP32_REFINE) TRY(dalloc(h, &h->cval32, nnz, st));
    // ---- buffers of the build sequence ----
    h->ovf_cap = n;
    TRY(dalloc(h, &h->qnext, 10, st));
    TRY(dalloc(h, &h->ovf0, n, st));
    TRY(dalloc(h, &h->ovf1, n, st));
    TRY(dalloc(h, &h->ovf2, n, st));
    TRY(dalloc(h, &h->ovf3, n, st));
    TRY(dalloc(h, &h->ovf3_sorted, n, st));
    TRY(dalloc(h, &h->cost_bucket, n, st));
    TRY(dalloc(h, &h->cost_hist, kCostBuckets, st));
    TRY(dalloc(h, &h->col_off, n, st));
    TRY(dalloc(h, &h->col_len, n, st));
    TRY(dalloc(h, &h->col_q, n, st));
    TRY(dalloc(h, &h->loops, n, st));
    TRY(dalloc(h, &h->flags, n, st));
    TRY(dalloc(h, &h->rho, n, st));
    TRY(dalloc(h, &h->pool_top, 1, st));
    TRY(dalloc(h, &h->Mcolptr, n + 1, st));
    TRY(dalloc(h, &h->Mrowptr, n + 1, st));
    TRY(dalloc(h, &h->row_count, n, st));
    TRY(dalloc(h, &h->cursor, n, st));
    h->scan_tmp_len = (n + 1023) / 1024 + 2;
    TRY(dalloc(h, &h->scan_tmp, h->scan_tmp_len, st));
    TRY(dalloc(h, &h->gwork, h->gstride * (size_t)h->grid_g, st));
    int status = RSAI_OK;
    {
        Nvtx range("rsai: first build");
        // result pool: if columns find it full, it grows (keeping what was
        // written) and only those columns run again
        // 10 entries per nonzero of an average column of A, plus 16: above
        // the nnz(M)/n of the configurations (15.5 on the 64^3 problem, 78 on
        // the n = 1e6 power law, where 6 per nonzero made part of the first
        // build run twice)
        const int64_t g_est = std::max<int64_t>(32, 10 * (nnz / std::max<int64_t>(1, n)) + 16);
        int64_t cap = std::min<int64_t>(n * g_est, n * n);
        h->pool_cap = cap;
        TRY(dalloc(h, &h->pool_rows, cap, st));
        TRY(dalloc(h, &h->pool_vals, cap, st));
        auto alloc_m = [&](int64_t c) -> int {
            int r = dalloc(h, &h->Mrows, c, st);
            if (r == RSAI_OK) r = dalloc(h, &h->Mvals_csc, c, st);
            if (r == RSAI_OK) r = dalloc(h, &h->Mcols, c, st);
            if (r == RSAI_OK) r = dalloc(h, &h->Mvals, c, st);
            if (r == RSAI_OK) r = dalloc(h, &h->tcols, c, st);
            if (r == RSAI_OK) r = dalloc(h, &h->tvals, c, st);
            if (r == RSAI_OK) r = dalloc(h, &h->tsrc, c, st);
            if (r == RSAI_OK) r = dalloc(h, &h->Mcsc_to_csr, c, st);
            return r;
        };
        auto release = [&](void *p) { dfree(h, p, st); };
        TRY(alloc_m(cap));
        TRY(cuda_status(enqueue_build(h, st, nullptr, size_global_slab)));
        int32_t *retry = nullptr;
        constexpr int kMaxRegrow = 6;
        bool settled = false;
        for (int attempt = 0; attempt <= kMaxRegrow; ++attempt) {
            unsigned long long top = 0;
            int32_t herr = 0;
            cudaMemcpyAsync(&top, h->pool_top, sizeof(top), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(&herr, h->err, sizeof(herr), cudaMemcpyDeviceToHost, st);
            TRY(cuda_status(cudaStreamSynchronize(st)));
            if ((int64_t)top <= h->pool_cap) {
                if (herr != 0) status = herr;
                settled = true;
                break;
            }
            if (attempt == kMaxRegrow) break;  // the last rerun still found the pool full
            // grow the pool (copying what fits), M's buffers with it
            const int64_t old_cap = h->pool_cap;
            // new reservations start at `top`; the columns to redo need at most `top`
            cap = std::min<int64_t>((int64_t)(2 * top + 1024), std::max<int64_t>(n * n, (int64_t)top + 1024));
            int32_t *nrows = nullptr;
            double *nvals = nullptr;
            TRY(dalloc(h, &nrows, cap, st));
            TRY(dalloc(h, &nvals, cap, st));
            cudaMemcpyAsync(nrows, h->pool_rows, sizeof(int32_t) * old_cap, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(nvals, h->pool_vals, sizeof(double) * old_cap, cudaMemcpyDeviceToDevice, st);
            void *old_bufs[] = {h->pool_rows, h->pool_vals, h->Mrows, h->Mvals_csc, h->Mcols,
                                h->Mvals, h->tcols, h->tvals, h->tsrc, h->Mcsc_to_csr};
            for (void *p : old_bufs) release(p);
            h->pool_rows = nrows;
            h->pool_vals = nvals;
            h->pool_cap = cap;
            TRY(alloc_m(cap));
            // the columns that found the pool full run again (from its current top)
            if (!retry) TRY(dalloc(h, &retry, n, st));
            cudaMemsetAsync(h->qnext + 7, 0, sizeof(uint32_t), st);
            k_collect_failed<<<blocks(n, 256), 256, 0, st>>>(h->flags, n, retry, h->qnext + 7);
            cudaMemsetAsync(h->dscal + kCtr + CTR_FAILED, 0, sizeof(unsigned long long), st);
            cudaMemsetAsync(h->err, 0, sizeof(int32_t), st);
            cudaMemsetAsync(h->row_count, 0, sizeof(int32_t) * (size_t)n, st);
            cudaMemsetAsync(h->cursor, 0, sizeof(int32_t) * (size_t)n, st);
            TRY(cuda_status(enqueue_bins(h, MODE_BUILD, dev_a(h), Frozen{}, h->dscal + kCtr, st, nullptr,
                                         size_global_slab, retry, h->qnext + 7)));
            TRY(cuda_status(enqueue_build_tail(h, st, nullptr)));
        }
        // columns still without room in the pool are flagged and counted as failed
        if (!settled) status = RSAI_ERR_WORKSPACE;
    }
#undef TRY
    return status;
}

rsai_handle *new_handle(const rsai_params *params, cudaStream_t st) {
    rsai_handle *h = new (std::nothrow) rsai_handle();
    if (!h) return nullptr;
    h->alloc_stream = st;
    h->allocator = g_allocator;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    h->params = *params;
    // the shapes the autotuner picks on the 64^3 convection-diffusion problem:
    // FP64 builds start in the half-warp bin with the register QR up to
    // |J| = 8, FP32+refine builds in the warp bin with the register QR up to 16
    if (params->precision == RSAI_FP64) {
        h->tuning.half_bin = 1;
        h->tuning.small_qr_max_p = 8;
    }
    return h;
}

int have_device() {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return 0;
    }
    return 1;
}

}  // namespace

extern "C" {

rsai_status rsai_build(const rsai_csr *A, const rsai_csc *Acsc, const rsai_params *params, void *stream,
                       rsai_handle **out) {
    Nvtx range("rsai_build");
    if (!out) return RSAI_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = rsai_params_check(params);
    if (rc != RSAI_OK) return (rsai_status)rc;
    rc = check_csr_host(A);
    if (rc != RSAI_OK) return (rsai_status)rc;
    if (!Acsc || !Acsc->col_ptr || !Acsc->row_idx || !Acsc->val) return RSAI_ERR_INVALID_ARG;
    if (Acsc->n != A->n || Acsc->nnz != A->nnz) return RSAI_ERR_SHAPE;
    if (!have_device()) return RSAI_ERR_NO_DEVICE;
    cudaStream_t st = (cudaStream_t)stream;
    rsai_handle *h = new_handle(params, st);
    if (!h) return RSAI_ERR_OOM;
    h->n = A->n;
    h->nnz = A->nnz;
    const int64_t n = h->n, nnz = h->nnz;
    h->cstart_h = {0, n};
    rc = dalloc(h, &h->row_ptr, n + 1, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->col_ptr, n + 1, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->col_idx, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->row_idx, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->val, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->cval, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->csc_to_csr, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->d_cstart, 2, st);
    if (rc == RSAI_OK) {
        bool ok = to_device(h->row_ptr, A->row_ptr, sizeof(int64_t) * (n + 1), st) == cudaSuccess &&
                  to_device(h->col_idx, A->col_idx, sizeof(int32_t) * nnz, st) == cudaSuccess &&
                  to_device(h->val, A->val, sizeof(double) * nnz, st) == cudaSuccess &&
                  to_device(h->col_ptr, Acsc->col_ptr, sizeof(int64_t) * (n + 1), st) == cudaSuccess &&
                  to_device(h->row_idx, Acsc->row_idx, sizeof(int32_t) * nnz, st) == cudaSuccess &&
                  to_device(h->cval, Acsc->val, sizeof(double) * nnz, st) == cudaSuccess &&
                  cudaMemcpyAsync(h->d_cstart, h->cstart_h.data(), sizeof(int64_t) * 2, cudaMemcpyHostToDevice,
                                  st) == cudaSuccess;
        if (!ok) rc = RSAI_ERR_CUDA;
    }
    if (rc == RSAI_OK) rc = build_common(h, st);
    if (rc != RSAI_OK && rc != RSAI_ERR_WORKSPACE) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        rsai_handle_free(h);
        return (rsai_status)rc;
    }
    *out = h;
    return (rsai_status)rc;
}

rsai_status rsai_build_batch(const rsai_csr *As, const rsai_csc *Acscs, int32_t count, const rsai_params *params,
                             void *stream, rsai_handle **out) {
    Nvtx range("rsai_build_batch");
    if (!out) return RSAI_ERR_INVALID_ARG;
    *out = nullptr;
    if (!As || !Acscs || count < 1) return RSAI_ERR_INVALID_ARG;
    int rc = rsai_params_check(params);
    if (rc != RSAI_OK) return (rsai_status)rc;
    std::vector<int64_t> cstart(count + 1, 0), estart(count + 1, 0);
    for (int b = 0; b < count; ++b) {
        rc = check_csr_host(&As[b]);
        if (rc != RSAI_OK) return (rsai_status)rc;
        const rsai_csc &C = Acscs[b];
        if (!C.col_ptr || !C.row_idx || !C.val) return RSAI_ERR_INVALID_ARG;
        if (C.n != As[b].n || C.nnz != As[b].nnz) return RSAI_ERR_SHAPE;
        cstart[b + 1] = cstart[b] + As[b].n;
        estart[b + 1] = estart[b] + As[b].nnz;
    }
    if (cstart[count] > INT32_MAX) return RSAI_ERR_SHAPE;
    if (!have_device()) return RSAI_ERR_NO_DEVICE;
    cudaStream_t st = (cudaStream_t)stream;
    rsai_handle *h = new_handle(params, st);
    if (!h) return RSAI_ERR_OOM;
    const int64_t n = cstart[count], nnz = estart[count];
    h->n = n;
    h->nnz = nnz;
    h->nblocks = count;
    h->cstart_h = cstart;
    int64_t *d_estart = nullptr;
    rc = dalloc(h, &h->row_ptr, n + 1, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->col_ptr, n + 1, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->col_idx, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->row_idx, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->val, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->cval, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->csc_to_csr, nnz, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->d_cstart, count + 1, st);
    if (rc == RSAI_OK) rc = dalloc(h, &d_estart, count + 1, st);
    if (rc == RSAI_OK) rc = dalloc(h, &h->col_block, n, st);
    for (int b = 0; rc == RSAI_OK && b < count; ++b) {
        const rsai_csr &R = As[b];
        const rsai_csc &C = Acscs[b];
        const int64_t c0 = cstart[b], e0 = estart[b];
        bool ok = to_device(h->row_ptr + c0, R.row_ptr, sizeof(int64_t) * R.n, st) == cudaSuccess &&
                  to_device(h->col_idx + e0, R.col_idx, sizeof(int32_t) * R.nnz, st) == cudaSuccess &&
                  to_device(h->val + e0, R.val, sizeof(double) * R.nnz, st) == cudaSuccess &&
                  to_device(h->col_ptr + c0, C.col_ptr, sizeof(int64_t) * C.n, st) == cudaSuccess &&
                  to_device(h->row_idx + e0, C.row_idx, sizeof(int32_t) * C.nnz, st) == cudaSuccess &&
                  to_device(h->cval + e0, C.val, sizeof(double) * C.nnz, st) == cudaSuccess;
        if (!ok) rc = RSAI_ERR_CUDA;
    }
    if (rc == RSAI_OK) {
        cudaMemcpyAsync(h->d_cstart, cstart.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_estart, estart.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st);
        k_col_block<<<blocks(n, 256), 256, 0, st>>>(h->d_cstart, count, n, h->col_block);
        k_shift_ptr<<<blocks(n + 1, 256), 256, 0, st>>>(h->row_ptr, n, h->col_block, d_estart, nnz);
        k_shift_ptr<<<blocks(n + 1, 256), 256, 0, st>>>(h->col_ptr, n, h->col_block, d_estart, nnz);
        k_shift_idx<<<blocks(n, 256), 256, 0, st>>>(h->row_ptr, h->col_idx, n, h->col_block, h->d_cstart);
        k_shift_idx<<<blocks(n, 256), 256, 0, st>>>(h->col_ptr, h->row_idx, n, h->col_block, h->d_cstart);
        if (cudaGetLastError() != cudaSuccess) rc = RSAI_ERR_CUDA;
    }
    if (rc == RSAI_OK) rc = build_common(h, st);
    if (rc != RSAI_OK && rc != RSAI_ERR_WORKSPACE) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        rsai_handle_free(h);
        return (rsai_status)rc;
    }
    *out = h;
    return (rsai_status)rc;
}

rsai_status rsai_get_block_stats(rsai_handle *h, void *stream, double *frob, int64_t *n_c, int64_t *nnz_M) {
    if (!h) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = h->nblocks;
    if (!h->bfrob2) {
        int rc = dalloc(h, &h->bfrob2, nb, st);
        if (rc == RSAI_OK) rc = dalloc(h, &h->bnc, nb, st);
        if (rc == RSAI_OK) rc = dalloc(h, &h->bnnz, nb, st);
        if (rc != RSAI_OK) return (rsai_status)rc;
    }
    k_block_stats<<<nb, 256, 0, st>>>(h->d_cstart, h->rho, h->flags, h->col_len, h->params.eps, h->bfrob2, h->bnc,
                                     h->bnnz);
    std::vector<double> f2(nb);
    std::vector<long long> c(nb), z(nb);
    cudaMemcpyAsync(f2.data(), h->bfrob2, sizeof(double) * nb, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(c.data(), h->bnc, sizeof(long long) * nb, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(z.data(), h->bnnz, sizeof(long long) * nb, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    for (int b = 0; b < nb; ++b) {
        if (frob) frob[b] = std::sqrt(f2[b]);
        if (n_c) n_c[b] = c[b];
        if (nnz_M) nnz_M[b] = z[b];
    }
    return RSAI_OK;
}

rsai_status rsai_set_values(rsai_handle *h, const double *A_val, void *stream) {
    if (!h || !A_val) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (to_device(h->val, A_val, sizeof(double) * h->nnz, st) != cudaSuccess) return RSAI_ERR_CUDA;
    k_csc_from_csr<<<blocks(h->nnz, 256), 256, 0, st>>>(h->val, h->csc_to_csr, h->cval, h->nnz);
    return (rsai_status)cuda_status(cudaGetLastError());
}

rsai_status rsai_rebuild(rsai_handle *h, void *stream) {
    Nvtx range("rsai_rebuild");
    if (!h) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!h->graph) {
        cudaStream_t cap_st;
        if (cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking) != cudaSuccess) return RSAI_ERR_CUDA;
        cudaGraph_t g;
        cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal);
        cudaError_t e = enqueue_build(h, cap_st);
        cudaError_t e2 = cudaStreamEndCapture(cap_st, &g);
        cudaStreamDestroy(cap_st);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            cudaGetLastError();
            return RSAI_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return RSAI_ERR_CUDA;
    }
    return (rsai_status)cuda_status(cudaGraphLaunch(h->graph, st));
}

rsai_status rsai_get_stats(rsai_handle *h, void *stream, rsai_stats *out) {
    if (!h || !out) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long s[kCounts + 2];
    int32_t herr = 0;
    std::vector<double> nb((size_t)h->nblocks);
    // every read on the caller's stream, one wait
    if (cudaMemcpyAsync(s, h->dscal, sizeof(s), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, h->err, sizeof(herr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(nb.data(), h->norm1_arr, sizeof(double) * nb.size(), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RSAI_ERR_CUDA;
    auto dbl = [&](int at) {
        double v;
        memcpy(&v, &s[at], sizeof(v));
        return v;
    };
    const unsigned long long *c = s + kCtr;
    memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->nnz_A = h->nnz;
    {
        double mx = 0.0;
        for (double v : nb) mx = std::max(mx, v);
        out->norm1_A = mx;
    }
    out->qr_flops = (double)c[CTR_QR];
    out->res_flops = (double)c[CTR_RES];
    out->refine_flops = (double)c[CTR_REFINE];
    out->refine_flops_f64 = (double)c[CTR_REFINE64];
    out->bytes = (double)c[CTR_BYTES];
    out->loops = (int64_t)c[CTR_LOOPS];
    out->solves = (int64_t)c[CTR_SOLVES];
    out->drops = (int64_t)c[CTR_DROPS];
    out->p_max = (int32_t)c[CTR_PMAX];
    out->q_max = (int32_t)c[CTR_QMAX];
    out->n_rank = (int64_t)c[CTR_RANK];
    out->n_nonfinite = (int64_t)c[CTR_NONFINITE];
    out->n_failed = (int64_t)c[CTR_FAILED];
    for (int b = 0; b < 3; ++b) out->cols_bin[b] = (int64_t)c[CTR_COUNT + b];
    out->cols_bin[0] += (int64_t)c[CTR_COUNT + kBinHalf];
    out->cols_bin_half = (int64_t)c[CTR_COUNT + kBinHalf];
    out->select_flops = (double)c[CTR_SELECT];
    out->frob = std::sqrt(dbl(kFrob2));
    out->n_c = (int64_t)s[kCounts + 0];
    out->nnz_M = (int64_t)s[kCounts + 1];
    return herr ? (rsai_status)herr : RSAI_OK;
}

rsai_status rsai_get_M(rsai_handle *h, int64_t *row_ptr, int32_t *col_idx, double *val, void *stream) {
    if (!h) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t nnzM = 0;
    if (cudaMemcpyAsync(&nnzM, h->Mrowptr + h->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return RSAI_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    if (row_ptr && cudaMemcpyAsync(row_ptr, h->Mrowptr, sizeof(int64_t) * (h->n + 1), cudaMemcpyDefault, st))
        return RSAI_ERR_CUDA;
    if (col_idx && cudaMemcpyAsync(col_idx, h->Mcols, sizeof(int32_t) * nnzM, cudaMemcpyDefault, st))
        return RSAI_ERR_CUDA;
    if (val && cudaMemcpyAsync(val, h->Mvals, sizeof(double) * nnzM, cudaMemcpyDefault, st)) return RSAI_ERR_CUDA;
    return (rsai_status)cuda_status(cudaStreamSynchronize(st));
}

rsai_status rsai_get_M_csc(rsai_handle *h, int64_t *col_ptr, int32_t *row_idx, int64_t *csc_to_csr, void *stream) {
    if (!h) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t nnzM = 0;
    if (cudaMemcpyAsync(&nnzM, h->Mcolptr + h->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return RSAI_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    if (col_ptr && cudaMemcpyAsync(col_ptr, h->Mcolptr, sizeof(int64_t) * (h->n + 1), cudaMemcpyDefault, st))
        return RSAI_ERR_CUDA;
    if (row_idx && cudaMemcpyAsync(row_idx, h->Mrows, sizeof(int32_t) * nnzM, cudaMemcpyDefault, st))
        return RSAI_ERR_CUDA;
    if (csc_to_csr && cudaMemcpyAsync(csc_to_csr, h->Mcsc_to_csr, sizeof(int64_t) * nnzM, cudaMemcpyDefault, st))
        return RSAI_ERR_CUDA;
    return (rsai_status)cuda_status(cudaStreamSynchronize(st));
}

rsai_status rsai_spmv(const rsai_csr *A, const double *x, double *y, void *stream) {
    int rc = check_csr_host(A);
    if (rc != RSAI_OK) return (rsai_status)rc;
    if (!x || !y) return RSAI_ERR_INVALID_ARG;
    if (!have_device()) return RSAI_ERR_NO_DEVICE;
    return (rsai_status)cuda_status(launch_spmv(A->n, A->row_ptr, A->col_idx, A->val, x, y, (cudaStream_t)stream));
}

rsai_status rsai_spmv_grad_values(const rsai_csr *A, const double *gy, const double *x, double *gval, void *stream) {
    if (!A || !A->row_ptr || !A->col_idx) return RSAI_ERR_INVALID_ARG;
    if (A->n <= 0 || A->nnz < 0 || A->n > INT32_MAX) return RSAI_ERR_SHAPE;
    if (!gy || !x || !gval) return RSAI_ERR_INVALID_ARG;
    if (!have_device()) return RSAI_ERR_NO_DEVICE;
    return (rsai_status)cuda_status(
        launch_spmv_grad_values(A->n, A->row_ptr, A->col_idx, gy, x, gval, (cudaStream_t)stream));
}

rsai_status rsai_get_columns(rsai_handle *h, double *rho, int32_t *loops, int32_t *flags, void *stream) {
    if (!h) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)h->n;
    if (rho && cudaMemcpyAsync(rho, h->rho, sizeof(double) * n, cudaMemcpyDefault, st)) return RSAI_ERR_CUDA;
    if (loops && cudaMemcpyAsync(loops, h->loops, sizeof(int32_t) * n, cudaMemcpyDefault, st)) return RSAI_ERR_CUDA;
    if (flags && cudaMemcpyAsync(flags, h->flags, sizeof(int32_t) * n, cudaMemcpyDefault, st)) return RSAI_ERR_CUDA;
    return (rsai_status)cuda_status(cudaStreamSynchronize(st));
}

rsai_status rsai_set_allocator(rsai_alloc_fn alloc, rsai_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return RSAI_ERR_INVALID_ARG;
    g_allocator = Allocator{alloc, release, alloc ? ctx : nullptr};
    return RSAI_OK;
}

rsai_status rsai_apply(rsai_handle *h, const double *x, double *y, void *stream) {
    if (!h || !x || !y) return RSAI_ERR_INVALID_ARG;
    return (rsai_status)cuda_status(
        launch_spmv(h->n, h->Mrowptr, h->Mcols, h->Mvals, x, y, (cudaStream_t)stream));
}

rsai_status rsai_bicgstab(const rsai_csr *A, rsai_handle *M, const double *b, double *x, double rtol, int32_t maxit,
                          int32_t *iters, double *relres, void *stream) {
    Nvtx range("rsai_bicgstab");
    int rc = check_csr_host(A);
    if (rc != RSAI_OK) return (rsai_status)rc;
    if (!b || !x || !iters || !relres || maxit < 0 || !(rtol > 0.0)) return RSAI_ERR_INVALID_ARG;
    if (M && M->n != A->n) return RSAI_ERR_SHAPE;
    int it = 0;
    double rr = 0.0;
    const cudaStream_t st = (cudaStream_t)stream;
    // the workspace comes from the installed allocator when there is one
    const Allocator a = g_allocator;
    double *work = nullptr;
    const size_t wb = bicgstab_workspace_bytes(A->n);
    if (a.alloc) {
        work = (double *)raw_alloc(a, wb, st);
        if (!work) return RSAI_ERR_OOM;
    }
    rc = bicgstab_run(A->n, A->row_ptr, A->col_idx, A->val, M ? M->Mrowptr : nullptr, M ? M->Mcols : nullptr,
                      M ? M->Mvals : nullptr, b, x, rtol, maxit, &it, &rr, st, work);
    if (work) raw_free(a, work, wb, st);
    *iters = it;
    *relres = rr;
    return (rsai_status)rc;
}

}  // extern "C"

namespace {

// values of A for a frozen-pattern pass: CSR copy + CSC through the map
int frozen_values(rsai_handle *h, const double *A_val, cudaStream_t st, DevA *out) {
    if (!h->fval) {
        int rc = dalloc(h, &h->fval, h->nnz, st);
        if (rc == RSAI_OK) rc = dalloc(h, &h->fcval, h->nnz, st);
        if (rc == RSAI_OK) rc = dalloc(h, &h->fctr, CTR_COUNT + kBinSlots, st);
        if (rc != RSAI_OK) return rc;
    }
    cudaMemsetAsync(h->fctr, 0, sizeof(unsigned long long) * (CTR_COUNT + kBinSlots), st);
    if (cudaMemcpyAsync(h->fval, A_val, sizeof(double) * h->nnz, cudaMemcpyDefault, st) != cudaSuccess)
        return RSAI_ERR_CUDA;
    k_csc_from_csr<<<blocks(h->nnz, 256), 256, 0, st>>>(h->fval, h->csc_to_csr, h->fcval, h->nnz);
    *out = DevA{h->n, h->row_ptr, h->col_idx, h->fval, h->col_ptr, h->row_idx, h->fcval, nullptr};
    return cuda_status(cudaGetLastError());
}

int64_t nnz_of_M(rsai_handle *h, cudaStream_t st) {
    int64_t nnzM = -1;
    if (cudaMemcpyAsync(&nnzM, h->Mrowptr + h->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -1;
    return nnzM;
}

int finish_frozen(rsai_handle *h, cudaStream_t st) {
    int32_t herr = 0;
    cudaMemcpyAsync(&herr, h->err, sizeof(herr), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    return herr;
}

}  // namespace

extern "C" {

rsai_status rsai_refit(rsai_handle *h, const double *A_val, double *M_val, double *rho2, void *stream) {
    Nvtx range("rsai_refit");
    if (!h || !A_val) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nnzM = nnz_of_M(h, st);
    if (nnzM < 0) return RSAI_ERR_CUDA;
    DevA A;
    int rc = frozen_values(h, A_val, st, &A);
    if (rc != RSAI_OK) return (rsai_status)rc;
    double *mv = M_val, *r2 = rho2;
    double *tmp = nullptr;
    const size_t tmp_bytes = sizeof(double) * (size_t)(nnzM + h->n + 1);
    if (!mv || !r2) {  // outputs the caller skipped go to a temporary
        tmp = (double *)raw_alloc(h->allocator, tmp_bytes, st);
        if (!tmp) return RSAI_ERR_OOM;
        if (!mv) mv = tmp;
        if (!r2) r2 = tmp + nnzM;
    }
    Frozen F{};
    F.Mcolptr = h->Mcolptr;
    F.Mrows = h->Mrows;
    F.Mcsc_to_csr = h->Mcsc_to_csr;
    F.Mval_csr = mv;
    F.rho2 = r2;
    cudaMemsetAsync(h->err, 0, sizeof(int32_t), st);
    cudaError_t e = enqueue_bins(h, MODE_REFIT, A, F, h->fctr, st);
    if (tmp) raw_free(h->allocator, tmp, tmp_bytes, st);
    if (e != cudaSuccess) return RSAI_ERR_CUDA;
    return (rsai_status)finish_frozen(h, st);
}

rsai_status rsai_backward(rsai_handle *h, const double *A_val, const double *grad_M, const double *grad_rho2,
                          double *grad_A, void *stream) {
    Nvtx range("rsai_backward");
    if (!h || !A_val || !grad_M || !grad_A) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nnzM = nnz_of_M(h, st);
    if (nnzM < 0) return RSAI_ERR_CUDA;
    DevA A;
    int rc = frozen_values(h, A_val, st, &A);
    if (rc != RSAI_OK) return (rsai_status)rc;
    // offsets of the I_k (|I_k| recorded by the build)
    if (!h->qoff && (rc = dalloc(h, &h->qoff, h->n + 1, st)) != RSAI_OK) return (rsai_status)rc;
    if (scan_counts(h, h->col_q, h->qoff, st) != cudaSuccess) return RSAI_ERR_CUDA;
    int64_t qtot = 0;
    cudaMemcpyAsync(&qtot, h->qoff + h->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    if (qtot > h->pool_q_cap) {
        int rc2 = dalloc(h, &h->poolI, qtot, st);
        if (rc2 == RSAI_OK) rc2 = dalloc(h, &h->poolR, qtot, st);
        if (rc2 == RSAI_OK) rc2 = dalloc(h, &h->poolW, qtot, st);
        if (rc2 != RSAI_OK) return (rsai_status)rc2;
        h->pool_q_cap = qtot;
    }
    if (nnzM > h->adj_m_cap) {
        int rc2 = dalloc(h, &h->alphaM, nnzM, st);
        if (rc2 == RSAI_OK) rc2 = dalloc(h, &h->xM, nnzM, st);
        if (rc2 == RSAI_OK) rc2 = dalloc(h, &h->Mcsr_to_csc, nnzM, st);
        if (rc2 != RSAI_OK) return (rsai_status)rc2;
        h->adj_m_cap = nnzM;
    }
    Frozen F{};
    F.Mcolptr = h->Mcolptr;
    F.Mrows = h->Mrows;
    F.Mcsc_to_csr = h->Mcsc_to_csr;
    F.grad_M = grad_M;
    F.grad_rho2 = grad_rho2;
    F.qoff = h->qoff;
    F.poolI = h->poolI;
    F.poolR = h->poolR;
    F.poolW = h->poolW;
    F.alphaM = h->alphaM;
    F.xM = h->xM;
    cudaMemsetAsync(h->err, 0, sizeof(int32_t), st);
    if (enqueue_bins(h, MODE_BACKWARD, A, F, h->fctr, st) != cudaSuccess) return RSAI_ERR_CUDA;
    if (launch_adjoint_gather(h->n, nnzM, h->row_ptr, h->col_idx, h->Mrowptr, h->Mcols, h->Mcsc_to_csr,
                              h->Mcsr_to_csc, h->qoff, h->poolI, h->poolR, h->poolW, h->alphaM, h->xM, grad_A,
                              st) != cudaSuccess)
        return RSAI_ERR_CUDA;
    return (rsai_status)finish_frozen(h, st);
}

rsai_status rsai_get_tuning(const rsai_handle *h, rsai_tuning *t) {
    if (!h || !t) return RSAI_ERR_INVALID_ARG;
    *t = h->tuning;
    return RSAI_OK;
}

rsai_status rsai_set_tuning(rsai_handle *h, const rsai_tuning *t) {
    if (!h || !t) return RSAI_ERR_INVALID_ARG;
    const int w = t->warp_bin_warps;
    if (w != 1 && w != 2 && w != 4 && w != 8) return RSAI_ERR_INVALID_ARG;
    if (t->warp_bin_ctas_per_sm < 0 || t->small_qr_max_p < 0 || t->small_qr_max_p > kSmallP ||
        t->global_bin_ctas < 0 || (t->half_bin != 0 && t->half_bin != 1))
        return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = h->alloc_stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    const rsai_tuning old = h->tuning;
    h->tuning = *t;
    const bool fp32 = h->params.precision == RSAI_FP32_REFINE;
    h->capW.small_p = t->small_qr_max_p;
    h->capH.small_p = t->small_qr_max_p;
    int occ = occupancy_bin_warp(fp32, w, h->capW);
    if (occ < 1 || occupancy_bin_half(fp32, w, h->capH) < 1) {
        h->tuning = old;
        h->capW.small_p = old.small_qr_max_p;
        h->capH.small_p = old.small_qr_max_p;
        return RSAI_ERR_INVALID_ARG;
    }
    if (plan_h(h, fp32) != RSAI_OK) return RSAI_ERR_CUDA;
    if (t->warp_bin_ctas_per_sm > 0) occ = std::min(occ, t->warp_bin_ctas_per_sm);
    h->grid_w = h->sms * occ;
    h->capW2.small_p = t->small_qr_max_p;
    if (plan_w2(h, fp32) != RSAI_OK) return RSAI_ERR_CUDA;
    if (t->global_bin_ctas > 0) {
        const int want = std::min(t->global_bin_ctas, h->sms);
        if (want > h->grid_g || (h->gwork && want < h->grid_g)) {
            // the slab follows the CTA count (one workspace per CTA); the new one
            // first, so that a failed allocation leaves the old one in place
            char *slab = nullptr;
            int rc = dalloc(h, &slab, h->gstride * (size_t)want, st);
            if (rc != RSAI_OK) return (rsai_status)rc;
            if (h->gwork) dfree(h, h->gwork, st);
            h->gwork = slab;
        }
        h->grid_g = want;
    }
    if (h->graph) {  // the launch shapes are part of the recorded graph
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return RSAI_OK;
}

rsai_status rsai_build_phase_times(rsai_handle *h, void *stream, double *ms) {
    if (!h || !ms) return RSAI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[RSAI_PHASE_COUNT + 1];
    for (auto &e : ev) cudaEventCreate(&e);
    cudaError_t e = enqueue_build(h, st, ev);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[RSAI_PHASE_COUNT]);
    if (e == cudaSuccess) {
        for (int i = 0; i < RSAI_PHASE_COUNT; ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
            ms[i] = t;
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    return (rsai_status)cuda_status(e);
}

rsai_status rsai_peak_fma(int32_t fp64, void *stream, double *flops_per_s) {
    if (!flops_per_s) return RSAI_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return RSAI_ERR_NO_DEVICE;
    }
    return (rsai_status)cuda_status(run_peak_fma(fp64 != 0, (cudaStream_t)stream, flops_per_s));
}

}  // extern "C"
