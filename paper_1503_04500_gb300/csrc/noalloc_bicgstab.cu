// noalloc_bicgstab.cu -- rsai_bicgstab_noalloc: the preconditioned BiCGStab
// solve for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they solve: code running inside another framework's memory pool or
// plugin interface that forbids allocations during execution, real-time loops
// where an allocation (and its implicit synchronisation) is not allowed, or
// processes whose device memory is fully reserved up front.  For them this
// entry point runs the same right-preconditioned BiCGStab as rsai_bicgstab
// with every work vector in one file-scope device array of fixed size,
// reserved when the library is loaded and held by every GPU that loads it
// until the process exits.
//
// Limit: n <= kNoAllocMaxN (65536); larger problems are rejected with
// RSAI_ERR_TOO_LARGE.  The array holds 9 work vectors of kNoAllocMaxN doubles
// plus the partial sums and scalars of the dot products (about 4.7 MB).
//
// Sharing: every call uses the same array and leaves its last contents there.
// Each call initialises what it reads before reading it (r, r^, p, v, y and
// the scalars are set at the start), so no state carries over between calls,
// but calls whose work overlaps on the GPU (on different streams, or from
// several host threads without ordering) race on the array and give wrong
// results: order them on one stream.
//
// Set-up: the device address of the array is looked up with
// cudaGetSymbolAddress the first time the entry point runs on each device
// (with that device current) and cached; make that first call before any
// stream capture begins.
#include <mutex>

#include "kernels.h"

namespace rsai {

constexpr int64_t kNoAllocMaxN = 65536;
constexpr int64_t kNoAllocPartials = 512;  // >= the dot kernels' partial sums
constexpr int64_t kNoAllocWords = 9 * kNoAllocMaxN + kNoAllocPartials + 16;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocWords];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_dev[kMaxDevices] = {nullptr};

// device address of the array on the current device (looked up once per device)
int scratch_address(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RSAI_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RSAI_ERR_CUDA;
        }
        g_scratch_dev[dev] = (double *)p;
    }
    *out = g_scratch_dev[dev];
    return RSAI_OK;
}

unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace rsai

using namespace rsai;

extern "C" rsai_status rsai_bicgstab_noalloc(const rsai_csr *A, const rsai_csr *M, const double *b, double *x,
                                             double rtol, int32_t maxit, int32_t *iters, double *relres,
                                             void *stream) {
    if (!A || !A->row_ptr || !A->col_idx || !A->val || !b || !x || !iters || !relres) return RSAI_ERR_INVALID_ARG;
    if (maxit < 0 || !(rtol > 0.0)) return RSAI_ERR_INVALID_ARG;
    if (A->n <= 0 || A->nnz < 0) return RSAI_ERR_SHAPE;
    if (M && (!M->row_ptr || !M->col_idx || !M->val)) return RSAI_ERR_INVALID_ARG;
    if (M && M->n != A->n) return RSAI_ERR_SHAPE;
    if (A->n > kNoAllocMaxN) return RSAI_ERR_TOO_LARGE;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return RSAI_ERR_NO_DEVICE;
    }
    double *buf = nullptr;
    int rc = scratch_address(&buf);
    if (rc != RSAI_OK) return (rsai_status)rc;

    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = A->n;
    const size_t vb = sizeof(double) * (size_t)n;
    double *r = buf, *rhat = r + n, *p = rhat + n, *v = p + n, *s = v + n, *t = s + n, *y = t + n, *tmp = y + n,
           *tmp2 = tmp + n, *partials = tmp2 + n, *sc = partials + kNoAllocPartials;
    const bool prec = M != nullptr;
    const int T = 256;
    double h[16];
    int status = RSAI_ERR_NOT_CONVERGED;
    int it = 0;
    auto fetch = [&](int upto) -> bool {
        if (cudaMemcpyAsync(h, sc, sizeof(double) * upto, cudaMemcpyDeviceToHost, st) != cudaSuccess) return false;
        return cudaStreamSynchronize(st) == cudaSuccess;
    };
    auto applyM = [&](const double *in, double *out) -> const double * {
        if (!prec) return in;
        launch_spmv(n, M->row_ptr, M->col_idx, M->val, in, out, st);
        return out;
    };
    const int64_t *Arp = A->row_ptr;
    const int32_t *Aci = A->col_idx;
    const double *Av = A->val;
    k_bicg_init<<<nblocks(n, T), T, 0, st>>>(n, b, r, rhat, p, v, y, sc);
    launch_dot(n, b, b, partials, sc + 9, st);
    if (!fetch(10)) return RSAI_ERR_CUDA;
    const double nb = sqrt(h[9]);
    if (nb == 0.0) {
        cudaMemsetAsync(x, 0, vb, st);
        *iters = 0;
        *relres = 0.0;
        return (rsai_status)(cudaStreamSynchronize(st) == cudaSuccess ? RSAI_OK : RSAI_ERR_CUDA);
    }
    for (it = 1; it <= maxit; ++it) {
        launch_dot(n, rhat, r, partials, sc + 0, st);
        k_bicg_p<<<nblocks(n, T), T, 0, st>>>(n, sc, r, v, p);
        launch_spmv(n, Arp, Aci, Av, applyM(p, tmp), v, st);
        launch_dot(n, rhat, v, partials, sc + 4, st);
        k_bicg_alpha<<<1, 1, 0, st>>>(sc);
        k_bicg_s<<<nblocks(n, T), T, 0, st>>>(n, sc, r, v, s);
        launch_dot(n, s, s, partials, sc + 7, st);
        if (!fetch(9)) { status = RSAI_ERR_CUDA; break; }
        if (h[0] == 0.0) { status = RSAI_ERR_BREAKDOWN; break; }
        if (sqrt(h[7]) / nb < rtol) {
            k_bicg_half<<<nblocks(n, T), T, 0, st>>>(n, sc, p, y);
            status = RSAI_OK;
            break;
        }
        launch_spmv(n, Arp, Aci, Av, applyM(s, tmp), t, st);
        launch_dot(n, t, s, partials, sc + 5, st);
        launch_dot(n, t, t, partials, sc + 6, st);
        if (!fetch(9)) { status = RSAI_ERR_CUDA; break; }
        if (h[6] == 0.0) { status = RSAI_ERR_BREAKDOWN; break; }
        k_bicg_omega<<<1, 1, 0, st>>>(sc);
        k_bicg_update<<<nblocks(n, T), T, 0, st>>>(n, sc, p, s, t, y, r);
        launch_dot(n, r, r, partials, sc + 8, st);
        if (!fetch(9)) { status = RSAI_ERR_CUDA; break; }
        if (sqrt(h[8]) / nb < rtol) { status = RSAI_OK; break; }
        if (h[3] == 0.0) { status = RSAI_ERR_BREAKDOWN; break; }
        k_bicg_shift<<<1, 1, 0, st>>>(sc);
    }
    if (it > maxit) it = maxit;
    if (prec) launch_spmv(n, M->row_ptr, M->col_idx, M->val, y, x, st);
    else cudaMemcpyAsync(x, y, vb, cudaMemcpyDeviceToDevice, st);
    launch_spmv(n, Arp, Aci, Av, x, tmp, st);
    k_axpy_sub<<<nblocks(n, T), T, 0, st>>>(n, b, tmp, tmp2);
    launch_dot(n, tmp2, tmp2, partials, sc + 10, st);
    double rr = 0.0;
    cudaMemcpyAsync(&rr, sc + 10, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    *iters = it;
    *relres = sqrt(rr) / nb;
    return (rsai_status)status;
}
