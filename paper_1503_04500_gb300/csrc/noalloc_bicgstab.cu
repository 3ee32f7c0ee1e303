// noalloc_bicgstab.cu -- rsai_bicgstab_noalloc: the preconditioned BiCGStab
// solve for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they solve: code running inside another framework's memory pool or
// plugin interface that forbids allocations during execution, real-time loops
// where an allocation (and its implicit synchronisation) is not allowed, or
// processes whose device memory is fully reserved up front.  For them this
// entry point runs rsai_bicgstab's solver (bicgstab_run, the same code) with
// its workspace in one file-scope device array of fixed size, reserved when
// the library is loaded and held by every GPU that loads it until the process
// exits.
//
// Limit: n <= kNoAllocMaxN (65536); larger problems are rejected with
// RSAI_ERR_TOO_LARGE.  The array holds 9 work vectors of kNoAllocMaxN doubles
// plus the partial sums and scalars of the dot products (about 4.7 MB).
//
// Sharing: every call uses the same array and leaves its last contents there.
// The solver sets every vector and scalar it reads before reading it
// (r, r^, p, v, y and the scalars at its start), so no state carries over
// between calls, but calls whose work overlaps on the GPU (on different
// streams, or from several host threads without ordering) race on the array
// and give wrong results: order them on one stream.
//
// Set-up: the first call on each device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress and keeps it for the
// later calls on that device; make that first call while no stream of the
// process is being captured.  The solve itself waits for the stream at every
// iteration, so it never runs inside a capture.  A cudaDeviceReset unloads the
// library's device code, and the kept address is then stale: do not call this
// entry point on a device after resetting it.
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
    if (A->n > kNoAllocMaxN || bicgstab_workspace_bytes(A->n) > sizeof(g_noalloc_scratch))
        return RSAI_ERR_TOO_LARGE;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return RSAI_ERR_NO_DEVICE;
    }
    double *work = nullptr;
    const int rc = scratch_address(&work);
    if (rc != RSAI_OK) return (rsai_status)rc;
    int it = 0;
    double rr = 0.0;
    const int status = bicgstab_run(A->n, A->row_ptr, A->col_idx, A->val, M ? M->row_ptr : nullptr,
                                    M ? M->col_idx : nullptr, M ? M->val : nullptr, b, x, rtol, maxit, &it, &rr,
                                    (cudaStream_t)stream, work);
    *iters = it;
    *relres = rr;
    return (rsai_status)status;
}
