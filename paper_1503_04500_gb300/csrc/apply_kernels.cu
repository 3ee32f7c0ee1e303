// apply_kernels.cu -- CSR SpMV (y = M x, y = A x) and the vector kernels of
// right-preconditioned BiCGStab (Eq. 1.2: A M y = b, x = M y; Section 5).
//
// Every reduction has a fixed order (fixed grid, fixed tree), so repeated
// solves give identical iterates.
#include "kernels.h"

namespace rsai {

// 8 lanes per row; lanes stride over the row, then a 3-step shuffle tree.
__global__ void k_spmv(int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                       const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t row = g >> 3;
    int sub = threadIdx.x & 7;
    double acc = 0.0;
    if (row < n) {
        int64_t a = row_ptr[row], b = row_ptr[row + 1];
        for (int64_t e = a + sub; e < b; e += 8) acc = fma(val[e], x[col_idx[e]], acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (row < n && sub == 0) y[row] = acc;
}

// gval[e] = gy[i] x[col(e)] for every stored entry e of row i: the gradient
// of y = A x with respect to the stored values of A.  8 lanes per row, one
// write per entry, no reduction.
__global__ void k_spmv_grad_values(int64_t n, const int64_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col_idx, const double *__restrict__ gy,
                                   const double *__restrict__ x, double *__restrict__ gval) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t row = g >> 3;
    int sub = threadIdx.x & 7;
    if (row >= n) return;
    const double gr = gy[row];
    const int64_t a = row_ptr[row], b = row_ptr[row + 1];
    for (int64_t e = a + sub; e < b; e += 8) gval[e] = gr * x[col_idx[e]];
}

constexpr int kDotBlocks = 304;
constexpr int kDotThreads = 256;

__global__ void k_dot_partial(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                              double *partials) {
    __shared__ double sh[kDotThreads];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads)
        s = fma(x[i], y[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kDotThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double *partials, double *out) {
    __shared__ double sh[512];
    double s = 0.0;
    for (int i = threadIdx.x; i < kDotBlocks; i += 512) s += partials[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 256; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_spmv_grad_values(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *gy,
                                    const double *x, double *gval, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int T = 256;
    k_spmv_grad_values<<<(unsigned)((n * 8 + T - 1) / T), T, 0, st>>>(n, row_ptr, col_idx, gy, x, gval);
    return cudaGetLastError();
}

cudaError_t launch_spmv(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                        const double *x, double *y, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t threads = n * 8;
    int64_t grid = (threads + 255) / 256;
    k_spmv<<<(unsigned)grid, 256, 0, st>>>(n, row_ptr, col_idx, val, x, y);
    return cudaGetLastError();
}

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *partials, double *out, cudaStream_t st) {
    k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(n, x, y, partials);
    k_dot_final<<<1, 512, 0, st>>>(partials, out);
    return cudaGetLastError();
}

}  // namespace rsai

// BiCGStab vector steps; scalars live on the device:
// sc[0] rho, sc[1] rho_old, sc[2] alpha, sc[3] omega, sc[4] (rhat,v), sc[5] (t,s),
// sc[6] (t,t), sc[7] (s,s), sc[8] (r,r)
namespace rsai {

__global__ void k_bicg_p(int64_t n, const double *sc, const double *r, const double *v, double *p) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double beta = (sc[0] / sc[1]) * (sc[2] / sc[3]);
    p[i] = r[i] + beta * (p[i] - sc[3] * v[i]);
}

__global__ void k_bicg_alpha(double *sc) { sc[2] = sc[0] / sc[4]; }

__global__ void k_bicg_s(int64_t n, const double *sc, const double *r, const double *v, double *s) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) s[i] = r[i] - sc[2] * v[i];
}

__global__ void k_bicg_half(int64_t n, const double *sc, const double *p, double *y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += sc[2] * p[i];
}

__global__ void k_bicg_omega(double *sc) { sc[3] = (sc[6] != 0.0) ? sc[5] / sc[6] : 0.0; }

__global__ void k_bicg_update(int64_t n, const double *sc, const double *p, const double *s, const double *t,
                              double *y, double *r) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] += sc[2] * p[i] + sc[3] * s[i];
    r[i] = s[i] - sc[3] * t[i];
}

__global__ void k_bicg_shift(double *sc) { sc[1] = sc[0]; }

__global__ void k_bicg_init(int64_t n, const double *b, double *r, double *rhat, double *p, double *v, double *y,
                            double *sc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        r[i] = b[i];
        rhat[i] = b[i];
        p[i] = 0.0;
        v[i] = 0.0;
        y[i] = 0.0;
    }
    if (i == 0) { sc[1] = 1.0; sc[2] = 1.0; sc[3] = 1.0; }
}

__global__ void k_axpy_sub(int64_t n, const double *b, const double *ax, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = b[i] - ax[i];
}

}  // namespace rsai

// ---------------------------------------------------------------------------
// host driver of BiCGStab (same steps as the textbook method the oracle uses)
namespace rsai {

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

size_t bicgstab_workspace_bytes(int64_t n) {
    return sizeof(double) * (size_t)(n > 0 ? n : 1) * 9 + sizeof(double) * (kDotBlocks + 16);
}

int bicgstab_run(int64_t n, const int64_t *Arp, const int32_t *Aci, const double *Av, const int64_t *Mrp,
                 const int32_t *Mci, const double *Mv, const double *b, double *x, double rtol, int maxit,
                 int *iters, double *relres, cudaStream_t st, double *work) {
    const size_t vb = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *buf = work;
    const bool own = work == nullptr;  // else the caller's workspace of bicgstab_workspace_bytes(n)
    if (own && cudaMallocAsync((void **)&buf, bicgstab_workspace_bytes(n), st) != cudaSuccess)
        return RSAI_ERR_OOM;
    double *r = buf, *rhat = r + n, *p = rhat + n, *v = p + n, *s = v + n, *t = s + n, *y = t + n, *tmp = y + n,
           *tmp2 = tmp + n, *partials = tmp2 + n, *sc = partials + kDotBlocks;
    const bool prec = Mrp != nullptr;
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
        launch_spmv(n, Mrp, Mci, Mv, in, out, st);
        return out;
    };
    k_bicg_init<<<blocks_for(n, T), T, 0, st>>>(n, b, r, rhat, p, v, y, sc);
    launch_dot(n, b, b, partials, sc + 9, st);
    if (!fetch(10)) { if (own) cudaFreeAsync(buf, st); return RSAI_ERR_CUDA; }
    const double nb = sqrt(h[9]);
    if (nb == 0.0) {
        cudaMemsetAsync(x, 0, vb, st);
        *iters = 0;
        *relres = 0.0;
        if (own) cudaFreeAsync(buf, st);
        return RSAI_OK;
    }
    for (it = 1; it <= maxit; ++it) {
        launch_dot(n, rhat, r, partials, sc + 0, st);
        k_bicg_p<<<blocks_for(n, T), T, 0, st>>>(n, sc, r, v, p);
        launch_spmv(n, Arp, Aci, Av, applyM(p, tmp), v, st);
        launch_dot(n, rhat, v, partials, sc + 4, st);
        k_bicg_alpha<<<1, 1, 0, st>>>(sc);
        k_bicg_s<<<blocks_for(n, T), T, 0, st>>>(n, sc, r, v, s);
        launch_dot(n, s, s, partials, sc + 7, st);
        if (!fetch(9)) { status = RSAI_ERR_CUDA; break; }
        // rho = r^T r = 0, or r^T v = 0 (alpha undefined): the recurrences break down
        if (h[0] == 0.0 || h[4] == 0.0) { status = RSAI_ERR_BREAKDOWN; break; }
        if (sqrt(h[7]) / nb < rtol) {
            k_bicg_half<<<blocks_for(n, T), T, 0, st>>>(n, sc, p, y);
            status = RSAI_OK;
            break;
        }
        launch_spmv(n, Arp, Aci, Av, applyM(s, tmp), t, st);
        launch_dot(n, t, s, partials, sc + 5, st);
        launch_dot(n, t, t, partials, sc + 6, st);
        if (!fetch(9)) { status = RSAI_ERR_CUDA; break; }
        if (h[6] == 0.0) { status = RSAI_ERR_BREAKDOWN; break; }
        k_bicg_omega<<<1, 1, 0, st>>>(sc);
        k_bicg_update<<<blocks_for(n, T), T, 0, st>>>(n, sc, p, s, t, y, r);
        launch_dot(n, r, r, partials, sc + 8, st);
        if (!fetch(9)) { status = RSAI_ERR_CUDA; break; }
        if (sqrt(h[8]) / nb < rtol) { status = RSAI_OK; break; }
        if (h[3] == 0.0) { status = RSAI_ERR_BREAKDOWN; break; }
        k_bicg_shift<<<1, 1, 0, st>>>(sc);
    }
    if (it > maxit) it = maxit;
    // x = M y, true residual
    if (prec) launch_spmv(n, Mrp, Mci, Mv, y, x, st);
    else cudaMemcpyAsync(x, y, vb, cudaMemcpyDeviceToDevice, st);
    launch_spmv(n, Arp, Aci, Av, x, tmp, st);
    k_axpy_sub<<<blocks_for(n, T), T, 0, st>>>(n, b, tmp, tmp2);
    launch_dot(n, tmp2, tmp2, partials, sc + 10, st);
    double rr = 0.0;
    cudaMemcpyAsync(&rr, sc + 10, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (own) cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSAI_ERR_CUDA;
    *iters = it;
    *relres = sqrt(rr) / nb;
    return status;
}

}  // namespace rsai
