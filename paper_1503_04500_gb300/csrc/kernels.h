// kernels.h -- declarations shared by the host code and the kernel files.
#pragma once

#include "column.cuh"

namespace rsai {

constexpr int kBlockThreads = 512;  // CTA team size of bins C and G (measured: 1.3x faster than 256)
constexpr int kWarpsPerCta = 4;     // warps per CTA in bin W
constexpr int kStatBlocks = 256;    // blocks of the per-column statistics reduction
// Column counts per bin in the global counters (after the CTR_COUNT work
// counters): 0 = warp bins W and W2, 1 = CTA bin, 2 = global bin, 3 = bin H
// (also included in 0's total when the statistics are read)
constexpr int kBinHalf = 3;
constexpr int kBinSlots = 4;

// input checks, ||A||_1, statistics, scan, assembly
__global__ void k_check_ptr(const int64_t *ptr, int64_t n, int64_t nnz, int32_t *err);
__global__ void k_check_idx(const int64_t *ptr, const int32_t *idx, int64_t n, int32_t *err, int empty_is_error);
__global__ void k_csc_map(DevA A, int64_t *csc_to_csr, int32_t *err);
__global__ void k_csc_from_csr(const double *csr_val, const int64_t *csc_to_csr, double *cval, int64_t nnz);
__global__ void k_to_f32(const double *in, float *out, int64_t n);
__global__ void k_norm1(const int64_t *col_ptr, const double *cval, int64_t n, const int32_t *col_block,
                        double *out);
__global__ void k_collect_failed(const int32_t *flags, int64_t n, int32_t *list, uint32_t *count);
// largest-first order of a column queue (cost buckets: bit length of a proxy)
constexpr int kCostBuckets = 32;
__global__ void k_cost_buckets(const int32_t *list, const uint32_t *count, const int64_t *col_ptr,
                               const int32_t *row_idx, const int64_t *row_ptr, uint8_t *bucket, uint32_t *hist);
__global__ void k_cost_offsets(uint32_t *hist);
__global__ void k_cost_scatter(const int32_t *list, const uint32_t *count, const uint8_t *bucket, uint32_t *offset,
                               int32_t *out);
__global__ void k_col_block(const int64_t *cstart, int32_t nblocks, int64_t n, int32_t *col_block);
__global__ void k_shift_ptr(int64_t *ptr, int64_t n, const int32_t *col_block, const int64_t *estart,
                            int64_t nnz_total);
__global__ void k_shift_idx(const int64_t *ptr, int32_t *idx, int64_t n, const int32_t *col_block,
                            const int64_t *cstart);
__global__ void k_block_stats(const int64_t *cstart, const double *rho, const int32_t *flags, const int32_t *len,
                              double eps, double *frob2, long long *nc, long long *nnz);
__global__ void k_column_stats(const double *rho, const int32_t *flags, const int32_t *len, int64_t n, double eps,
                               double *partial, unsigned long long *counts);
__global__ void k_column_stats_final(const double *partial, double *frob2);
__global__ void k_tau_fixed(const double *norm1, double tol, double *tau, int32_t nblocks);
__global__ void k_scan_blocks(const int32_t *in, int64_t n, int64_t *out, int64_t *block_sums);
__global__ void k_scan_sums(int64_t *block_sums, int64_t nb, int64_t *total);
__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *block_sums, const int64_t *total);
__global__ void k_pool_to_csc(const int64_t *col_off, const int32_t *col_len, const int32_t *pool_rows,
                              const double *pool_vals, const int64_t *Mcolptr, int32_t *Mrows, double *Mvals,
                              int32_t *row_count, int64_t n);
__global__ void k_csc_to_rows(const int64_t *Mcolptr, const int32_t *Mrows, const double *Mvals,
                              const int64_t *Mrowptr, int32_t *cursor, int32_t *tcols, double *tvals,
                              int64_t *tsrc, int64_t n);
__global__ void k_sort_rows(const int64_t *Mrowptr, const int32_t *tcols, const double *tvals, const int64_t *tsrc,
                            int32_t *Mcols, double *Mvals_csr, int64_t *csc_to_csr_M, int64_t n);

template <typename T> size_t work_bytes(const Caps &c);

cudaError_t launch_bin_warp(int mode, bool fp32, int grid, int warps, const DevA &A, const DevParams &P,
                            const Caps &cap, const ColQueue &Q, const ColOut &O, const Frozen &F,
                            unsigned long long *gctr, bool last, cudaStream_t st);
cudaError_t launch_bin_half(int mode, bool fp32, int grid, int warps, const DevA &A, const DevParams &P,
                            const Caps &cap, const ColQueue &Q, const ColOut &O, const Frozen &F,
                            unsigned long long *gctr, bool last, cudaStream_t st);
cudaError_t launch_bin_block(int mode, bool fp32, int grid, const DevA &A, const DevParams &P, const Caps &cap,
                             const ColQueue &Q, const ColOut &O, const Frozen &F, unsigned long long *gctr,
                             bool last, char *gwork, size_t gstride, int bin, cudaStream_t st);
cudaError_t launch_adjoint_gather(int64_t n, int64_t nnzM, const int64_t *row_ptr, const int32_t *col_idx,
                                  const int64_t *Mrowptr, const int32_t *Mcols, const int64_t *Mcsc_to_csr,
                                  int64_t *Mcsr_to_csc, const int64_t *qoff, const int32_t *poolI,
                                  const double *poolR, const double *poolW, const double *alphaM,
                                  const double *xM, double *grad, cudaStream_t st);
int occupancy_bin_warp(bool fp32, int warps, const Caps &cap);
int occupancy_bin_half(bool fp32, int warps, const Caps &cap);
int occupancy_bin_block(bool fp32, const Caps &cap, bool global_work);

// apply / solver kernels (apply_kernels.cu)
cudaError_t launch_spmv(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                        const double *x, double *y, cudaStream_t st);
// gval[e] = gy[row(e)] * x[col(e)] over the stored entries of a CSR matrix
cudaError_t launch_spmv_grad_values(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *gy,
                                    const double *x, double *gval, cudaStream_t st);
cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *partials, double *out, cudaStream_t st);
int bicgstab_run(int64_t n, const int64_t *Arp, const int32_t *Aci, const double *Av, const int64_t *Mrp,
                 const int32_t *Mci, const double *Mv, const double *b, double *x, double rtol, int maxit,
                 int *iters, double *relres, cudaStream_t st, double *work = nullptr);
// device bytes bicgstab_run needs as its workspace for size n
size_t bicgstab_workspace_bytes(int64_t n);

// BiCGStab vector steps (apply_kernels.cu); scalars on the device
__global__ void k_bicg_p(int64_t n, const double *sc, const double *r, const double *v, double *p);
__global__ void k_bicg_alpha(double *sc);
__global__ void k_bicg_s(int64_t n, const double *sc, const double *r, const double *v, double *s);
__global__ void k_bicg_half(int64_t n, const double *sc, const double *p, double *y);
__global__ void k_bicg_omega(double *sc);
__global__ void k_bicg_update(int64_t n, const double *sc, const double *p, const double *s, const double *t,
                              double *y, double *r);
__global__ void k_bicg_shift(double *sc);
__global__ void k_bicg_init(int64_t n, const double *b, double *r, double *rhat, double *p, double *v, double *y,
                            double *sc);
__global__ void k_axpy_sub(int64_t n, const double *b, const double *ax, double *out);

// FMA-chain peak (peak_kernels.cu)
cudaError_t run_peak_fma(bool fp64, cudaStream_t st, double *flops_per_s);

}  // namespace rsai
