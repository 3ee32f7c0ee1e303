// setup_kernels.cu -- the kernels around the column algorithm: input checks
// (status codes, never a trap), the CSC->CSR map, ||A||_1 and the fixed drop
// threshold (Eq. 4.3), batch offsets, the per-column statistics, the
// assembly of M (CSC from the result pool, then CSR with sorted rows), and the
// second pass of the adjoint.  The bins themselves are in build_kernels.cu.
#include "kernels.h"

namespace rsai {

// ---------------------------------------------------------------------------
// input checks (status codes, never a trap)

__global__ void k_check_ptr(const int64_t *ptr, int64_t n, int64_t nnz, int32_t *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == 0 && ptr[0] != 0) set_error(err, RSAI_ERR_INDEX_RANGE);
    if (i == n && ptr[n] != nnz) set_error(err, RSAI_ERR_SHAPE);
    if (i < n && ptr[i] > ptr[i + 1]) set_error(err, RSAI_ERR_INDEX_RANGE);
}

// Runs after k_check_ptr on the same stream: if a pointer array was found
// invalid (err set), its entries are not used as indices.
__global__ void k_check_idx(const int64_t *ptr, const int32_t *idx, int64_t n, int32_t *err, int empty_is_error) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || *(volatile int32_t *)err != 0) return;
    int64_t a = ptr[i], b = ptr[i + 1];
    if (empty_is_error && a == b) set_error(err, RSAI_ERR_EMPTY_COLUMN);
    for (int64_t e = a; e < b; ++e) {
        int32_t v = idx[e];
        if (v < 0 || v >= n) { set_error(err, RSAI_ERR_INDEX_RANGE); return; }
        if (e > a && idx[e - 1] >= v) { set_error(err, RSAI_ERR_UNSORTED); return; }
    }
}

// CSR position of every CSC entry; checks that both describe the same matrix.
// Runs after the pointer and index checks on the same stream and does nothing
// if they found an error (its indices would not be safe to follow).
__global__ void k_csc_map(DevA A, int64_t *csc_to_csr, int32_t *err) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= A.n || *(volatile int32_t *)err != 0) return;
    for (int64_t e = A.col_ptr[j]; e < A.col_ptr[j + 1]; ++e) {
        int32_t i = A.row_idx[e];
        int64_t lo = A.row_ptr[i];
        int len = (int)(A.row_ptr[i + 1] - lo);
        int pos = find_i32(A.col_idx + lo, len, (int32_t)j);
        if (pos < 0 || A.val[lo + pos] != A.cval[e]) {
            set_error(err, RSAI_ERR_SHAPE);
            csc_to_csr[e] = -1;
        } else {
            csc_to_csr[e] = lo + pos;
        }
    }
}

// CSC values from CSR values through the map (after new values arrive)
__global__ void k_csc_from_csr(const double *csr_val, const int64_t *csc_to_csr, double *cval, int64_t nnz) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz) cval[e] = csr_val[csc_to_csr[e]];
}

// out = in rounded to float (round to nearest), the FP32 QR's copy of A's values
__global__ void k_to_f32(const double *in, float *out, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) out[e] = __double2float_rn(in[e]);
}

// ||A||_1 = max_j sum_i |a_ij| (Eq. 4.3), per block of columns; nonnegative
// doubles order like their bits
// ||A||_1 per block: the column abs-sums, max-combined as the bit patterns of
// non-negative doubles (which order like the values).  A warp whose columns
// share one block reduces first and makes one atomic update.
__global__ void k_norm1(const int64_t *col_ptr, const double *cval, int64_t n, const int32_t *col_block,
                        double *out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    int b = -1;
    if (j < n) {
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) s += fabs(cval[e]);
        b = col_block ? col_block[j] : 0;
    }
    unsigned long long key = (unsigned long long)__double_as_longlong(s);
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (__all_sync(0xffffffffu, b == b0 || b < 0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
        if ((threadIdx.x & 31) == 0 && b0 >= 0) atomicMax((unsigned long long *)&out[b0], key);
    } else if (b >= 0) {
        atomicMax((unsigned long long *)&out[b], key);
    }
}

// columns flagged FAILED (e.g. the result pool was full), for a second run
__global__ void k_collect_failed(const int32_t *flags, int64_t n, int32_t *list, uint32_t *count) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n && (flags[k] & RSAI_COL_FAILED)) list[atomicAdd(count, 1u)] = (int32_t)k;
}

// block of every column from the block start offsets
__global__ void k_col_block(const int64_t *cstart, int32_t nblocks, int64_t n, int32_t *col_block) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    int lo = 0, hi = nblocks;  // last b with cstart[b] <= j
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (cstart[mid] <= j) lo = mid; else hi = mid;
    }
    col_block[j] = lo;
}

// pointers and indices of members copied side by side become one
// block-diagonal matrix: pointers += nnz offset, indices += column offset
__global__ void k_shift_ptr(int64_t *ptr, int64_t n, const int32_t *col_block, const int64_t *estart,
                            int64_t nnz_total) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) ptr[i] += estart[col_block[i]];
    if (i == n) ptr[n] = nnz_total;
}
__global__ void k_shift_idx(const int64_t *ptr, int32_t *idx, int64_t n, const int32_t *col_block,
                            const int64_t *cstart) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t off = (int32_t)cstart[col_block[i]];
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) idx[e] += off;
}

// per-block ||AM - I||_F^2, n_c and nnz(M) in a fixed order (one CTA per block)
__global__ void k_block_stats(const int64_t *cstart, const double *rho, const int32_t *flags, const int32_t *len,
                              double eps, double *frob2, long long *nc, long long *nnz) {
    __shared__ double sh[256];
    __shared__ long long s1[256], s2[256];
    const int b = blockIdx.x;
    double a = 0.0;
    long long c = 0, z = 0;
    for (int64_t k = cstart[b] + threadIdx.x; k < cstart[b + 1]; k += 256) {
        const bool failed = flags[k] & RSAI_COL_FAILED;
        if (!failed) a = fma(rho[k], rho[k], a);
        c += (failed || abskey(rho[k]) > abskey(eps)) ? 1 : 0;
        z += len[k];
    }
    sh[threadIdx.x] = a;
    s1[threadIdx.x] = c;
    s2[threadIdx.x] = z;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        frob2[b] = sh[0];
        nc[b] = s1[0];
        nnz[b] = s2[0];
    }
}

// ---------------------------------------------------------------------------
// adjoint, second pass: dL/dA(i,j) = sum over the columns k of row j of M of
//   r_k(i) alpha_k(j) - w_k(i) x_k(j)      (k ascending: fixed order)

__global__ void k_invert_map(const int64_t *map, int64_t n, int64_t *inv) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) inv[map[e]] = e;
}

__global__ void k_adjoint_gather(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col_idx,
                                 const int64_t *Mrowptr, const int32_t *Mcols, const int64_t *Mcsr_to_csc,
                                 const int64_t *qoff, const int32_t *poolI, const double *poolR,
                                 const double *poolW, const double *alphaM, const double *xM, double *grad) {
    // one thread per nonzero A(i,j) (CSR position e); its row by binary search
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int64_t lo = 0, hi = n;  // last row with row_ptr[row] <= e
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (row_ptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int32_t i = (int32_t)lo;
    const int32_t j = col_idx[e];
    double acc = 0.0;
    for (int64_t f = Mrowptr[j]; f < Mrowptr[j + 1]; ++f) {
        const int32_t kk = Mcols[f];
        const int64_t ce = Mcsr_to_csc[f];
        const int64_t a = qoff[kk];
        const int pos = find_i32(poolI + a, (int)(qoff[kk + 1] - a), i);
        if (pos >= 0) acc += poolR[a + pos] * alphaM[ce] - poolW[a + pos] * xM[ce];
    }
    grad[e] = acc;
}

// ---------------------------------------------------------------------------
// statistics over the per-column outputs in a fixed order (deterministic)

__global__ void k_column_stats(const double *rho, const int32_t *flags, const int32_t *len, int64_t n, double eps,
                               double *partial /* [kStatBlocks] */, unsigned long long *counts /* [2] */) {
    __shared__ double sh[256];
    double a = 0.0;
    unsigned long long nc = 0, nnz = 0;
    for (int64_t k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (int64_t)kStatBlocks * 256) {
        double r = rho[k];
        bool failed = flags[k] & RSAI_COL_FAILED;
        if (!failed) a = fma(r, r, a);
        nc += (failed || abskey(r) > abskey(eps)) ? 1 : 0;
        nnz += (unsigned long long)len[k];
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
        nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counts[0], nc);
        atomicAdd(&counts[1], nnz);
    }
}

__global__ void k_column_stats_final(const double *partial, double *frob2) {
    __shared__ double sh[kStatBlocks];
    sh[threadIdx.x] = partial[threadIdx.x];
    __syncthreads();
    for (int o = kStatBlocks / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *frob2 = sh[0];
}

// tol / ||A||_1, the threshold of the fixed drop rule, once per build and block
__global__ void k_tau_fixed(const double *norm1, double tol, double *tau, int32_t nblocks) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblocks) tau[b] = tol / norm1[b];
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 counts into int64 offsets (three passes)

__global__ void k_scan_blocks(const int32_t *in, int64_t n, int64_t *out, int64_t *block_sums) {
    __shared__ int64_t sh[1024];
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    int64_t v = (i < n) ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t t = (threadIdx.x >= (unsigned)o) ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;
    if (threadIdx.x == 1023) block_sums[blockIdx.x] = sh[1023];
}

__global__ void k_scan_sums(int64_t *block_sums, int64_t nb, int64_t *total) {
    // one block: sequential chunks, carried offset
    __shared__ int64_t sh[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        int64_t v = (i < nb) ? block_sums[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int64_t t = (threadIdx.x >= (unsigned)o) ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) block_sums[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *block_sums, const int64_t *total) {
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    if (i < n) out[i] += block_sums[blockIdx.x];
    if (i == 0) out[n] = *total;
}

// ---------------------------------------------------------------------------
// assembly of M: pool segments -> CSC -> CSR (rows sorted by column)

// warp per column: copy the column's pool segment to its CSC slot, count rows
__global__ void k_pool_to_csc(const int64_t *col_off, const int32_t *col_len, const int32_t *pool_rows,
                              const double *pool_vals, const int64_t *Mcolptr, int32_t *Mrows, double *Mvals,
                              int32_t *row_count, int64_t n) {
    int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= n) return;
    int64_t src = col_off[k], dst = Mcolptr[k];
    int len = col_len[k];
    for (int c = lane; c < len; c += 32) {
        int32_t r = pool_rows[src + c];
        Mrows[dst + c] = r;
        Mvals[dst + c] = pool_vals[src + c];
        atomicAdd(&row_count[r], 1);
    }
}

// warp per column: drop each entry into its row (unordered within the row)
__global__ void k_csc_to_rows(const int64_t *Mcolptr, const int32_t *Mrows, const double *Mvals,
                              const int64_t *Mrowptr, int32_t *cursor, int32_t *tcols, double *tvals,
                              int64_t *tsrc, int64_t n) {
    int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= n) return;
    for (int64_t e = Mcolptr[k] + lane; e < Mcolptr[k + 1]; e += 32) {
        int32_t r = Mrows[e];
        int64_t pos = Mrowptr[r] + atomicAdd(&cursor[r], 1);
        tcols[pos] = (int32_t)k;
        tvals[pos] = Mvals[e];
        tsrc[pos] = e;
    }
}

// warp per row: place every entry at its rank among the row's column indices
__global__ void k_sort_rows(const int64_t *Mrowptr, const int32_t *tcols, const double *tvals, const int64_t *tsrc,
                            int32_t *Mcols, double *Mvals_csr, int64_t *csc_to_csr_M, int64_t n) {
    int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (r >= n) return;
    int64_t a = Mrowptr[r], b = Mrowptr[r + 1];
    for (int64_t e = a + lane; e < b; e += 32) {
        int32_t key = tcols[e];
        int64_t rank = 0;
        for (int64_t f = a; f < b; ++f) rank += (tcols[f] < key);
        Mcols[a + rank] = key;
        Mvals_csr[a + rank] = tvals[e];
        csc_to_csr_M[tsrc[e]] = a + rank;
    }
}

// ---------------------------------------------------------------------------
// largest-first order of the global bin's queue (longest processing time
// first, so that the biggest columns do not start last and leave the other
// SMs idle).  Cost proxy of column k: the entries of the rows of A(:,k), i.e.
// the size of the first candidate set of new columns (Algorithm 1);
// columns are bucketed by its bit length, buckets taken in decreasing order.

__global__ void k_cost_buckets(const int32_t *list, const uint32_t *count, const int64_t *col_ptr,
                               const int32_t *row_idx, const int64_t *row_ptr, uint8_t *bucket,
                               uint32_t *hist /* [kCostBuckets] */) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)*count) return;
    const int32_t k = list[t];
    int64_t cost = 0;
    for (int64_t e = col_ptr[k]; e < col_ptr[k + 1]; ++e) {
        const int32_t i = row_idx[e];
        cost += row_ptr[i + 1] - row_ptr[i];
    }
    const int b = min(kCostBuckets - 1, 64 - __clzll((unsigned long long)cost));
    bucket[t] = (uint8_t)b;
    atomicAdd(&hist[b], 1u);
}

// hist -> start offsets, largest bucket first (one warp)
__global__ void k_cost_offsets(uint32_t *hist) {
    const int lane = threadIdx.x;
    uint32_t v = (lane < kCostBuckets) ? hist[kCostBuckets - 1 - lane] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane < kCostBuckets) hist[kCostBuckets - 1 - lane] = incl - v;
}

__global__ void k_cost_scatter(const int32_t *list, const uint32_t *count, const uint8_t *bucket, uint32_t *offset,
                               int32_t *out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)*count) return;
    out[atomicAdd(&offset[bucket[t]], 1u)] = list[t];
}

// adjoint launcher
cudaError_t launch_adjoint_gather(int64_t n, int64_t nnzM, const int64_t *row_ptr, const int32_t *col_idx,
                                  const int64_t *Mrowptr, const int32_t *Mcols, const int64_t *Mcsc_to_csr,
                                  int64_t *Mcsr_to_csc, const int64_t *qoff, const int32_t *poolI,
                                  const double *poolR, const double *poolW, const double *alphaM,
                                  const double *xM, double *grad, cudaStream_t st) {
    if (nnzM > 0) k_invert_map<<<(unsigned)((nnzM + 255) / 256), 256, 0, st>>>(Mcsc_to_csr, nnzM, Mcsr_to_csc);
    int64_t nnzA = 0;
    cudaMemcpyAsync(&nnzA, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return cudaGetLastError();
    if (nnzA > 0)
        k_adjoint_gather<<<(unsigned)((nnzA + 255) / 256), 256, 0, st>>>(n, nnzA, row_ptr, col_idx, Mrowptr, Mcols,
                                                                        Mcsr_to_csc, qoff, poolI, poolR, poolW,
                                                                        alphaM, xM, grad);
    return cudaGetLastError();
}

}  // namespace rsai
