// warp_small.cuh -- register-resident Householder QR and sorts for small LS
// problems on a group of W lanes of one warp (W = 32: a warp per column; W = 16:
// half a warp per column, two columns per warp): |J| = p <= 16, |I| = q <= W*R,
// the common case of stencil matrices.
//
// Lane l of the group holds rows l, l+W, ..., l+(R-1)W of B (R registers per
// column); the loops over the Householder step j and the trailing columns c
// are unrolled so that every register index is a compile-time constant.  The
// (p - j) dot products of a step are all-reduced together over the group.  B
// is read from and written back to the team workspace (column-major, ld = q),
// leaving R above the diagonal and the reflector tails below it, exactly as
// the shared-memory version does, so the solves that follow are unchanged.
// Every shuffle names only the group's own lanes.
#pragma once

#include "common.cuh"

namespace rsai {

constexpr int kSmallP = 16;
constexpr int kSmallQ = 64;  // rows of the 32-lane version (two per lane)

// lanes of the calling thread's group of W lanes (W = 16 or 32)
template <int W> __device__ __forceinline__ unsigned lanes_mask() {
    static_assert(W == 16 || W == 32, "lane groups are half warps or warps");
    if constexpr (W == 32) return 0xffffffffu;
    else return 0xffffu << (threadIdx.x & 16);
}

template <int W, typename T> __device__ __forceinline__ T lanes_sum_t(T x, unsigned mask) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

__host__ __device__ constexpr int ilog2_c(int m) { return m <= 1 ? 0 : 1 + ilog2_c(m >> 1); }

// Square root and quotient of the register QR's Householder steps.  In FP32
// (the factorization that the FP64 refinement step corrects) the hardware
// approximations (rsqrtf, __fdividef, about 2 ulp) replace the correctly
// rounded sequences; in FP64 they stay exact.
__device__ __forceinline__ float qr_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double qr_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float qr_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qr_div(double a, double b) { return a / b; }

// All-reduce of M values (M a power of two <= W) over a group of W lanes: on
// entry lane l holds partial sums x[0..M); on exit every lane holds the M
// totals.  Reduce-scatter by recursive halving (at the level with xor distance
// o the lanes with bit o set keep the upper half of their values, the others
// the lower half, and each adds its partner's copy of the half it keeps), plain
// butterfly levels once a lane holds one value, then an all-gather from the
// lanes that own each total.  M - 1 + (log2 W - log2 M) + M shuffles instead of
// M log2 W for M separate reductions.
template <int M, int W, typename T> __device__ __forceinline__ void lanes_allreduce_vec(T (&x)[M], unsigned mask) {
    static_assert(M <= W, "one value per lane at most after the reduce-scatter");
    constexpr int L = ilog2_c(M);
    constexpr int LW = ilog2_c(W);
    const int lane = threadIdx.x & (W - 1);
#pragma unroll
    for (int lv = 0; lv < L; ++lv) {
        const int o = (W >> 1) >> lv;
        const int h = M >> (lv + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int t = 0; t < h; ++t) {
            const T send = upper ? x[t] : x[t + h];
            const T keep = upper ? x[t + h] : x[t];
            x[t] = keep + __shfl_xor_sync(mask, send, o);
        }
    }
#pragma unroll
    for (int o = (W >> 1) >> L; o > 0; o >>= 1) x[0] += __shfl_xor_sync(mask, x[0], o);
    if (M == 1) return;
    const T mine = x[0];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        int src = 0;
#pragma unroll
        for (int lv = 0; lv < L; ++lv) src |= ((c >> (L - 1 - lv)) & 1) << (LW - 1 - lv);
        x[c] = __shfl_sync(mask, mine, src, W);
    }
}

// One Householder update on the register tile: the dot products of v with
// the trailing columns j+1..15 and with rhs (16 - j values, all-reduced
// together in a block of M >= 16 - j), then C <- C - (2 / v^T v) v (v^T C).
template <int M, int W, int R, typename T>
__device__ __forceinline__ void step_update(int j, T (&b)[R][kSmallP], T (&rr)[R], const T (&v)[R], T two_over,
                                            unsigned mask) {
    T x[M];
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int c = j + 1 + u;
        T acc = T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (c < kSmallP) acc += v[r] * b[r][c];
            else if (c == kSmallP) acc += v[r] * rr[r];
        }
        x[u] = acc;
    }
    lanes_allreduce_vec<M, W>(x, mask);
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int c = j + 1 + u;
        const T f = x[u] * two_over;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (c < kSmallP) b[r][c] -= f * v[r];
            else if (c == kSmallP) rr[r] -= f * v[r];
        }
    }
}

// Householder QR of B (q x p, ld q; q <= W*R, p <= 16) applied to rhs, then back
// substitution into rhs[0..p).  vhead/tau receive v_j(j) and 2 / v_j^T v_j.
// Returns the rank flag.  The back substitution multiplies by reciprocals of
// the diagonal of R formed once, one per lane, instead of dividing at each of
// its steps.
//
// Columns p..15 are zero-filled, so every operation on them is a no-op: the
// unrolled loops run branch-free over all 16 slots; only the steps j >= p are
// skipped.  Not inlined: the unrolled body is large and the column algorithm
// calls the solve from several places.
template <int W, int R, typename T>
__device__ __noinline__ int lanes_qr_small(T *B, int q, int p, T *rhs, T *vhead, T *tau, T small) {
    static_assert(kSmallP <= W, "row i < 16 of R lives in lane i");
    const unsigned mask = lanes_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    T b[R][kSmallP];
    T rr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = lane + W * r;
        const bool have = row < q;
#pragma unroll
        for (int c = 0; c < kSmallP; ++c) b[r][c] = (c < p && have) ? B[c * q + row] : T(0);
        rr[r] = have ? rhs[row] : T(0);
    }
    T dg = T(0);  // R_ll in lane l
    int rank = 0;
#pragma unroll
    for (int j = 0; j < kSmallP; ++j) {
        if (j < p) {
            // reflector of column j over rows >= j (rows >= q hold zeros); row j < W is in r = 0
            T v[R];
            v[0] = (lane >= j) ? b[0][j] : T(0);
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = b[r][j];
            T ss = T(0);
#pragma unroll
            for (int r = 0; r < R; ++r) ss += v[r] * v[r];
            const T sigma = lanes_sum_t<W>(ss, mask);
            const T x0 = __shfl_sync(mask, b[0][j], j, W);
            const T nrm = qr_sqrt(sigma);
            const T alpha = (x0 >= T(0)) ? -nrm : nrm;
            const T vh = x0 - alpha;
            const T vv = sigma - x0 * x0 + vh * vh;
            if (lane == j) v[0] = vh;
            const T two_over = (vv > T(0)) ? qr_div(T(2), vv) : T(0);
            {
                // j is a constant in each unrolled step, so one branch survives
                const int m = kSmallP - j;
                if (m > 8) step_update<16, W, R>(j, b, rr, v, two_over, mask);
                else if (m > 4) step_update<8, W, R>(j, b, rr, v, two_over, mask);
                else if (m > 2) step_update<4, W, R>(j, b, rr, v, two_over, mask);
                else if (m > 1) step_update<2, W, R>(j, b, rr, v, two_over, mask);
                else step_update<1, W, R>(j, b, rr, v, two_over, mask);
            }
            if (lane == j) {
                b[0][j] = alpha;  // R_jj; rows > j keep the reflector tail
                dg = alpha;
            }
            if (lane == 0) {
                vhead[j] = vh;
                tau[j] = two_over;
            }
            rank |= (fabs(alpha) <= small) ? 1 : 0;
        }
    }
    // back substitution on R (row i of R lives in lane i, slot b[0])
    const T rdi = (fabs(dg) <= small) ? T(0) : T(1) / dg;
    T x = T(0);
#pragma unroll
    for (int i = kSmallP - 1; i >= 0; --i) {
        if (i < p) {
            const T ri = __shfl_sync(mask, rdi, i, W);
            const T yi = __shfl_sync(mask, rr[0], i, W);
            const T xi = (ri == T(0)) ? T(0) : yi * ri;
            if (lane == i) x = xi;
            if (lane < i) rr[0] -= b[0][i] * xi;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = lane + W * r;
#pragma unroll
        for (int c = 0; c < kSmallP; ++c)
            if (c < p && row < q) B[c * q + row] = b[r][c];
    }
    if (lane < p) rhs[lane] = x;
    __syncwarp(mask);
    return rank;
}

// rhs <- R^{-1} Q^T rhs with the reflectors left in B, vhead and tau by lanes_qr_small
template <int W, int R, typename T>
__device__ __noinline__ void lanes_apply_qt_small(const T *B, int q, int p, T *rhs, const T *vhead, const T *tau,
                                                  T small) {
    const unsigned mask = lanes_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    T rr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) rr[r] = (lane + W * r < q) ? rhs[lane + W * r] : T(0);
    T rrow[kSmallP];  // row `lane` of R (for the back substitution)
#pragma unroll
    for (int j = 0; j < kSmallP; ++j) {
        const bool live = j < p;
        rrow[j] = (live && lane < q) ? B[j * q + lane] : T(0);
        const T tv = live ? tau[j] : T(0);
        const T vh = live ? vhead[j] : T(0);
        T v[R];
        v[0] = (lane > j) ? rrow[j] : ((lane == j) ? vh : T(0));
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = (live && lane + W * r < q) ? B[j * q + lane + W * r] : T(0);
        T dd = T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) dd += v[r] * rr[r];
        const T d = lanes_sum_t<W>(dd, mask);
        const T f = (tv > T(0)) ? d * tv : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) rr[r] -= f * v[r];
    }
    // reciprocal of R_ll in lane l, as in lanes_qr_small
    const T dl = (lane < p) ? B[lane * q + lane] : T(0);
    const T rdi = (fabs(dl) <= small) ? T(0) : T(1) / dl;
    T x = T(0);
#pragma unroll
    for (int i = kSmallP - 1; i >= 0; --i) {
        if (i < p) {
            const T ri = __shfl_sync(mask, rdi, i, W);
            const T yi = __shfl_sync(mask, rr[0], i, W);
            const T xi = (ri == T(0)) ? T(0) : yi * ri;
            if (lane == i) x = xi;
            if (lane < i) rr[0] -= rrow[i] * xi;
        }
    }
    if (lane < p) rhs[lane] = x;
    __syncwarp(mask);
}

// Bitonic sort of buf[0..len) on a group of W lanes in registers, E elements
// per lane (element e = r*W + lane); len <= W*E.  Ascending, padded with
// INT32_MAX.
template <int W, int E>
__device__ __noinline__ void lanes_sort_regs(int32_t *buf, int len) {
    const unsigned mask = lanes_mask<W>();
    const int lane = threadIdx.x & (W - 1);
    int32_t x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        int e = r * W + lane;
        x[r] = (e < len) ? buf[e] : INT32_MAX;
    }
    constexpr int N = W * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= W) {
                const int jr = j / W;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int rp = r ^ jr;
                    if (rp > r) {
                        const bool up = ((r * W) & k) == 0;
                        int32_t a = x[r], b = x[rp];
                        if ((a > b) == up) { x[r] = b; x[rp] = a; }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int e = r * W + lane;
                    const int32_t other = __shfl_xor_sync(mask, x[r], j);
                    const bool up = (e & k) == 0;
                    const bool lower = (lane & j) == 0;
                    // lower element of an ascending pair keeps the min
                    const bool keep_min = (lower == up);
                    x[r] = keep_min ? min(x[r], other) : max(x[r], other);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) buf[r * W + lane] = x[r];
    __syncwarp(mask);
}

}  // namespace rsai
