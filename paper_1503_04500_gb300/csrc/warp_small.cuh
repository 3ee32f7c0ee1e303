// warp_small.cuh -- register-resident Householder QR for small LS problems on
// one warp (|J| = p <= 16, |I| = q <= 64), the common case of stencil
// matrices.
//
// Lane l holds rows l and l+32 of B (two registers per column); the loops over
// the Householder step j and the trailing columns c are unrolled so that every
// register index is a compile-time constant.  The (p - j) dot products of a
// step are independent warp reductions that the compiler interleaves.  B is
// read from and written back to the team workspace (column-major, ld = q),
// leaving R above the diagonal and the reflector tails below it, exactly as the
// shared-memory version does, so the solves that follow are unchanged.
#pragma once

#include "common.cuh"

namespace rsai {

constexpr int kSmallP = 16;
constexpr int kSmallQ = 64;

template <typename T> __device__ __forceinline__ T warp_sum_t(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
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

// All-reduce of M values (M a power of two <= 32) over the warp: on entry
// lane l holds partial sums x[0..M); on exit every lane holds the M totals.
// Reduce-scatter by recursive halving (at the level with xor distance o the
// lanes with bit o set keep the upper half of their values, the others the
// lower half, and each adds its partner's copy of the half it keeps), plain
// butterfly levels once a lane holds one value, then an all-gather from the
// lanes that own each total.  M - 1 + (5 - log2 M) + M shuffles and
// 4 + M - log2 M additions instead of 5 M of each for M separate reductions.
template <int M, typename T> __device__ __forceinline__ void warp_allreduce_vec(T (&x)[M]) {
    constexpr int L = ilog2_c(M);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int lv = 0; lv < L; ++lv) {
        const int o = 16 >> lv;
        const int h = M >> (lv + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int t = 0; t < h; ++t) {
            const T send = upper ? x[t] : x[t + h];
            const T keep = upper ? x[t + h] : x[t];
            x[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 >> L; o > 0; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
    if (M == 1) return;
    const T mine = x[0];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        int src = 0;
#pragma unroll
        for (int lv = 0; lv < L; ++lv) src |= ((c >> (L - 1 - lv)) & 1) << (4 - lv);
        x[c] = __shfl_sync(0xffffffffu, mine, src);
    }
}

// One Householder update on the register tile: the dot products of v with
// the trailing columns j+1..15 and with rhs (16 - j values, all-reduced
// together in a block of M >= 16 - j), then C <- C - (2 / v^T v) v (v^T C).
template <int M, typename T>
__device__ __forceinline__ void step_update(int j, T (&b0)[kSmallP], T (&b1)[kSmallP], T &r0, T &r1, T v0, T v1,
                                            T two_over) {
    T x[M];
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int c = j + 1 + u;
        x[u] = (c < kSmallP) ? v0 * b0[c] + v1 * b1[c] : ((c == kSmallP) ? v0 * r0 + v1 * r1 : T(0));
    }
    warp_allreduce_vec<M>(x);
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int c = j + 1 + u;
        const T f = x[u] * two_over;
        if (c < kSmallP) {
            b0[c] -= f * v0;
            b1[c] -= f * v1;
        } else if (c == kSmallP) {
            r0 -= f * v0;
            r1 -= f * v1;
        }
    }
}

// Householder QR of B (q x p, ld q) applied to rhs, then back substitution into
// rhs[0..p).  vhead/tau receive v_j(j) and 2 / v_j^T v_j.  Returns the rank
// flag.  The back substitution multiplies by reciprocals of the diagonal of R
// formed once, one per lane, instead of dividing at each of its steps.
//
// Columns p..15 are zero-filled, so every operation on them is a no-op: the
// unrolled loops run branch-free over all 16 slots; only the steps j >= p are
// skipped.  Not inlined: the unrolled body is large and the column algorithm
// calls the solve from several places.
template <typename T>
__device__ __noinline__ int warp_qr_small(T *B, int q, int p, T *rhs, T *vhead, T *tau, T small) {
    const int lane = threadIdx.x & 31;
    const bool h0 = lane < q, h1 = lane + 32 < q;
    T b0[kSmallP], b1[kSmallP];
#pragma unroll
    for (int c = 0; c < kSmallP; ++c) {
        b0[c] = (c < p && h0) ? B[c * q + lane] : T(0);
        b1[c] = (c < p && h1) ? B[c * q + lane + 32] : T(0);
    }
    T r0 = h0 ? rhs[lane] : T(0);
    T r1 = h1 ? rhs[lane + 32] : T(0);
    T dg = T(0);  // R_ll in lane l
    int rank = 0;
#pragma unroll
    for (int j = 0; j < kSmallP; ++j) {
        if (j < p) {
            // reflector of column j over rows >= j (rows >= q hold zeros)
            T v0 = (lane >= j) ? b0[j] : T(0);
            T v1 = b1[j];
            const T sigma = warp_sum_t(v0 * v0 + v1 * v1);
            const T x0 = __shfl_sync(0xffffffffu, b0[j], j);
            const T nrm = qr_sqrt(sigma);
            const T alpha = (x0 >= T(0)) ? -nrm : nrm;
            const T vh = x0 - alpha;
            const T vv = sigma - x0 * x0 + vh * vh;
            if (lane == j) v0 = vh;
            const T two_over = (vv > T(0)) ? qr_div(T(2), vv) : T(0);
            {
                // j is a constant in each unrolled step, so one branch survives
                const int m = kSmallP - j;
                if (m > 8) step_update<16>(j, b0, b1, r0, r1, v0, v1, two_over);
                else if (m > 4) step_update<8>(j, b0, b1, r0, r1, v0, v1, two_over);
                else if (m > 2) step_update<4>(j, b0, b1, r0, r1, v0, v1, two_over);
                else if (m > 1) step_update<2>(j, b0, b1, r0, r1, v0, v1, two_over);
                else step_update<1>(j, b0, b1, r0, r1, v0, v1, two_over);
            }
            if (lane == j) {
                b0[j] = alpha;  // R_jj; rows > j keep the reflector tail
                dg = alpha;
            }
            if (lane == 0) {
                vhead[j] = vh;
                tau[j] = two_over;
            }
            rank |= (fabs(alpha) <= small) ? 1 : 0;
        }
    }
    // back substitution on R (row i of R lives in lane i, slot b0)
    const T rdi = (fabs(dg) <= small) ? T(0) : T(1) / dg;
    T x = T(0);
#pragma unroll
    for (int i = kSmallP - 1; i >= 0; --i) {
        if (i < p) {
            const T ri = __shfl_sync(0xffffffffu, rdi, i);
            const T yi = __shfl_sync(0xffffffffu, r0, i);
            const T xi = (ri == T(0)) ? T(0) : yi * ri;
            if (lane == i) x = xi;
            if (lane < i) r0 -= b0[i] * xi;
        }
    }
#pragma unroll
    for (int c = 0; c < kSmallP; ++c) {
        if (c < p) {
            if (h0) B[c * q + lane] = b0[c];
            if (h1) B[c * q + lane + 32] = b1[c];
        }
    }
    if (lane < p) rhs[lane] = x;
    __syncwarp();
    return rank;
}

// rhs <- R^{-1} Q^T rhs with the reflectors left in B, vhead and tau by warp_qr_small
template <typename T>
__device__ __noinline__ void warp_apply_qt_small(const T *B, int q, int p, T *rhs, const T *vhead, const T *tau,
                                                 T small) {
    const int lane = threadIdx.x & 31;
    const bool h0 = lane < q, h1 = lane + 32 < q;
    T r0 = h0 ? rhs[lane] : T(0);
    T r1 = h1 ? rhs[lane + 32] : T(0);
    T rrow[kSmallP];  // row `lane` of R (for the back substitution)
#pragma unroll
    for (int j = 0; j < kSmallP; ++j) {
        const bool live = j < p;
        rrow[j] = (live && h0) ? B[j * q + lane] : T(0);
        const T tv = live ? tau[j] : T(0);
        const T vh = live ? vhead[j] : T(0);
        T v0 = (lane > j) ? rrow[j] : ((lane == j) ? vh : T(0));
        T v1 = (live && h1) ? B[j * q + lane + 32] : T(0);
        const T d = warp_sum_t(v0 * r0 + v1 * r1);
        const T f = (tv > T(0)) ? d * tv : T(0);
        r0 -= f * v0;
        r1 -= f * v1;
    }
    // reciprocal of R_ll in lane l, as in warp_qr_small
    const T dl = (lane < p) ? B[lane * q + lane] : T(0);
    const T rdi = (fabs(dl) <= small) ? T(0) : T(1) / dl;
    T x = T(0);
#pragma unroll
    for (int i = kSmallP - 1; i >= 0; --i) {
        if (i < p) {
            const T ri = __shfl_sync(0xffffffffu, rdi, i);
            const T yi = __shfl_sync(0xffffffffu, r0, i);
            const T xi = (ri == T(0)) ? T(0) : yi * ri;
            if (lane == i) x = xi;
            if (lane < i) r0 -= rrow[i] * xi;
        }
    }
    if (lane < p) rhs[lane] = x;
    __syncwarp();
}

// Bitonic sort of buf[0..len) on one warp in registers, E elements per lane
// (element e = r*32 + lane); len <= 32*E.  Ascending, padded with INT32_MAX.
template <int E>
__device__ __noinline__ void warp_sort_regs(int32_t *buf, int len) {
    const int lane = threadIdx.x & 31;
    int32_t x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        int e = r * 32 + lane;
        x[r] = (e < len) ? buf[e] : INT32_MAX;
    }
    constexpr int N = 32 * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j >> 5;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int rp = r ^ jr;
                    if (rp > r) {
                        const bool up = ((r * 32) & k) == 0;
                        int32_t a = x[r], b = x[rp];
                        if ((a > b) == up) { x[r] = b; x[rp] = a; }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int e = r * 32 + lane;
                    const int32_t other = __shfl_xor_sync(0xffffffffu, x[r], j);
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
    for (int r = 0; r < E; ++r) buf[r * 32 + lane] = x[r];
    __syncwarp();
}

}  // namespace rsai
