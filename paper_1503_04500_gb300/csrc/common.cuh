// common.cuh -- device-side building blocks shared by the RSAI kernels.
//
// A "team" is the group of threads that works on one column of M at a time:
// half a warp (HalfTeam, two columns per warp) or a warp (WarpTeam) for small
// least-squares problems, a whole CTA (BlockTeam) for larger ones.  The column
// algorithm (column.cuh) is written once against this interface: rank()/size,
// sync(), sums, maxima, argmax with a (value desc, index asc) order, exclusive
// scans and a bitonic sort.  lanes_sum() reduces over the team's lanes within
// one warp (the whole team unless it spans several warps).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>

#include "../../include/rsai.h"

namespace rsai {

// ----------------------------------------------------------------------------
// Device view of A (CSR for rows A(i,:), CSC for columns A(:,j); Section 2).
struct DevA {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *val;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *cval;
    const float *cval32;  // FP32 copy of cval for the FP32 QR's gathers (NULL: convert on load)
};

// A(i,j) of CSC entry e in the QR's precision.  The FP32 copy holds the same
// round-to-nearest values that a conversion on load would give.
template <typename T> __device__ __forceinline__ T csc_value(const DevA &A, int64_t e);
template <> __device__ __forceinline__ double csc_value<double>(const DevA &A, int64_t e) { return A.cval[e]; }
template <> __device__ __forceinline__ float csc_value<float>(const DevA &A, int64_t e) {
    return A.cval32 ? A.cval32[e] : __double2float_rn(A.cval[e]);
}

// Parameters as the kernels see them (rsai_params plus derived values).
struct DevParams {
    int c, l_max, drop_mode, precision;
    int init_a;  // initial pattern J_k^(0) of Algorithm 1: 0 = {k}, 1 = rows of A(:,k)
    int spai;    // 1: SPAI's most profitable indices (Eqs. 2.5-2.7) instead of the dominant rows
    double eps, tol, tie_band;
    const double *norm1;       // ||A||_1 per block (one block unless a batch)
    const double *tau_fixed;   // tol / ||A||_1 per block
    const int32_t *col_block;  // block of each column (NULL: one block)
};

// Work counters of one team, summed into the global statistics at the end.
enum Counter {
    CTR_QR = 0, CTR_RES, CTR_REFINE, CTR_REFINE64, CTR_BYTES, CTR_LOOPS, CTR_SOLVES, CTR_DROPS,
    CTR_PMAX, CTR_QMAX, CTR_COLS, CTR_RANK, CTR_NONFINITE, CTR_NC, CTR_FROB2, CTR_FAILED, CTR_SELECT,
    CTR_COUNT
};

// Per-column outputs.
struct ColOut {
    int64_t *col_off;   // offset of the column in the result pool
    int32_t *col_len;   // nnz(m_k)
    int32_t *col_q;     // |I_k| of the final pattern
    double *rho;        // ||r_k||
    int32_t *loops;
    int32_t *flags;     // RSAI_COL_*
    int32_t *pool_rows; // J_k (ascending)
    double *pool_vals;  // m_k(J_k)
    int64_t pool_cap;
    unsigned long long *pool_top;
    int32_t *err;       // first device error code (0 = none)
};

// Frozen-pattern passes (refit, backward): the pattern of M and the buffers
// they read and write.  Unused (NULL) in the build.
enum { MODE_BUILD = 0, MODE_REFIT = 1, MODE_BACKWARD = 2 };
struct Frozen {
    const int64_t *Mcolptr;      // CSC of M: column k is J_k
    const int32_t *Mrows;
    const int64_t *Mcsc_to_csr;  // CSR position of each CSC entry of M
    double *Mval_csr;            // refit: new values of M (CSR order)
    double *rho2;                // refit: ||r_k||^2
    const double *grad_M;        // backward: dL/dM (CSR order of M)
    const double *grad_rho2;     // backward: dL/d(rho_k^2) or NULL
    const int64_t *qoff;         // backward: offset of column k's I_k in the pools
    int32_t *poolI;              // backward: I_k
    double *poolR, *poolW;       // backward: r_k(I_k), (B_k z_k)(I_k)
    double *alphaM, *xM;         // backward: -z + 2 g x and x, per entry of M (CSC order)
};

// Queue of columns for one bin.
struct ColQueue {
    const int32_t *cols;      // explicit list (NULL = 0..n-1)
    const uint32_t *count;    // length of the list on the device (NULL = use n)
    int64_t n;
    uint32_t *next;           // work counter (zeroed before the launch)
    int32_t *ovf_cols;        // where columns that outgrow the bin go
    uint32_t *ovf_count;
    int64_t ovf_cap;
};

// ----------------------------------------------------------------------------
template <typename T> struct Unit;
template <> struct Unit<float> { static constexpr double u = 5.9604644775390625e-08; };
template <> struct Unit<double> { static constexpr double u = 1.1102230246251565e-16; };

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int len, int32_t v) {
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int find_i32(const int32_t *a, int len, int32_t v) {
    int p = lower_bound_i32(a, len, v);
    return (p < len && a[p] == v) ? p : -1;
}

// |x| of a double as an ordered integer key: for x >= 0 the IEEE bit pattern
// orders like the value, so comparisons of magnitudes need no FP64 pipe.
__device__ __forceinline__ long long abskey(double x) {
    return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double key_value(long long k) { return __longlong_as_double(k); }
__device__ __forceinline__ bool finite_bits(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// (a, i) ordered by a descending, then i ascending: true if (a,i) comes first.
__device__ __forceinline__ bool dom_before(long long a, int i, long long b, int j) {
    return a > b || (a == b && i < j);
}

// ----------------------------------------------------------------------------
// Half a warp: lanes 0-15 or 16-31 of a warp work on one column; the two
// halves of a warp run their columns side by side.  Every shuffle and
// synchronisation names only the half's own lanes, so the two halves may
// take different paths through the column algorithm.
struct HalfTeam {
    static constexpr int SIZE = 16;
    static constexpr int LANES = 16;
    unsigned mask;  // this half's lanes
    __device__ __forceinline__ HalfTeam() : mask(0xffffu << (threadIdx.x & 16)) {}
    __device__ __forceinline__ int rank() const { return threadIdx.x & 15; }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    template <typename V> __device__ __forceinline__ V sum(V x) const {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
        return x;
    }
    template <typename V> __device__ __forceinline__ V lanes_sum(V x) const { return sum(x); }
    template <typename V> __device__ __forceinline__ V maxv(V x) const {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            V y = __shfl_xor_sync(mask, x, o);
            x = y > x ? y : x;
        }
        return x;
    }
    __device__ __forceinline__ void argmax(long long &a, int &i) const {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            long long b = __shfl_xor_sync(mask, a, o);
            int j = __shfl_xor_sync(mask, i, o);
            if (dom_before(b, j, a, i)) { a = b; i = j; }
        }
    }
    __device__ __forceinline__ int scan(int x, int *total) const {
        const int lane = rank();
        int inc = x;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            int y = __shfl_up_sync(mask, inc, o, 16);
            if (lane >= o) inc += y;
        }
        *total = __shfl_sync(mask, inc, 15, 16);
        return inc - x;
    }
    template <typename V> __device__ __forceinline__ V bcast(V x, int src) const {
        return __shfl_sync(mask, x, src, 16);
    }
};

struct WarpTeam {
    static constexpr int SIZE = 32;
    static constexpr int LANES = 32;
    static constexpr unsigned mask = 0xffffffffu;
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    template <typename V> __device__ __forceinline__ V sum(V x) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return x;
    }
    template <typename V> __device__ __forceinline__ V lanes_sum(V x) const { return sum(x); }
    template <typename V> __device__ __forceinline__ V maxv(V x) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            V y = __shfl_xor_sync(0xffffffffu, x, o);
            x = y > x ? y : x;
        }
        return x;
    }
    // argmax under dom_before; returns the winner to every lane
    __device__ __forceinline__ void argmax(long long &a, int &i) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            long long b = __shfl_xor_sync(0xffffffffu, a, o);
            int j = __shfl_xor_sync(0xffffffffu, i, o);
            if (dom_before(b, j, a, i)) { a = b; i = j; }
        }
    }
    // exclusive prefix sum over ranks; *total gets the sum
    __device__ __forceinline__ int scan(int x, int *total) const {
        int lane = rank();
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        *total = __shfl_sync(0xffffffffu, inc, 31);
        return inc - x;
    }
    template <typename V> __device__ __forceinline__ V bcast(V x, int src) const {
        return __shfl_sync(0xffffffffu, x, src);
    }
};

// A whole CTA of NT threads; `red` is NT/32+1 words of shared scratch (8 bytes
// each, holding any reduced type), `redi` as many ints.
template <int NT> struct BlockTeam {
    static constexpr int SIZE = NT;
    static constexpr int LANES = 32;
    static constexpr int NW = NT / 32;
    unsigned long long *red;
    int *redi;
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    // sum over the 32 lanes of the calling warp only
    template <typename V> __device__ __forceinline__ V lanes_sum(V x) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return x;
    }
    template <typename V> __device__ __forceinline__ V &slot(int w) const { return *reinterpret_cast<V *>(&red[w]); }
    template <typename V> __device__ __forceinline__ V sum(V x) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) slot<V>(threadIdx.x >> 5) = x;
        __syncthreads();
        V s = slot<V>(0);
#pragma unroll
        for (int w = 1; w < NW; ++w) s += slot<V>(w);
        return s;
    }
    template <typename V> __device__ __forceinline__ V maxv(V x) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            V y = __shfl_xor_sync(0xffffffffu, x, o);
            x = y > x ? y : x;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) slot<V>(threadIdx.x >> 5) = x;
        __syncthreads();
        V s = slot<V>(0);
#pragma unroll
        for (int w = 1; w < NW; ++w) s = slot<V>(w) > s ? slot<V>(w) : s;
        return s;
    }
    __device__ __forceinline__ void argmax(long long &a, int &i) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            long long b = __shfl_xor_sync(0xffffffffu, a, o);
            int j = __shfl_xor_sync(0xffffffffu, i, o);
            if (dom_before(b, j, a, i)) { a = b; i = j; }
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { slot<long long>(threadIdx.x >> 5) = a; redi[threadIdx.x >> 5] = i; }
        __syncthreads();
        a = slot<long long>(0);
        i = redi[0];
#pragma unroll
        for (int w = 1; w < NW; ++w)
            if (dom_before(slot<long long>(w), redi[w], a, i)) { a = slot<long long>(w); i = redi[w]; }
    }
    __device__ __forceinline__ int scan(int x, int *total) const {
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        __syncthreads();
        if (lane == 31) redi[w] = inc;
        __syncthreads();
        int before = 0, tot = 0;
#pragma unroll
        for (int v = 0; v < NW; ++v) {
            int s = redi[v];
            if (v < w) before += s;
            tot += s;
        }
        *total = tot;
        return before + inc - x;
    }
    template <typename V> __device__ __forceinline__ V bcast(V x, int src) const {
        __syncthreads();
        if ((int)threadIdx.x == src) slot<V>(NW) = x;
        __syncthreads();
        return slot<V>(NW);
    }
};

// Teams that fit in one warp (one column per warp or half-warp): register QR
// and register sorts, no kept factor between loops.
template <class Team> struct is_lane_team { static constexpr bool value = false; };
template <> struct is_lane_team<WarpTeam> { static constexpr bool value = true; };
template <> struct is_lane_team<HalfTeam> { static constexpr bool value = true; };

// Bitonic sort of buf[0..len) ascending in shared memory; buf must have room
// for the next power of two (padded with INT32_MAX).
template <class Team>
__device__ __noinline__ void team_sort_i32_smem(Team team, int32_t *buf, int len) {
    int N = 1;
    while (N < len) N <<= 1;
    for (int i = len + team.rank(); i < N; i += Team::SIZE) buf[i] = INT32_MAX;
    team.sync();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = team.rank(); i < N; i += Team::SIZE) {
                int ixj = i ^ j;
                if (ixj > i) {
                    int32_t a = buf[i], b = buf[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) { buf[i] = b; buf[ixj] = a; }
                }
            }
            team.sync();
        }
    }
}

// out = unique(sorted in[0..len)); returns the count (identical on all ranks).
template <class Team>
__device__ int team_unique_i32(const Team &team, const int32_t *in, int len, int32_t *out) {
    int base = 0;
    for (int c0 = 0; c0 < len; c0 += Team::SIZE) {
        int i = c0 + team.rank();
        int f = (i < len) && (i == 0 || in[i] != in[i - 1]);
        int tot;
        int pos = team.scan(f, &tot);
        if (f) out[base + pos] = in[i];
        base += tot;
    }
    team.sync();
    return base;
}

__device__ __forceinline__ void set_error(int32_t *err, int code) {
    atomicCAS(err, 0, code);
}

}  // namespace rsai
