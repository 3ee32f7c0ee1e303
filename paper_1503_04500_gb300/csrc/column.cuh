// column.cuh -- one column of RSAI(tol) on one team (warp or CTA).
//
// Per column k (Section 3 Algorithm 1, Section 4 Eq. 4.3):
//   J = {k}, R = {}, l = 0
//   solve(J); drop(J); r = A m - e_k on S = I u {k}; rho = ||r||
//   while rho > eps and l < l_max:
//     Rhat = top-c of {i in S : |r_i| > band, i not in R} by (|r_i| desc, i asc)
//            with a tie band; R += Rhat                        (Eq. 3.2)
//     Jhat = cols(A(Rhat,:)) \ J
//     l += 1; if Jhat is empty: continue
//     J += Jhat; solve(J); drop(J); residual                   (Eq. 4.3)
//
// solve(J): I = rows of A(:,J) (Section 2), B = A(I,J) gathered into the team's
// workspace (column-major, leading dimension q), e = e_k(I), Householder QR of
// B applied to e, back substitution (Eq. 2.3).  In RSAI_FP32_REFINE the QR runs
// in float; the residual of the float solution is formed in double from the
// sparse columns of A, one correction is solved with the float factors and
// added in double.  The residual r_k, its norm, the dominant-row choice, the
// drop test and the stopping test are double in both precisions.
//
// A column whose problem outgrows the team's workspace returns OVERFLOW; the
// caller hands it to the next (larger) bin, which restarts it from J = {k}.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "warp_small.cuh"

namespace rsai {

struct Caps {
    int qcap;      // max |I| (rows of the LS problem); |S| <= qcap + 1
    int pcap;      // max |J|
    int scap;      // sort buffer (power of two)
    int rcap;      // max |R| (dominant rows used so far)
    int64_t bcap;  // max q*p elements of B
    int hcap;      // slots of the J -> position hash (power of two >= 2*pcap), 0 = none
    int small_p;   // largest |J| solved by the register-resident warp QR (0: never)
    int stage_bytes;  // shared memory for staging QR panels (global-memory bins), 0 = none
    int append;       // CTA bins: keep the factor between loops and append to it (Section 3)
    int dcap;         // max number of distinct columns dropped from J (they are not charged again on re-entry)
    int spai;         // SPAI selection: a score per candidate column (scap of them)
};

// Columns of one compact-WY panel (global-memory bins)
constexpr int kPanel = 16;

template <typename T> struct Work {
    T *B, *vhead, *tau, *rhs;
    double *m, *r, *z, *wv;
    long long *ctr;
    int32_t *I, *S, *J, *Jn, *Rset, *buf, *buf2, *Rhat, *hkey, *hval;
    int32_t *D;        // columns dropped from J so far, ascending
    double *sc;        // SPAI: the score s_j of each candidate (Caps::spai)
    int32_t *Ip, *Jp;  // factor position of each sorted I / J entry (Caps::append)
    T *qte;            // Q^T e_k(I) of the kept factor, factor row order (Caps::append)
    // Global-memory bins (Caps::stage_bytes > 0): the reflectors as factored,
    // in panels: pnb[j0] reflectors start at j0, and column j of the panel's
    // compact-WY T (H_j0 ... H_j0+nb-1 = I - V T V^T) is Tst[j * kPanel + s],
    // s <= j - j0.  A reflector factored on its own is a panel of one, T = tau.
    T *Tst;
    int32_t *pnb;
    char *stage = nullptr;  // panel staging area (shared memory), not part of the carved workspace

    __host__ __device__ static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
    __host__ __device__ static size_t bytes(const Caps &c) {
        size_t b = 0;
        b += align16(sizeof(T) * (size_t)c.bcap);
        b += 2 * align16(sizeof(T) * (size_t)c.pcap);
        b += align16(sizeof(T) * (size_t)(c.qcap + 1));
        b += align16(sizeof(double) * (size_t)c.pcap);
        b += align16(sizeof(double) * (size_t)(c.qcap + 1));
        b += align16(sizeof(double) * (size_t)c.pcap);
        b += align16(sizeof(double) * (size_t)(c.qcap + 1));
        b += align16(sizeof(long long) * CTR_COUNT);
        b += align16(sizeof(int32_t) * (size_t)c.qcap);
        b += align16(sizeof(int32_t) * (size_t)(c.qcap + 1));
        b += 2 * align16(sizeof(int32_t) * (size_t)c.pcap);
        b += align16(sizeof(int32_t) * (size_t)c.rcap);
        b += 2 * align16(sizeof(int32_t) * (size_t)c.scap);
        b += align16(sizeof(int32_t) * 32);
        b += 2 * align16(sizeof(int32_t) * (size_t)c.hcap);
        b += align16(sizeof(int32_t) * (size_t)c.dcap);
        if (c.spai) b += align16(sizeof(double) * (size_t)c.scap);
        if (c.append) {
            b += align16(sizeof(int32_t) * (size_t)c.qcap);
            b += align16(sizeof(int32_t) * (size_t)c.pcap);
            b += align16(sizeof(T) * (size_t)(c.qcap + 1));
        }
        if (c.stage_bytes > 0) {
            b += align16(sizeof(T) * (size_t)c.pcap * kPanel);
            b += align16(sizeof(int32_t) * (size_t)c.pcap);
        }
        return b;
    }
    __device__ void carve(char *base, const Caps &c) {
        size_t o = 0;
        B = (T *)(base + o); o += align16(sizeof(T) * (size_t)c.bcap);
        vhead = (T *)(base + o); o += align16(sizeof(T) * (size_t)c.pcap);
        tau = (T *)(base + o); o += align16(sizeof(T) * (size_t)c.pcap);
        rhs = (T *)(base + o); o += align16(sizeof(T) * (size_t)(c.qcap + 1));
        m = (double *)(base + o); o += align16(sizeof(double) * (size_t)c.pcap);
        r = (double *)(base + o); o += align16(sizeof(double) * (size_t)(c.qcap + 1));
        z = (double *)(base + o); o += align16(sizeof(double) * (size_t)c.pcap);
        wv = (double *)(base + o); o += align16(sizeof(double) * (size_t)(c.qcap + 1));
        ctr = (long long *)(base + o); o += align16(sizeof(long long) * CTR_COUNT);
        I = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.qcap);
        S = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)(c.qcap + 1));
        J = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.pcap);
        Jn = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.pcap);
        Rset = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.rcap);
        buf = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.scap);
        buf2 = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.scap);
        Rhat = (int32_t *)(base + o); o += align16(sizeof(int32_t) * 32);
        hkey = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.hcap);
        hval = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.hcap);
        D = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.dcap);
        sc = nullptr;
        if (c.spai) {
            sc = (double *)(base + o); o += align16(sizeof(double) * (size_t)c.scap);
        }
        Ip = Jp = nullptr;
        qte = nullptr;
        if (c.append) {
            Ip = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.qcap);
            Jp = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.pcap);
            qte = (T *)(base + o); o += align16(sizeof(T) * (size_t)(c.qcap + 1));
        }
        Tst = nullptr;
        pnb = nullptr;
        if (c.stage_bytes > 0) {
            Tst = (T *)(base + o); o += align16(sizeof(T) * (size_t)c.pcap * kPanel);
            pnb = (int32_t *)(base + o); o += align16(sizeof(int32_t) * (size_t)c.pcap);
        }
    }
};

enum ColStatus { COL_DONE = 0, COL_OVERFLOW = 1 };

// Entries of a CSR row loaded together in the row-driven loops
constexpr int kRowGroup = 4;

// Rows per lane of the register QR: q <= 64 on a warp, q <= 48 on half a warp
template <class Team> constexpr int kRegRows = Team::SIZE == 16 ? 3 : 2;

// Sort buf[0..len) ascending: registers and shuffles on a warp or half warp
// (up to 256 elements), bitonic in shared memory otherwise.
template <class Team>
__device__ void team_sort_i32(const Team &team, int32_t *buf, int len) {
    if constexpr (is_lane_team<Team>::value) {
        constexpr int W = Team::SIZE;
        if (len <= W) { lanes_sort_regs<W, 1>(buf, len); return; }
        if (len <= 2 * W) { lanes_sort_regs<W, 2>(buf, len); return; }
        if (len <= 4 * W) { lanes_sort_regs<W, 4>(buf, len); return; }
        if (len <= 8 * W) { lanes_sort_regs<W, 8>(buf, len); return; }
        if constexpr (W == 16) {
            if (len <= 16 * W) { lanes_sort_regs<W, 16>(buf, len); return; }
        }
    }
    team_sort_i32_smem(team, buf, len);
}

__host__ __device__ inline int next_pow2(int x) {
    int n = 1;
    while (n < x) n <<= 1;
    return n;
}

// Algorithmic flops of one solve on (q,p) appended to a factorisation of
// (q0,p0) (p0 = 0: from scratch): the reflectors of the old columns applied to
// the new ones, Householder steps p0..p-1 on the stacked rows (norm, then every
// trailing column and the right-hand side), and the back substitution.
__device__ __forceinline__ long long solve_flops(long long q0, long long p0, long long q, long long p) {
    long long mm = p - p0;
    long long f = 4 * mm * (p0 * q0 - p0 * (p0 - 1) / 2);
    long long s2 = mm * (mm + 1) * (2 * mm + 1) / 6;
    f += (q - p) * (2 * mm + 2 * mm * (mm + 1)) + mm * (mm + 1) + 4 * s2;
    return f + p * p;
}

// rhs[0..p) <- R^{-1} rhs[0..p) (column-oriented, in place)
template <class Team, typename T>
__device__ void back_substitute_team(const Team &team, const T *B, int q, int p, T *rhs, T small) {
    const int me = team.rank();
    for (int i = p - 1; i >= 0; --i) {
        T d = B[(int64_t)i * q + i];
        T xi = (fabs(d) <= small) ? T(0) : rhs[i] / d;
        team.sync();
        for (int c = me; c < i; c += Team::SIZE) rhs[c] -= B[(int64_t)i * q + c] * xi;
        if (me == 0) rhs[i] = xi;
        team.sync();
    }
}

// Householder QR of B (q x p, column-major, ld q) applied to rhs, then back
// substitution into rhs[0..p).  Keeps the reflectors (v_j below the diagonal
// of B, heads in vhead, tau = 2 / v^T v in tau) for the refinement solve.  Returns the
// rank flag.  Team-generic: the norm of the pivot column is one team
// reduction; the trailing columns (and rhs) are dealt out to the team's warps,
// each warp forming its column's dot product with the reflector (lanes over
// rows, one warp reduction) and applying the update itself, so a step costs
// one team synchronisation instead of one per column.  Not inlined.
// One Householder step j on B (q x p, ld q) and rhs: the reflector of column j
// over rows >= j, applied to the columns c in [c_begin, p) and to rhs.  The
// norm is one team reduction; the columns are dealt out to the team's warps,
// each warp forming its column's dot product (lanes over rows, one warp
// reduction) and applying the update itself.  Stores R_jj, v_j(j), v_j^T v_j.
template <class Team, typename T>
__device__ __forceinline__ void householder_step(const Team &team, T *B, int q, int p, T *rhs, T *vhead, T *taus,
                                                 int j, int c_begin, T small, int &rank_flag) {
    const int me = team.rank();
    constexpr int LN = Team::LANES;  // lanes of one group: the team itself, or one warp of a CTA
    constexpr int NW = Team::SIZE / LN;
    const int lane = me % LN, wid = me / LN;
    T *col = B + (int64_t)j * q;
    T part = 0;
    for (int i = j + me; i < q; i += Team::SIZE) part += col[i] * col[i];
    const T sigma = team.sum(part);
    const T x0 = col[j];
    const T nrm = sqrt(sigma);
    const T alpha = (x0 >= T(0)) ? -nrm : nrm;
    const T v0 = x0 - alpha;
    const T vtv = sigma - x0 * x0 + v0 * v0;
    const T two_over = (vtv > T(0)) ? T(2) / vtv : T(0);
    if (two_over > T(0)) {
        for (int c = c_begin + wid; c <= p; c += NW) {
            T *t = (c < p) ? B + (int64_t)c * q : rhs;
            T d = 0;
            for (int i = j + lane; i < q; i += LN) d += ((i == j) ? v0 : col[i]) * t[i];
            d = team.lanes_sum(d);
            const T f = d * two_over;
            for (int i = j + lane; i < q; i += LN) t[i] -= f * ((i == j) ? v0 : col[i]);
        }
    }
    team.sync();
    if (me == 0) {
        col[j] = alpha;
        vhead[j] = v0;
        taus[j] = two_over;
    }
    rank_flag |= (fabs(alpha) <= small) ? 1 : 0;
    team.sync();
}

// Householder QR of B (q x p, column-major, ld q) applied to rhs, then back
// substitution into rhs[0..p).  Keeps the reflectors (v_j below the diagonal
// of B, heads in vhead, tau = 2 / v^T v in tau) for the refinement solve.  Returns the
// rank flag.  Team-generic, one team synchronisation per step; not inlined.
template <class Team, typename T>
__device__ __noinline__ int qr_solve_team(Team team, T *B, int q, int p, T *rhs, T *vhead, T *taus, T small) {
    int rank_flag = 0;
    for (int j = 0; j < p; ++j) householder_step(team, B, q, p, rhs, vhead, taus, j, j + 1, small, rank_flag);
    back_substitute_team(team, B, q, p, rhs, small);
    return rank_flag;
}

// Householder steps j_start..p-1 on B and rhs, no back substitution (rhs is
// left holding Q^T rhs): a factor from scratch (j_start = 0) that is kept for
// later updates, or the appended block of the QR update.  Not inlined.
template <class Team, typename T>
__device__ __noinline__ int qr_factor_team(Team team, T *B, int q, int p, T *rhs, T *vhead, T *taus, T small,
                                           int j_start) {
    int rank_flag = 0;
    for (int j = j_start; j < p; ++j) householder_step(team, B, q, p, rhs, vhead, taus, j, j + 1, small, rank_flag);
    return rank_flag;
}

// Compact-WY pieces shared by the panel factorization and the QR update.
// V: nb explicit reflectors (zeros above the diagonal, heads on it) of
// length qq in shared memory, ld qq; taus: their 2 / v^T v.  wy_form_T forms
// T from V alone; the staged factorization forms it alongside instead
// (panel_factor_fused), so wy_form_T has no caller at present.
// T (kPanel x kPanel in tm) of H_0 ... H_{nb-1} = I - V T V^T:
// y(s,t) = v_s^T v_t (s < t), then column by column
// T(t,t) = tau_t, T(0:t, t) = -tau_t T(0:t, 0:t) y(0:t, t).
template <class Team, typename T>
__device__ __forceinline__ void wy_form_T(const Team &team, const T *V, int qq, int nb, const T *taus, T *tm) {
    const int me = team.rank();
    const int lane = me & 31, wid = me >> 5;
    constexpr int NW = (Team::SIZE + 31) / 32;
    for (int pair = wid; pair < nb * nb; pair += NW) {
        const int s_ = pair / nb, t_ = pair - s_ * nb;
        if (s_ >= t_) continue;
        const T *vs = V + (int64_t)s_ * qq, *vt = V + (int64_t)t_ * qq;
        T d = 0;
        for (int r = t_ + lane; r < qq; r += 32) d += vs[r] * vt[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) tm[s_ * kPanel + t_] = d;
    }
    team.sync();
    for (int t = 0; t < nb; ++t) {
        const T tau = taus[t];
        T val = T(0);
        if (me < t) {
            T acc = 0;
            for (int s2 = me; s2 < t; ++s2) acc += tm[me * kPanel + s2] * tm[s2 * kPanel + t];
            val = -tau * acc;
        }
        team.sync();
        if (me < t) tm[me * kPanel + t] = val;
        if (me == t) tm[t * kPanel + t] = tau;
        team.sync();
    }
}

// Columns c in [c_lo, c_hi] of B (ld q; c == p stands for rhs), rows
// j0..j0+qq-1: C <- C - V (T^T (V^T C)).  Each warp takes kCols columns at a
// time (four in FP32, two in FP64) so that every reflector value read from
// shared memory serves kCols columns, kRows rows per lane and pass.  A pass
// over kRows full rows of a full panel takes a path without per-element bounds
// tests (a warp's missing columns read its first column again and store
// nothing).  Ends with a team synchronisation.
template <class Team, typename T>
__device__ __forceinline__ void wy_apply(const Team &team, const T *V, int qq, int nb, const T *tm, T *B, int q,
                                         int p, T *rhs, int j0, int c_lo, int c_hi) {
    const int me = team.rank();
    const int lane = me & 31, wid = me >> 5;
    constexpr int NW = (Team::SIZE + 31) / 32;
    constexpr int kCols = sizeof(T) == 8 ? 2 : 4;  // W of kCols x kPanel values stays in registers
    constexpr int kRows = 4;
    const bool full_panel = nb == kPanel;
    for (int c0 = c_lo + wid * kCols; c0 <= c_hi; c0 += NW * kCols) {
        T *tc[kCols];
        bool has[kCols];
#pragma unroll
        for (int x = 0; x < kCols; ++x) {
            const int c = c0 + x;
            has[x] = c <= c_hi;
            tc[x] = !has[x] ? nullptr : ((c < p) ? B + (int64_t)c * q + j0 : rhs + j0);
        }
        T *tf[kCols];  // the fast path's columns: a missing one reads column c0
#pragma unroll
        for (int x = 0; x < kCols; ++x) tf[x] = has[x] ? tc[x] : tc[0];
        const bool all_cols = full_panel;  // every present column on the fast path
        T wv[kCols][kPanel];
#pragma unroll
        for (int x = 0; x < kCols; ++x)
#pragma unroll
            for (int u = 0; u < kPanel; ++u) wv[x][u] = T(0);
        // W = V^T C; kRows rows per pass (r, r + 32, ...), their loads issued before any use
        for (int r = lane; r < qq; r += 32 * kRows) {
            T cr[kRows][kCols];
            if (all_cols && r + 32 * (kRows - 1) < qq) {
#pragma unroll
                for (int y = 0; y < kRows; ++y)
#pragma unroll
                    for (int x = 0; x < kCols; ++x) cr[y][x] = tf[x][r + 32 * y];
#pragma unroll
                for (int u = 0; u < kPanel; ++u) {
                    const T *vu = V + (int64_t)u * qq + r;
                    T v[kRows];
#pragma unroll
                    for (int y = 0; y < kRows; ++y) v[y] = vu[32 * y];
#pragma unroll
                    for (int x = 0; x < kCols; ++x)
#pragma unroll
                        for (int y = 0; y < kRows; ++y) wv[x][u] += v[y] * cr[y][x];
                }
                continue;
            }
#pragma unroll
            for (int y = 0; y < kRows; ++y)
#pragma unroll
                for (int x = 0; x < kCols; ++x) cr[y][x] = (tc[x] && r + 32 * y < qq) ? tc[x][r + 32 * y] : T(0);
#pragma unroll
            for (int u = 0; u < kPanel; ++u) {
                if (u < nb) {
                    T v[kRows];
#pragma unroll
                    for (int y = 0; y < kRows; ++y) v[y] = (r + 32 * y < qq) ? V[(int64_t)u * qq + r + 32 * y] : T(0);
#pragma unroll
                    for (int x = 0; x < kCols; ++x)
#pragma unroll
                        for (int y = 0; y < kRows; ++y) wv[x][u] += v[y] * cr[y][x];
                }
            }
        }
#pragma unroll
        for (int x = 0; x < kCols; ++x)
#pragma unroll
            for (int u = 0; u < kPanel; ++u)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) wv[x][u] += __shfl_xor_sync(0xffffffffu, wv[x][u], o);
        // w2 = T^T w (kept in wv, highest u first so that lower entries are still w)
#pragma unroll
        for (int x = 0; x < kCols; ++x) {
#pragma unroll
            for (int u = kPanel - 1; u >= 0; --u) {
                T acc = 0;
#pragma unroll
                for (int s2 = 0; s2 <= u; ++s2)
                    if (u < nb) acc += tm[s2 * kPanel + u] * wv[x][s2];
                wv[x][u] = acc;
            }
        }
        for (int r = lane; r < qq; r += 32 * kRows) {
            T acc[kRows][kCols];
            if (all_cols && r + 32 * (kRows - 1) < qq) {
#pragma unroll
                for (int y = 0; y < kRows; ++y)
#pragma unroll
                    for (int x = 0; x < kCols; ++x) acc[y][x] = tf[x][r + 32 * y];
#pragma unroll
                for (int u = 0; u < kPanel; ++u) {
                    const T *vu = V + (int64_t)u * qq + r;
#pragma unroll
                    for (int y = 0; y < kRows; ++y) {
                        const T v = vu[32 * y];
#pragma unroll
                        for (int x = 0; x < kCols; ++x) acc[y][x] -= v * wv[x][u];
                    }
                }
#pragma unroll
                for (int y = 0; y < kRows; ++y)
#pragma unroll
                    for (int x = 0; x < kCols; ++x)
                        if (has[x]) tc[x][r + 32 * y] = acc[y][x];
                continue;
            }
#pragma unroll
            for (int y = 0; y < kRows; ++y)
#pragma unroll
                for (int x = 0; x < kCols; ++x) acc[y][x] = (tc[x] && r + 32 * y < qq) ? tc[x][r + 32 * y] : T(0);
#pragma unroll
            for (int u = 0; u < kPanel; ++u) {
                if (u < nb) {
#pragma unroll
                    for (int y = 0; y < kRows; ++y) {
                        const T v = (r + 32 * y < qq) ? V[(int64_t)u * qq + r + 32 * y] : T(0);
#pragma unroll
                        for (int x = 0; x < kCols; ++x) acc[y][x] -= v * wv[x][u];
                    }
                }
            }
#pragma unroll
            for (int y = 0; y < kRows; ++y)
#pragma unroll
                for (int x = 0; x < kCols; ++x)
                    if (tc[x] && r + 32 * y < qq) tc[x][r + 32 * y] = acc[y][x];
        }
    }
    team.sync();
}

// Head of the panel staging area (global-memory bins), in elements of T: the
// panel's T (kPanel x kPanel), the CTA reduction slots (kPanel per warp) and
// two kPanel-vectors of results; the staged panel V follows.
template <class Team> constexpr int kStageHead = kPanel * kPanel + (Team::SIZE / 32 + 2) * kPanel;

// Sum of kPanel values over the 32 lanes of a warp by halving exchanges (a
// lane keeps the half of its vector that its partner sends back summed): 16
// shuffles instead of 16 x 5.  Lanes 2e and 2e+1 end up holding the sum of
// entry rs_entry(lane) in v[0].
__device__ __forceinline__ int rs_entry(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}
template <typename T> __device__ __forceinline__ T warp_reduce_scatter16(T (&v)[kPanel], int lane) {
    static_assert(kPanel == 16, "the exchange pattern below is written for 16 values");
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// out[0..kPanel) = the sums of v[0..kPanel) over the CTA, visible to every
// thread on return (two synchronisations).  The warps' partial sums go through
// red, kPanel per warp; warp 0 adds them, lane l taking entry l % kPanel over
// every other warp and one shuffle joining the two halves.
template <class Team, typename T>
__device__ __forceinline__ void team_sum16(const Team &team, T (&v)[kPanel], T *red, T *out) {
    constexpr int NW = Team::SIZE / 32;
    const int me = team.rank(), lane = me & 31;
    const T sv = warp_reduce_scatter16(v, lane);
    if ((lane & 1) == 0) red[(me >> 5) * kPanel + rs_entry(lane)] = sv;
    team.sync();
    if (me < 32) {
        const int e = lane & (kPanel - 1);
        T a = T(0);
#pragma unroll
        for (int w = lane >> 4; w < NW; w += 2) a += red[w * kPanel + e];
        a += __shfl_xor_sync(0xffffffffu, a, 16);
        if (lane < kPanel) out[lane] = a;
    }
    team.sync();
}

// Asynchronous element copies global -> shared (cp.async, 4 or 8 bytes: no
// alignment beyond the element's own); cp_async_wait waits for the calling
// thread's copies.
template <typename T> __device__ __forceinline__ void cp_async_elem(T *smem_dst, const T *gmem_src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// rhs[0..p) <- R^{-1} rhs[0..p) for a CTA team, in blocks of kBS rows from
// the bottom: one warp solves the block's triangle (lane l holds row b0 + l
// and loads its row of the block into registers first), then every thread
// subtracts the block's part from the rows above.  Each row receives its
// terms in the same order (descending column) as the one-row-at-a-time
// version, so the results are identical.
template <class Team, typename T>
__device__ void back_substitute_blocked(const Team &team, const T *B, int q, int p, T *rhs, T small) {
    constexpr int kBS = sizeof(T) == 8 ? 16 : 32;
    const int me = team.rank();
    for (int b1 = p; b1 > 0;) {
        const int b0 = max(0, b1 - kBS);
        const int nbk = b1 - b0;
        if (me < 32) {
            const int i = b0 + me;
            const bool row = me < nbk;
            T rv[kBS];
#pragma unroll
            for (int u = 0; u < kBS; ++u) rv[u] = (row && u < nbk) ? B[(int64_t)(b0 + u) * q + i] : T(0);
            const T dd = row ? B[(int64_t)i * q + i] : T(1);
            T xi = row ? rhs[i] : T(0);
#pragma unroll
            for (int u = kBS - 1; u >= 0; --u) {
                if (u < nbk) {
                    const T rr = __shfl_sync(0xffffffffu, xi, u);
                    const T d = __shfl_sync(0xffffffffu, dd, u);
                    const T xr = (fabs(d) <= small) ? T(0) : rr / d;
                    if (me == u) xi = xr;
                    else if (me < u) xi -= rv[u] * xr;
                }
            }
            if (row) rhs[i] = xi;
        }
        team.sync();
        for (int c = me; c < b0; c += Team::SIZE) {
            T bv[kBS];
#pragma unroll
            for (int u = 0; u < kBS; ++u) bv[u] = (u < nbk) ? B[(int64_t)(b0 + u) * q + c] : T(0);
            T a = rhs[c];
#pragma unroll
            for (int u = kBS - 1; u >= 0; --u)
                if (u < nbk) a -= bv[u] * rhs[b0 + u];
            rhs[c] = a;
        }
        team.sync();
        b1 = b0;
    }
}

// Householder QR of the staged panel V (rows 0..qq-1, nb <= kPanel columns,
// ld qq, shared memory) with the T of its compact-WY form.  Step t makes one
// pass over rows r >= t for x.x (x = column t), c.x for the trailing panel
// columns c and v_s.x for the earlier reflectors s, and one CTA reduction of
// the kPanel sums.  Since v_t differs from x only in its head (v0 instead of
// x0), v_t.c = c.x + (v0 - x0) c_t and Y(s,t) = v_s.v_t = v_s.x + (v0 - x0) v_s(t).
// Y(s,t) is kept below the diagonal of tm (tm[t * kPanel + s]) and tau_t on it;
// after the last step one warp forms T(t,t) = tau_t and
// T(s,t) = -tau_t sum_{s <= s2 < t} T(s,s2) Y(s2,t) above it (tm[s * kPanel + t]).
// Leaves R on and above the diagonal, the reflector tails below it, and
// vhead[t] = v0, taus[t] = 2 / v^T v.
template <class Team, typename T>
__device__ __forceinline__ void panel_factor_fused(const Team &team, T *V, int qq, int nb, T *vhead, T *taus, T *tm,
                                                   T *red, T *out, T *out2, T small, int &rank_flag) {
    const int me = team.rank();
    for (int t = 0; t < nb; ++t) {
        T *x = V + (int64_t)t * qq;
        T acc[kPanel];
#pragma unroll
        for (int u = 0; u < kPanel; ++u) acc[u] = T(0);
        // two rows per thread and iteration: their loads are issued together
        int r = t + me;
        for (; r + Team::SIZE < qq; r += 2 * Team::SIZE) {
            const T xa = x[r], xb = x[r + Team::SIZE];
#pragma unroll
            for (int u = 0; u < kPanel; ++u) {
                if (u < nb) {
                    const T *vu = V + (int64_t)u * qq + r;
                    acc[u] += vu[0] * xa + vu[Team::SIZE] * xb;
                }
            }
        }
        if (r < qq) {
            const T xr = x[r];
#pragma unroll
            for (int u = 0; u < kPanel; ++u)
                if (u < nb) acc[u] += V[(int64_t)u * qq + r] * xr;
        }
        team_sum16(team, acc, red, out);
        const T sigma = out[t];
        const T x0 = x[t];
        const T nrm = sqrt(sigma);
        const T alpha = (x0 >= T(0)) ? -nrm : nrm;
        const T v0 = x0 - alpha;
        const T vtv = sigma - x0 * x0 + v0 * v0;
        const T two_over = (vtv > T(0)) ? T(2) / vtv : T(0);
        if (me < nb) {
            if (me == t) {
                tm[t * kPanel + t] = two_over;
            } else {
                const T d = out[me] + (v0 - x0) * V[(int64_t)me * qq + t];
                if (me > t) out2[me] = d * two_over;  // f_c for the trailing column c = me
                else tm[t * kPanel + me] = d;          // Y(s,t) for the earlier reflector s = me
            }
        }
        team.sync();
        if (two_over > T(0)) {
            int r2 = t + me;
            for (; r2 + Team::SIZE < qq; r2 += 2 * Team::SIZE) {
                const T va = (r2 == t) ? v0 : x[r2], vb = x[r2 + Team::SIZE];
#pragma unroll
                for (int u = 0; u < kPanel; ++u) {
                    if (u > t && u < nb) {
                        T *cu = V + (int64_t)u * qq + r2;
                        const T f = out2[u];
                        const T ca = cu[0], cb = cu[Team::SIZE];
                        cu[0] = ca - f * va;
                        cu[Team::SIZE] = cb - f * vb;
                    }
                }
            }
            if (r2 < qq) {
                const T vr = (r2 == t) ? v0 : x[r2];
#pragma unroll
                for (int u = 0; u < kPanel; ++u)
                    if (u > t && u < nb) V[(int64_t)u * qq + r2] -= out2[u] * vr;
            }
        }
        team.sync();
        if (me == 0) {
            x[t] = alpha;
            vhead[t] = v0;
            taus[t] = two_over;
        }
        rank_flag |= (fabs(alpha) <= small) ? 1 : 0;
    }
    // T from Y and tau: lane s of warp 0 holds row s of T
    if (me < 32) {
        const int sr = me;
        T trow[kPanel];
#pragma unroll
        for (int t = 0; t < kPanel; ++t) {
            trow[t] = T(0);
            if (t < nb) {
                const T tau = tm[t * kPanel + t];
                T a = T(0);
#pragma unroll
                for (int s2 = 0; s2 < t; ++s2)
                    if (s2 >= sr) a += trow[s2] * tm[t * kPanel + s2];
                if (sr < t) trow[t] = -tau * a;
                else if (sr == t) trow[t] = tau;
            }
        }
        if (sr < nb) {
#pragma unroll
            for (int t = 0; t < kPanel; ++t)
                if (t > sr && t < nb) tm[sr * kPanel + t] = trow[t];
        }
    }
    team.sync();
}

// rhs <- Q^T rhs with the reflectors in the panels they were factored in
// (pnb, Tst): per panel w = V^T rhs (one CTA reduction), y = T^T w, and
// rhs <- rhs - V y, with V = the explicit reflectors (vhead on the diagonal,
// the tails of B below it).  A panel is taken in sub-panels of as many
// reflectors as the staging area holds (the diagonal blocks of its T); each is
// copied there first (cp.async) and both passes read shared memory.  When
// fewer than two reflectors fit, or one is left, the rest of the panel reads
// its tails from the slab.
template <class Team, typename T>
__device__ __noinline__ void apply_qt_panels(Team team, const T *B, int q, int p, T *rhs, const T *vhead,
                                             const T *Tst, const int32_t *pnb, T *stage, int stage_bytes) {
    constexpr int NW = Team::SIZE / 32;
    const int me = team.rank();
    T *red = stage + kPanel * kPanel, *out = red + NW * kPanel, *out2 = out + kPanel;
    T *V = stage + kStageHead<Team>;
    const int64_t velems = (int64_t)stage_bytes / (int64_t)sizeof(T) - kStageHead<Team>;
    for (int jp = 0; jp < p;) {
        const int nbp = pnb[jp];
        // sub-panels of as many reflectors as the staging area holds (the
        // diagonal blocks of a panel's T are the T's of its sub-panels); a
        // sub-panel that cannot be staged reads its reflectors from the slab
        for (int js = 0; js < nbp;) {
            const int j0 = jp + js;
            const int qq = q - j0;
            const int64_t fit = velems / (int64_t)max(qq, 1);
            const bool staged = nbp - js > 1 && fit >= 2;
            const int nb = staged ? (int)min((int64_t)(nbp - js), fit) : nbp - js;
            if (staged) {
                for (int t = 0; t < nb; ++t) {
                    const T *src = B + (int64_t)(j0 + t) * q + j0;
                    T *dst = V + (int64_t)t * qq;
                    for (int r = me; r < qq; r += Team::SIZE) {
                        if (r > t) cp_async_elem(dst + r, src + r);
                        else dst[r] = (r == t) ? vhead[j0 + t] : T(0);
                    }
                }
                cp_async_wait();
                team.sync();
            }
            T acc[kPanel];
#pragma unroll
            for (int u = 0; u < kPanel; ++u) acc[u] = T(0);
            if (staged) {
                for (int r = me; r < qq; r += Team::SIZE) {
                    const T x = rhs[j0 + r];
#pragma unroll
                    for (int u = 0; u < kPanel; ++u)
                        if (u < nb) acc[u] += V[(int64_t)u * qq + r] * x;
                }
            } else {
                for (int i = j0 + me; i < q; i += Team::SIZE) {
                    const T x = rhs[i];
#pragma unroll
                    for (int u = 0; u < kPanel; ++u) {
                        if (u < nb) {
                            const int j = j0 + u;
                            const T v = (i > j) ? B[(int64_t)j * q + i] : ((i == j) ? vhead[j] : T(0));
                            acc[u] += v * x;
                        }
                    }
                }
            }
            team_sum16(team, acc, red, out);
            if (me < nb) {
                T y = 0;
                for (int s2 = 0; s2 <= me; ++s2) y += Tst[(int64_t)(j0 + me) * kPanel + js + s2] * out[s2];
                out2[me] = y;
            }
            team.sync();
            if (staged) {
                for (int r = me; r < qq; r += Team::SIZE) {
                    T a = rhs[j0 + r];
#pragma unroll
                    for (int u = 0; u < kPanel; ++u)
                        if (u < nb) a -= V[(int64_t)u * qq + r] * out2[u];
                    rhs[j0 + r] = a;
                }
            } else {
                for (int i = j0 + me; i < q; i += Team::SIZE) {
                    T a = rhs[i];
#pragma unroll
                    for (int u = 0; u < kPanel; ++u) {
                        if (u < nb) {
                            const int j = j0 + u;
                            const T v = (i > j) ? B[(int64_t)j * q + i] : ((i == j) ? vhead[j] : T(0));
                            a -= v * out2[u];
                        }
                    }
                    rhs[i] = a;
                }
            }
            team.sync();
            js += nb;
        }
        jp += nbp;
    }
}

// Blocked Householder QR (compact WY) for the bins whose workspace is in
// global memory.  Panels of nb <= kPanel columns (nb chosen so that rows j0..q
// of the panel fit the shared-memory staging area) are copied to shared
// memory (cp.async), factored there with their T (panel_factor_fused), written
// back, and turned into explicit reflectors V (zeros above the head, v(j) on
// the diagonal); with T upper triangular, H_1...H_nb = I - V T V^T, every
// trailing column and the right-hand side get
//   C <- C - V (T^T (V^T C))
// in one pass (one warp per four columns), so the trailing matrix in global memory
// is streamed once per panel instead of once per reflector.  Each panel's size
// and T are kept (pnb, Tst) for the QR update and the refinement.  A panel that
// does not fit four columns falls back to single Householder steps (panels of
// one).  The reflectors, R and rhs are those of the unblocked version up to
// rounding.  j_start > 0 factors only columns j_start..p-1 (the columns
// appended to a factor whose first j_start columns are done, Section 3);
// backsub = false leaves Q^T rhs in rhs.
template <class Team, typename T>
__device__ __noinline__ int qr_solve_staged(Team team, T *B, int q, int p, T *rhs, T *vhead, T *taus, T small,
                                            T *stage, int stage_bytes, T *Tst, int32_t *pnb,
                                            int j_start = 0, bool backsub = true) {
    const int me = team.rank();
    constexpr int NW = Team::SIZE / 32;
    T *tm = stage;                                  // kPanel x kPanel
    T *red = stage + kPanel * kPanel;               // reduction slots
    T *out = red + NW * kPanel, *out2 = out + kPanel;
    T *V = stage + kStageHead<Team>;                // panel, ld = q - j0
    const int64_t velems = (int64_t)stage_bytes / (int64_t)sizeof(T) - kStageHead<Team>;
    int rank_flag = 0;
    int j0 = j_start;
    while (j0 < p) {
        const int qq = q - j0;
        int nb = (int)min((int64_t)kPanel, velems / (int64_t)max(qq, 1));
        nb = min(nb, p - j0);
        if (nb < 4) {
            householder_step(team, B, q, p, rhs, vhead, taus, j0, j0 + 1, small, rank_flag);
            if (me == 0) {
                pnb[j0] = 1;
                Tst[(int64_t)j0 * kPanel] = taus[j0];
            }
            ++j0;
            continue;
        }
        // 1. stage rows j0..q-1 of the panel columns (asynchronous copies)
        for (int t = 0; t < nb; ++t) {
            const T *src = B + (int64_t)(j0 + t) * q + j0;
            for (int r = me; r < qq; r += Team::SIZE) cp_async_elem(V + (int64_t)t * qq + r, src + r);
        }
        cp_async_wait();
        team.sync();
        // 2. factor the panel in shared memory (local rows r = i - j0), T alongside
        panel_factor_fused(team, V, qq, nb, vhead + j0, taus + j0, tm, red, out, out2, small, rank_flag);
        // 3. panel back to B (R entries and reflector tails), 4. explicit V, T kept
        for (int idx = me; idx < nb * qq; idx += Team::SIZE) {
            const int t = idx / qq, r = idx - t * qq;
            B[(int64_t)(j0 + t) * q + j0 + r] = V[idx];
        }
        team.sync();
        for (int idx = me; idx < nb * qq; idx += Team::SIZE) {
            const int t = idx / qq, r = idx - t * qq;
            if (r < t) V[idx] = T(0);
            else if (r == t) V[idx] = vhead[j0 + t];
        }
        for (int e = me; e < nb * kPanel; e += Team::SIZE) {
            const int t = e / kPanel, s2 = e - t * kPanel;
            Tst[(int64_t)(j0 + t) * kPanel + s2] = (s2 <= t) ? tm[s2 * kPanel + t] : T(0);
        }
        if (me == 0) pnb[j0] = nb;
        team.sync();
        // 5. trailing columns and rhs, rows j0..q-1
        wy_apply(team, V, qq, nb, tm, B, q, p, rhs, j0, j0 + nb, p);
        j0 += nb;
    }
    if (backsub) back_substitute_blocked(team, B, q, p, rhs, small);
    return rank_flag;
}

// rhs <- Q^T rhs with the stored reflectors, then R^{-1}; not inlined
template <class Team, typename T>
__device__ __noinline__ void apply_qt_team(Team team, const T *B, int q, int p, T *rhs, const T *vhead,
                                           const T *taus, T small) {
    const int me = team.rank();
    for (int j = 0; j < p; ++j) {
        const T *col = B + (int64_t)j * q;
        const T v0 = vhead[j], tau = taus[j];
        if (tau > T(0)) {
            T d = 0;
            for (int i = me; i < q; i += Team::SIZE)
                if (i >= j) d += ((i == j) ? v0 : col[i]) * rhs[i];
            T sdot = team.sum(d);
            T f = sdot * tau;
            for (int i = me; i < q; i += Team::SIZE)
                if (i >= j) rhs[i] -= f * ((i == j) ? v0 : col[i]);
        }
        team.sync();
    }
    if constexpr (is_lane_team<Team>::value) back_substitute_team(team, B, q, p, rhs, small);
    else back_substitute_blocked(team, B, q, p, rhs, small);
}

// The QR update of Section 3, first half: the reflectors 0..p0-1 of a
// finished factor (built on q0 rows; every row below is zero in them) applied
// to the appended columns p0..p-1 of B (ld q), rows j..q0-1.  In the
// global-memory bins (pnb != nullptr) the reflectors go panel by panel as
// they were factored, each panel in compact-WY form with its stored T, split
// into sub-panels when its explicit V outgrows the staging area (q has grown
// since it was factored).  Sub-panels of fewer than four reflectors, and the
// shared-memory bins, take one reflector per pass, one warp per column.
template <class Team, typename T>
__device__ __noinline__ void qr_update_apply(Team team, T *B, int q, int p, int q0, int p0, const T *vhead,
                                             const T *taus, T *stage, int stage_bytes, const T *Tst,
                                             const int32_t *pnb) {
    const int me = team.rank();
    const int lane = me & 31, wid = me >> 5;
    constexpr int NW = (Team::SIZE + 31) / 32;
    T *tm = stage;
    T *V = stage + kStageHead<Team>;
    const int64_t velems = stage_bytes > 0 ? (int64_t)stage_bytes / (int64_t)sizeof(T) - kStageHead<Team> : 0;
    int j0 = 0;
    while (j0 < p0) {
        const int nb = pnb ? pnb[j0] : 1;
        // the panel in sub-panels of as many reflectors as the staging area holds:
        // the diagonal blocks of a panel's T are the T's of its sub-panels
        for (int js = 0; js < nb;) {
            const int j1 = j0 + js, qq = q0 - j1;
            const int ns = (int)min((int64_t)(nb - js), qq > 0 ? velems / (int64_t)qq : (int64_t)0);
            if (ns < 4) {  // one reflector, one warp per column
                const T *col = B + (int64_t)j1 * q;
                const T v0 = vhead[j1], two_over = taus[j1];
                if (two_over > T(0)) {
                    for (int c = p0 + wid; c < p; c += NW) {
                        T *t = B + (int64_t)c * q;
                        T d = 0;
                        for (int i = j1 + lane; i < q0; i += 32) d += ((i == j1) ? v0 : col[i]) * t[i];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                        const T f = d * two_over;
                        for (int i = j1 + lane; i < q0; i += 32) t[i] -= f * ((i == j1) ? v0 : col[i]);
                    }
                }
                team.sync();
                ++js;
                continue;
            }
            for (int t = 0; t < ns; ++t) {
                const T *src = B + (int64_t)(j1 + t) * q + j1;
                T *dst = V + (int64_t)t * qq;
                for (int r = me; r < qq; r += Team::SIZE) {
                    if (r > t) cp_async_elem(dst + r, src + r);
                    else dst[r] = (r == t) ? vhead[j1 + t] : T(0);
                }
            }
            cp_async_wait();
            for (int e = me; e < kPanel * kPanel; e += Team::SIZE) {
                const int s2 = e / kPanel, t = e - s2 * kPanel;
                tm[e] = (t < ns && s2 <= t) ? Tst[(int64_t)(j1 + t) * kPanel + js + s2] : T(0);
            }
            team.sync();
            wy_apply(team, V, qq, ns, tm, B, q, p, (T *)nullptr, j1, p0, p - 1);
            js += ns;
        }
        j0 += nb;
    }
}

// J = rows of A(:,k), ascending as the CSC keeps them; returns |J|, or -1 if
// it exceeds pcap, and in *bytes the algorithmic bytes of J's columns (12 per
// nonzero + 16 each).  Kept out of line: only the initial pattern of A uses it.
template <class Team>
__device__ __noinline__ int pattern_of_column(Team team, const int64_t *col_ptr, const int32_t *row_idx, int32_t k,
                                              int pcap, int32_t *J, long long *bytes) {
    const int me = team.rank();
    const int64_t e0 = col_ptr[k];
    const int len = (int)(col_ptr[k + 1] - e0);
    if (len > pcap) return -1;
    long long b = 0;
    for (int c = me; c < len; c += Team::SIZE) {
        const int32_t j = row_idx[e0 + c];
        J[c] = j;
        b += 12 * (col_ptr[j + 1] - col_ptr[j]) + 16;
    }
    *bytes = team.sum(b);
    team.sync();
    return len;
}

// J -> position in J: an open-addressing hash of J (hcap slots, warp bins)
// or a binary search of the sorted J (hcap = 0).
struct JSet {
    const int32_t *J, *hkey, *hval;
    int p, hcap;
    __device__ __forceinline__ unsigned slot(int32_t col) const {
        return ((unsigned)col * 0x9E3779B1u) >> (32 - __ffs(hcap) + 1);
    }
    __device__ __forceinline__ int find(int32_t col) const {
        if (hcap == 0) return find_i32(J, p, col);
        const unsigned mask = (unsigned)hcap - 1;
        unsigned sl = slot(col);
        for (;;) {
            const int32_t key = hkey[sl];
            if (key == col) return hval[sl];
            if (key == -1) return -1;
            sl = (sl + 1) & mask;
        }
    }
};

struct SpaiPick {
    int na;               // columns chosen (in buf, ascending); 0: no candidate; -1: overflow
    long long bytes, sel; // algorithmic bytes and selection flops
};

// SPAI's most profitable indices (Section 2, Eqs. 2.5-2.7).  L = rows of S
// with |r_i| > band (the same reading of r_i != 0 as the dominant rows);
// the candidates Jhat = cols(A(L,:)) \ J, each scored by one rank walking
// its CSC column: s_j = (r^T A e_j)^2 / ||A e_j||^2 in double (rho_j^2 =
// ||r||^2 - s_j, so the largest s_j are the smallest rho_j); the c best by
// (s_j desc, j asc) with a tie band of tie_band * ||r||^2, the scores
// compared as ordered integer keys (non-negative doubles).  The chosen
// columns go to buf in ascending order.  Returns their number, 0 when no
// candidate is left, -1 on overflow.
template <class Team>
__device__ __noinline__ SpaiPick spai_select(Team team, DevA A, int c, double tie_band, int scap, const int32_t *S,
                                             const double *r, int s, JSet Jset, int32_t *buf, int32_t *buf2,
                                             double *sc, int32_t *Rhat) {
    const int me = team.rank();
    SpaiPick out{0, 0, 0};
    long long rinf = 0;
    double rr = 0.0;
    for (int i = me; i < s; i += Team::SIZE) {
        rinf = max(rinf, abskey(r[i]));
        rr = fma(r[i], r[i], rr);
    }
    rinf = team.maxv(rinf);
    rr = team.sum(rr);
    const long long bk = abskey(tie_band * key_value(rinf));
    // column indices of the rows of L
    int tot = 0;
    long long byt = 0;
    for (int i0 = 0; i0 < s; i0 += Team::SIZE) {
        const int i = i0 + me;
        int len = 0;
        int64_t st = 0;
        if (i < s && abskey(r[i]) > bk) {
            const int32_t row = S[i];
            st = A.row_ptr[row];
            len = (int)(A.row_ptr[row + 1] - st);
            byt += 4LL * len + 16;
        }
        int part;
        const int off = tot + team.scan(len, &part);
        if (next_pow2(tot + part) > scap) {
            out.na = -1;
            return out;
        }
        for (int e = 0; e < len; ++e) buf[off + e] = A.col_idx[st + e];
        tot += part;
    }
    out.bytes += team.sum(byt);
    team.sync();
    if (tot == 0) return out;
    team_sort_i32(team, buf, tot);
    const int nu = team_unique_i32(team, buf, tot, buf2);
    int nc = 0;
    for (int i0 = 0; i0 < nu; i0 += Team::SIZE) {
        const int i = i0 + me;
        const int f = (i < nu) && (Jset.find(buf2[i]) < 0);
        int part;
        const int pos = team.scan(f, &part);
        if (f) buf[nc + pos] = buf2[i];
        nc += part;
    }
    team.sync();
    if (nc == 0) return out;
    // scores (Eq. 2.7)
    long long sf = 0;
    byt = 0;
    for (int t = me; t < nc; t += Team::SIZE) {
        const int32_t j = buf[t];
        double dot = 0.0, nrm = 0.0;
        const int64_t e0 = A.col_ptr[j], e1 = A.col_ptr[j + 1];
        for (int64_t e = e0; e < e1; ++e) {
            const double a = A.cval[e];
            const int pos = find_i32(S, s, A.row_idx[e]);
            if (pos >= 0) dot = fma(r[pos], a, dot);
            nrm = fma(a, a, nrm);
        }
        sc[t] = (nrm > 0.0) ? dot * dot / nrm : 0.0;
        sf += 4 * (e1 - e0) + 3;
        byt += 12 * (e1 - e0) + 16;
    }
    out.sel += team.sum(sf);
    out.bytes += team.sum(byt);
    team.sync();
    const bool take_all = nc <= c;
    long long hik = 0, lob = 0;
    if (!take_all) {
        // the c-th score of the (s_j desc, j asc) order: c rounds of argmax
        long long pa = LLONG_MAX;
        int pi = -1;
        for (int t = 0; t < c; ++t) {
            long long ba = -1;
            int bi = INT32_MAX;
            for (int u = me; u < nc; u += Team::SIZE) {
                const long long a = abskey(sc[u]);
                const int32_t j = buf[u];
                if (dom_before(pa, pi, a, j) && dom_before(a, j, ba, bi)) {
                    ba = a;
                    bi = j;
                }
            }
            team.argmax(ba, bi);
            pa = ba;
            pi = bi;
        }
        const double v = key_value(pa), sband = tie_band * rr;
        hik = abskey(v + sband);
        lob = __double_as_longlong(v - sband);  // negative bit pattern if v - sband < 0
    }
    int nabove = 0;
    if (!take_all) {
        for (int u = me; u < nc; u += Team::SIZE) nabove += abskey(sc[u]) > hik;
        nabove = team.sum(nabove);
    }
    const int need = c - nabove;
    int na = 0, tb = 0;
    for (int u0 = 0; u0 < nc; u0 += Team::SIZE) {
        const int u = u0 + me;
        int above = 0, tie = 0;
        if (u < nc && !take_all) {
            const long long a = abskey(sc[u]);
            above = a > hik;
            tie = (a >= lob) && (a <= hik);
        }
        int tpart;
        const int trank = team.scan(tie, &tpart);
        const int sel = (u < nc) && (take_all || above || (tie && tb + trank < need));
        int part;
        const int pos = team.scan(sel, &part);
        if (sel) Rhat[na + pos] = buf[u];
        na += part;
        tb += tpart;
    }
    team.sync();
    for (int t = me; t < na; t += Team::SIZE) buf[t] = Rhat[t];
    team.sync();
    out.na = na;
    return out;
}


template <class Team, typename T> struct Column {
    const Team &team;
    const DevA &A;
    const DevParams &P;
    const Caps &cap;
    Work<T> &w;
    int32_t k;
    int p, q, s, nR, l, nD;
    int64_t q0, p0;
    int rank_flag;
    double rho;
    T small_last;  // rank threshold of the last solve (reused by the adjoint)
    T fro2_f;      // ||B||_F^2 of the kept factor (Caps::append)
    bool fact_valid;  // B, vhead, tau, qte, Ip, Jp hold the factor of the current J (Caps::append)
    // per-column work counters (integers; committed only when the column finishes)
    long long c_qr, c_res, c_ref, c_ref64, c_bytes, c_sel;
    int c_solves, c_drops, c_pmax, c_qmax;

    __device__ Column(const Team &t, const DevA &a, const DevParams &pp, const Caps &c, Work<T> &ww, int32_t kk)
        : team(t), A(a), P(pp), cap(c), w(ww), k(kk) {}

    // J -> position in J: open-addressing hash (warp bins) or binary search.
    // The table's layout may depend on insertion order; lookups do not.
    __device__ __forceinline__ JSet jset() const { return JSet{w.J, w.hkey, w.hval, p, cap.hcap}; }
    __device__ void build_jhash() {
        if (cap.hcap == 0) return;
        for (int i = team.rank(); i < cap.hcap; i += Team::SIZE) w.hkey[i] = -1;
        team.sync();
        const unsigned mask = (unsigned)cap.hcap - 1;
        const JSet js = jset();
        for (int c = team.rank(); c < p; c += Team::SIZE) {
            const int32_t key = w.J[c];
            unsigned sl = js.slot(key);
            for (;;) {
                int32_t old = atomicCAS(&w.hkey[sl], -1, key);
                if (old == -1) { w.hval[sl] = c; break; }
                sl = (sl + 1) & mask;
            }
        }
        team.sync();
    }
    __device__ __forceinline__ int find_J(int32_t col) const { return jset().find(col); }

    // I = sorted rows of A(:,J) (Section 2).  Returns false on overflow.
    __device__ bool rows_of_J() {
        int base = 0;
        for (int c0 = 0; c0 < p; c0 += Team::SIZE) {
            int c = c0 + team.rank();
            int len = 0;
            int64_t st = 0;
            if (c < p) {
                st = A.col_ptr[w.J[c]];
                len = (int)(A.col_ptr[w.J[c] + 1] - st);
            }
            int tot;
            int off = team.scan(len, &tot);
            if (next_pow2(base + tot) > cap.scap) return false;
            for (int e = 0; e < len; e += 4) {
                int32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = (e + u < len) ? A.row_idx[st + e + u] : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (e + u < len) w.buf[base + off + e + u] = v[u];
            }
            base += tot;
        }
        team.sync();
        team_sort_i32(team, w.buf, base);
        int nq = team_unique_i32(team, w.buf, base, w.buf2);
        if (nq > cap.qcap) return false;
        for (int i = team.rank(); i < nq; i += Team::SIZE) w.I[i] = w.buf2[i];
        q = nq;
        team.sync();
        return true;
    }

    // Householder QR of B (q x p, ld q) applied to rhs, then back substitution
    // into rhs[0..p); the reflectors stay in B (tails), vhead and tau.
    __device__ void qr_solve(T small) {
        if constexpr (is_lane_team<Team>::value) {
            if (p > 2 && p <= cap.small_p && q <= Team::SIZE * kRegRows<Team>) {
                rank_flag = lanes_qr_small<Team::SIZE, kRegRows<Team>>(w.B, q, p, w.rhs, w.vhead, w.tau, small);
                return;
            }
        }
        if constexpr (!is_lane_team<Team>::value) {
            const bool keep = cap.append != 0;  // keep Q^T e_k for later updates
            if (cap.stage_bytes > 0 && p >= 2 * kPanel)
                rank_flag = qr_solve_staged<Team, T>(team, w.B, q, p, w.rhs, w.vhead, w.tau, small, (T *)w.stage,
                                                     cap.stage_bytes, w.Tst, w.pnb, 0, !keep);
            else if (keep) {
                rank_flag = qr_factor_team<Team, T>(team, w.B, q, p, w.rhs, w.vhead, w.tau, small, 0);
                single_panels(0);
            } else {
                rank_flag = qr_solve_team<Team, T>(team, w.B, q, p, w.rhs, w.vhead, w.tau, small);
            }
            if (keep) {
                // a factor from scratch: factor order = sorted order
                const int me = team.rank();
                for (int i = me; i < q; i += Team::SIZE) {
                    w.qte[i] = w.rhs[i];
                    w.Ip[i] = i;
                }
                for (int c = me; c < p; c += Team::SIZE) w.Jp[c] = c;
                team.sync();
                back_substitute_blocked(team, w.B, q, p, w.rhs, small);
                fact_valid = true;
            }
            return;
        }
        rank_flag = qr_solve_team<Team, T>(team, w.B, q, p, w.rhs, w.vhead, w.tau, small);
    }

    // Reflectors j0..p-1 factored one at a time: panels of one (global-memory bins)
    __device__ void single_panels(int j0) {
        if (w.pnb == nullptr) return;
        for (int j = j0 + team.rank(); j < p; j += Team::SIZE) {
            w.pnb[j] = 1;
            w.Tst[(int64_t)j * kPanel] = w.tau[j];
        }
        team.sync();
    }

    // factor row of sorted I position i / factor column of sorted J position c
    __device__ __forceinline__ int frow(int i) const {
        if constexpr (is_lane_team<Team>::value) return i;
        else return cap.append ? w.Ip[i] : i;
    }
    __device__ __forceinline__ int fcol(int c) const {
        if constexpr (is_lane_team<Team>::value) return c;
        else return cap.append ? w.Jp[c] : c;
    }

    // rhs <- R^{-1} Q^T rhs with the stored reflectors
    __device__ void apply_qt_solve(T small) {
        if constexpr (is_lane_team<Team>::value) {
            if (p > 2 && p <= cap.small_p && q <= Team::SIZE * kRegRows<Team>) {
                lanes_apply_qt_small<Team::SIZE, kRegRows<Team>>(w.B, q, p, w.rhs, w.vhead, w.tau, small);
                return;
            }
        }
        if constexpr (!is_lane_team<Team>::value) {
            if (w.pnb != nullptr) {
                apply_qt_panels<Team, T>(team, w.B, q, p, w.rhs, w.vhead, w.Tst, w.pnb, (T *)w.stage,
                                         cap.stage_bytes);
                back_substitute_blocked(team, w.B, q, p, w.rhs, small);
                return;
            }
        }
        apply_qt_team<Team, T>(team, w.B, q, p, w.rhs, w.vhead, w.tau, small);
    }

    // S = I u {k}; r = A(:,J) m - e_k on S in double (Eq. 2.4), row by row
    // through the CSR of A: in ascending j on the warp bins (the oracle's
    // order), a fixed lane-strided order and butterfly on the CTA bins.
    // `refine`: the residual of a refinement step (counted as refinement work).
    __device__ void residual(bool refine = false) {
        const int me = team.rank();
        int pk = lower_bound_i32(w.I, q, k);
        bool has_k = pk < q && w.I[pk] == k;
        s = has_k ? q : q + 1;
        for (int i = me; i < s; i += Team::SIZE) {
            int32_t row;
            if (has_k) row = w.I[i];
            else row = (i < pk) ? w.I[i] : (i == pk ? k : w.I[i - 1]);
            w.S[i] = row;
        }
        double ss = 0.0;
        int cnt = 0;
        if constexpr (!is_lane_team<Team>::value) {
            // CTA teams: a warp per row, its lanes over the row's entries (rows of
            // I can hold hundreds), summed by a fixed butterfly.  The global-memory
            // bins search a copy of J in the staging area (shared memory).
            const int32_t *Js = w.J;
            if (cap.stage_bytes > 0 && (size_t)p * sizeof(int32_t) <= (size_t)cap.stage_bytes) {
                int32_t *jc = reinterpret_cast<int32_t *>(w.stage);
                for (int c = me; c < p; c += Team::SIZE) jc[c] = w.J[c];
                Js = jc;
            }
            team.sync();
            const int lane = me & 31;
            constexpr int NWR = Team::SIZE / 32;
            for (int i = me >> 5; i < s; i += NWR) {
                const int32_t row = w.S[i];
                const int64_t e0 = A.row_ptr[row], e1 = A.row_ptr[row + 1];
                double acc = 0.0;
                for (int64_t e = e0 + lane; e < e1; e += 32) {
                    const int pos = find_i32(Js, p, A.col_idx[e]);
                    if (pos >= 0) { acc = fma(A.val[e], w.m[pos], acc); ++cnt; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (row == k) acc -= 1.0;
                if (lane == 0) {
                    w.r[i] = acc;
                    if (!refine) ss = fma(acc, acc, ss);
                }
            }
        } else {
            team.sync();
            for (int i = me; i < s; i += Team::SIZE) {
                const int32_t row = w.S[i];
                const int64_t e0 = A.row_ptr[row], e1 = A.row_ptr[row + 1];
                double acc = 0.0;
                for (int64_t e = e0; e < e1; e += kRowGroup) {
                    int32_t cj[kRowGroup];
                    double av[kRowGroup];
#pragma unroll
                    for (int u = 0; u < kRowGroup; ++u) {
                        cj[u] = (e + u < e1) ? A.col_idx[e + u] : -1;
                        av[u] = (e + u < e1) ? A.val[e + u] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < kRowGroup; ++u) {
                        int pos = (cj[u] >= 0) ? find_J(cj[u]) : -1;
                        if (pos >= 0) { acc = fma(av[u], w.m[pos], acc); ++cnt; }
                    }
                }
                if (row == k) acc -= 1.0;
                w.r[i] = acc;
                if (!refine) ss = fma(acc, acc, ss);
            }
        }
        // the refinement step reads r only; its norm is not formed
        if (!refine) rho = sqrt(team.sum(ss));
        long long nnzJ = team.sum(cnt);
        if (refine) c_ref64 += 2 * nnzJ + 2 * (long long)s;
        else c_res += 2 * nnzJ + 2 * (long long)s;
        team.sync();
    }

    // One step of refinement (FP32_REFINE): r = B m - e in double,
    // m += R^{-1} Q^T (-r) with the factor of the last solve.
    __device__ __forceinline__ void refine_step(T small) {
        const int me = team.rank();
        residual(true);
        int pk = lower_bound_i32(w.I, q, k);
        bool has_k = pk < q && w.I[pk] == k;
        for (int i = me; i < q; i += Team::SIZE) {
            int si = (has_k || i < pk) ? i : i + 1;
            w.rhs[frow(i)] = (T)(-w.r[si]);
        }
        team.sync();
        apply_qt_solve(small);
        for (int c = me; c < p; c += Team::SIZE) w.m[c] += (double)w.rhs[fcol(c)];
        team.sync();
        c_ref += 4LL * q * p + (long long)p * p;
    }

    __device__ __forceinline__ void count_solve(bool append) {
        c_qr += append ? solve_flops(q0, p0, q, p) : solve_flops(0, 0, q, p);
        q0 = q;
        p0 = p;
        c_solves += 1;
        c_pmax = max(c_pmax, p);
        c_qmax = max(c_qmax, q);
    }

    // Solve the LS problem on the current J (Eq. 2.3).  `append`: J extends
    // the previously solved J by Jhat (the paper's QR update; counted as
    // such).  The CTA bins (Caps::append) then update the kept factor instead
    // of refactoring when the last solve left one.
    __device__ bool solve(bool append) {
        const int me = team.rank();
        if constexpr (!is_lane_team<Team>::value) {
            if (cap.append && append && fact_valid) {
                const int st = update_factor();
                if (st == 0) return false;
                if (st > 0) {
                    if (P.precision == RSAI_FP32_REFINE) refine_step(small_last);
                    count_solve(append);
                    return true;
                }
            }
            fact_valid = false;
        }
        build_jhash();
        if (!rows_of_J()) return false;
        if ((int64_t)q * p > cap.bcap) return false;
        // B = A(I,J), zero-filled
        int64_t qp = (int64_t)q * p;
        for (int64_t i = me; i < qp; i += Team::SIZE) w.B[i] = T(0);
        for (int i = me; i < q; i += Team::SIZE) w.rhs[i] = (w.I[i] == k) ? T(1) : T(0);
        team.sync();
        T fro2 = 0;
        // column by column: column J[c] of A (CSC, the entries rows_of_J has just
        // read) placed by the position of its rows in I
        for (int c = me; c < p; c += Team::SIZE) {
            const int32_t j = w.J[c];
            const int64_t e0 = A.col_ptr[j], e1 = A.col_ptr[j + 1];
            T *Bc = w.B + (int64_t)c * q;
            for (int64_t e = e0; e < e1; e += 4) {
                int32_t ri[4];
                T av[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    ri[u] = (e + u < e1) ? A.row_idx[e + u] : -1;
                    av[u] = (e + u < e1) ? csc_value<T>(A, e + u) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (ri[u] >= 0) {
                        const T a = av[u];
                        Bc[find_i32(w.I, q, ri[u])] = a;
                        fro2 += a * a;
                    }
                }
            }
        }
        const T fro2s = team.sum(fro2);
        if constexpr (!is_lane_team<Team>::value) fro2_f = fro2s;
        T fro = sqrt(fro2s);
        team.sync();
        const T small = T(q) * T(2.0 * Unit<T>::u) * fro;
        small_last = small;
        rank_flag = 0;
        if (q < p) {  // more unknowns than rows: only possible for singular A
            for (int c = me; c < p; c += Team::SIZE) w.m[c] = 0.0;
            rank_flag = 1;
            team.sync();
        } else {
            qr_solve(small);
            for (int c = me; c < p; c += Team::SIZE) w.m[c] = (double)w.rhs[c];
            team.sync();
            if (P.precision == RSAI_FP32_REFINE) refine_step(small);
        }
        count_solve(append);
        return true;
    }

    // The QR update of Section 3 (CTA bins).  J grew by Jhat (sorted, in
    // w.buf[0..p - p0)) since the last solve, whose factor is kept in factor
    // order: the rows and columns of earlier solves first, in the order in
    // which they entered, the new ones after them (w.Ip / w.Jp give the factor
    // position of each sorted I / J entry, w.qte holds Q^T e_k).  The new rows
    // of I are zero in the old columns, so the old reflectors act on the
    // appended columns only (qr_update_apply); the appended block is then
    // factored below row p0.  Returns 1 when m holds the solution, 0 on
    // overflow, -1 when the caller has to solve from scratch (q < p).
    __device__ int update_factor() {
        const int me = team.rank();
        const int qo = (int)q0, po = (int)p0, nj = p - po;
        fact_valid = false;
        // Jhat and the old sorted I are kept (rows_of_J reuses buf; the
        // residual rewrites S afterwards)
        for (int b = me; b < nj; b += Team::SIZE) w.Jn[b] = w.buf[b];
        for (int i = me; i < qo; i += Team::SIZE) w.S[i] = w.I[i];
        team.sync();
        build_jhash();
        if (!rows_of_J()) return 0;
        if ((int64_t)q * p > cap.bcap) return 0;
        if (q < p || q > cap.scap || p > cap.scap) return -1;
        // factor rows: old rows keep theirs, new rows follow in ascending order
        int32_t *ipn = w.buf2, *jpn = w.buf;
        int base = 0;
        for (int i0 = 0; i0 < q; i0 += Team::SIZE) {
            const int i = i0 + me;
            const int io = (i < q) ? find_i32(w.S, qo, w.I[i]) : 0;
            const int fnew = (i < q) && (io < 0);
            int tot;
            const int pos = team.scan(fnew, &tot);
            if (i < q) ipn[i] = fnew ? qo + base + pos : w.Ip[io];
            base += tot;
        }
        // factor columns: the old ones keep theirs, Jhat follows in ascending
        // order (an old column is the (c - b)-th of the old sorted J when b
        // entries of Jhat precede it)
        for (int c = me; c < p; c += Team::SIZE) {
            const int b = lower_bound_i32(w.Jn, nj, w.J[c]);
            jpn[c] = (b < nj && w.Jn[b] == w.J[c]) ? po + b : w.Jp[min(max(c - b, 0), po - 1)];
        }
        team.sync();
        for (int i = me; i < q; i += Team::SIZE) w.Ip[i] = ipn[i];
        for (int c = me; c < p; c += Team::SIZE) w.Jp[c] = jpn[c];
        // B: leading dimension q0 -> q in place (column 0 stays).  Old flat
        // index o moves to (o / q0) q + o % q0 >= o, so chunks taken from the
        // top down, each read into registers before any of it is written,
        // never overwrite an entry that is still to be read.
        if (q > qo) {
            constexpr int K = 8;
            constexpr int64_t chunk = (int64_t)K * Team::SIZE;
            for (int64_t hi = (int64_t)qo * po; hi > qo; hi -= chunk) {
                const int64_t lo = max((int64_t)qo, hi - chunk);
                T v[K];
#pragma unroll
                for (int u = 0; u < K; ++u) {
                    const int64_t o = lo + me + (int64_t)u * Team::SIZE;
                    v[u] = (o < hi) ? w.B[o] : T(0);
                }
                team.sync();
#pragma unroll
                for (int u = 0; u < K; ++u) {
                    const int64_t o = lo + me + (int64_t)u * Team::SIZE;
                    if (o < hi) w.B[(o / qo) * q + o % qo] = v[u];
                }
            }
            team.sync();
            const int nr = q - qo;
            for (int64_t idx = me; idx < (int64_t)po * nr; idx += Team::SIZE) {
                const int c = (int)(idx / nr);
                w.B[(int64_t)c * q + qo + (idx - (int64_t)c * nr)] = T(0);
            }
        }
        for (int64_t idx = (int64_t)po * q + me; idx < (int64_t)p * q; idx += Team::SIZE) w.B[idx] = T(0);
        for (int f = qo + me; f < q; f += Team::SIZE) w.qte[f] = T(0);
        team.sync();
        // the appended columns, placed by the factor row of each entry
        T fro2 = 0;
        for (int b = me; b < nj; b += Team::SIZE) {
            const int32_t j = w.Jn[b];
            T *Bc = w.B + (int64_t)(po + b) * q;
            for (int64_t e = A.col_ptr[j]; e < A.col_ptr[j + 1]; ++e) {
                const T a = csc_value<T>(A, e);
                const int ii = find_i32(w.I, q, A.row_idx[e]);
                if (ii >= 0) Bc[w.Ip[ii]] = a;
                fro2 += a * a;
            }
        }
        fro2_f += team.sum(fro2);
        const T small = T(q) * T(2.0 * Unit<T>::u) * sqrt(fro2_f);
        small_last = small;
        // e_k on the new rows: k enters I late when a drop had removed it
        if (me == 0) {
            const int ik = lower_bound_i32(w.I, q, k);
            if (ik < q && w.I[ik] == k && w.Ip[ik] >= qo) w.qte[w.Ip[ik]] = T(1);
        }
        team.sync();
        qr_update_apply<Team, T>(team, w.B, q, p, qo, po, w.vhead, w.tau, (T *)w.stage, cap.stage_bytes, w.Tst,
                                 w.pnb);
        if (cap.stage_bytes > 0 && p >= 2 * kPanel) {
            qr_solve_staged<Team, T>(team, w.B, q, p, w.qte, w.vhead, w.tau, small, (T *)w.stage, cap.stage_bytes,
                                     w.Tst, w.pnb, po, false);
        } else {
            qr_factor_team<Team, T>(team, w.B, q, p, w.qte, w.vhead, w.tau, small, po);
            single_panels(po);
        }
        int rf = 0;
        for (int j = me; j < p; j += Team::SIZE) rf |= (fabs(w.B[(int64_t)j * q + j]) <= small) ? 1 : 0;
        rank_flag = team.sum(rf) > 0 ? 1 : 0;
        for (int j = me; j < p; j += Team::SIZE) w.rhs[j] = w.qte[j];
        team.sync();
        back_substitute_blocked(team, w.B, q, p, w.rhs, small);
        for (int c = me; c < p; c += Team::SIZE) w.m[c] = (double)w.rhs[w.Jp[c]];
        team.sync();
        fact_valid = true;
        return 1;
    }

    // D = D u (dropped columns of J not yet in D); `kept` marks the columns
    // that stay.  False if D outgrows its capacity.
    template <class Kept> __device__ bool note_dropped(Kept kept) {
        const int me = team.rank();
        int nt = 0;
        for (int c0 = 0; c0 < p; c0 += Team::SIZE) {
            const int c = c0 + me;
            const int f = (c < p) && !kept(c) && find_i32(w.D, nD, w.J[c]) < 0;
            int tot;
            const int pos = team.scan(f, &tot);
            if (f) w.buf2[nt + pos] = w.J[c];
            nt += tot;
        }
        team.sync();
        if (nD + nt > cap.dcap) return false;
        // merge by ranks (both sorted and disjoint) into buf, then back into D
        for (int a = me; a < nD; a += Team::SIZE) w.buf[a + lower_bound_i32(w.buf2, nt, w.D[a])] = w.D[a];
        for (int b = me; b < nt; b += Team::SIZE) w.buf[b + lower_bound_i32(w.D, nD, w.buf2[b])] = w.buf2[b];
        team.sync();
        nD += nt;
        for (int a = me; a < nD; a += Team::SIZE) w.D[a] = w.buf[a];
        team.sync();
        return true;
    }

    // Eq. 4.3: drop |m_j| <= tau, keep at least the largest, re-solve once.
    // Magnitudes are compared as ordered integer keys (exact).
    // Returns 1 if J lost entries (the caller re-solves once), 0 if not, -1
    // if the set of dropped columns outgrows this bin.
    __device__ int drop() {
        if (P.drop_mode == RSAI_DROP_NONE) return 0;
        const int me = team.rank();
        const int blk = P.col_block ? P.col_block[k] : 0;
        const double tau = (P.drop_mode == RSAI_DROP_ADAPTIVE) ? P.eps / ((double)p * P.norm1[blk]) : P.tau_fixed[blk];
        const long long tk = abskey(tau);
        int nkeep = 0;
        long long ba = -1;
        int bi = INT32_MAX;
        for (int c = me; c < p; c += Team::SIZE) {
            long long a = abskey(w.m[c]);
            nkeep += (a > tk);
            if (dom_before(a, c, ba, bi)) { ba = a; bi = c; }
        }
        const int keep_total = team.sum(nkeep);
        if (keep_total == p) return 0;
        if (keep_total == 0) {
            team.argmax(ba, bi);
            if (p == 1) return 0;
            if (!note_dropped([&](int c) { return c == bi; })) return -1;
            int32_t jb = w.J[bi];
            team.sync();
            if (me == 0) w.J[0] = jb;
            p = 1;
            team.sync();
        } else {
            if (!note_dropped([&](int c) { return abskey(w.m[c]) > tk; })) return -1;
            int base = 0;
            for (int c0 = 0; c0 < p; c0 += Team::SIZE) {
                int c = c0 + me;
                int f = (c < p) && (abskey(w.m[c]) > tk);
                int tot;
                int pos = team.scan(f, &tot);
                if (f) w.Jn[base + pos] = w.J[c];
                base += tot;
            }
            team.sync();
            for (int c = me; c < base; c += Team::SIZE) w.J[c] = w.Jn[c];
            p = base;
            team.sync();
        }
        c_drops += 1;
        return 1;
    }

    // Top-c dominant rows of S \ R (Algorithm 1, Eq. 3.2) into w.Rhat; returns
    // their number (0: no candidate left).  |r_i| enters only as ordered
    // integer keys; the tie band needs three double operations per call.
    __device__ int dominant_rows() {
        const int me = team.rank();
        long long rinf = 0;
        for (int i = me; i < s; i += Team::SIZE) rinf = max(rinf, abskey(w.r[i]));
        rinf = team.maxv(rinf);
        const double band = P.tie_band * key_value(rinf);
        const long long bk = abskey(band);
        int ncand = 0;
        for (int i = me; i < s; i += Team::SIZE)
            ncand += (abskey(w.r[i]) > bk) && (find_i32(w.Rset, nR, w.S[i]) < 0);
        ncand = team.sum(ncand);
        if (ncand == 0) return 0;
        const int c = P.c;
        const bool take_all = ncand <= c;
        long long hik = 0, lob = 0;
        if (!take_all) {
            // the c-th element of the (|r| desc, i asc) order: c rounds of argmax,
            // each over the candidates strictly after the previous pick
            long long pa = LLONG_MAX;
            int pi = -1;
            for (int t = 0; t < c; ++t) {
                long long ba = -1;
                int bi = INT32_MAX;
                for (int i = me; i < s; i += Team::SIZE) {
                    long long a = abskey(w.r[i]);
                    int32_t row = w.S[i];
                    if (a > bk && dom_before(pa, pi, a, row) && dom_before(a, row, ba, bi) &&
                        find_i32(w.Rset, nR, row) < 0) {
                        ba = a;
                        bi = row;
                    }
                }
                team.argmax(ba, bi);
                pa = ba;
                pi = bi;
            }
            const double v = key_value(pa);
            hik = abskey(v + band);
            lob = __double_as_longlong(v - band);  // negative bit pattern if v - band < 0
        }
        // selection in index order: all candidates, or (above v + band) +
        // (lowest-index entries within [v - band, v + band] up to c)
        int nabove = 0;
        if (!take_all) {
            for (int i = me; i < s; i += Team::SIZE) {
                long long a = abskey(w.r[i]);
                nabove += (a > bk) && (a > hik) && (find_i32(w.Rset, nR, w.S[i]) < 0);
            }
            nabove = team.sum(nabove);
        }
        const int need = c - nabove;
        int base = 0, tbase = 0;
        for (int i0 = 0; i0 < s; i0 += Team::SIZE) {
            int i = i0 + me;
            int cand = 0, above = 0, tie = 0;
            if (i < s) {
                long long a = abskey(w.r[i]);
                cand = (a > bk) && (find_i32(w.Rset, nR, w.S[i]) < 0);
                if (cand && !take_all) {
                    above = a > hik;
                    tie = (a >= lob) && (a <= hik);
                }
            }
            int ttot;
            int trank = team.scan(tie, &ttot);
            int sel = take_all ? cand : (above || (tie && (tbase + trank) < need));
            int tot;
            int pos = team.scan(sel, &tot);
            if (sel) w.Rhat[base + pos] = w.S[i];
            base += tot;
            tbase += ttot;
        }
        team.sync();
        return base;
    }

    // R = R u Rhat (sorted); false if R outgrows its capacity
    __device__ bool add_to_R(int nh) {
        if (nR + nh > cap.rcap) return false;
        if (team.rank() == 0) {
            for (int t = 0; t < nh; ++t) {
                int32_t x = w.Rhat[t];
                int at = nR + t;
                while (at > 0 && w.Rset[at - 1] > x) { w.Rset[at] = w.Rset[at - 1]; --at; }
                w.Rset[at] = x;
            }
        }
        nR += nh;
        team.sync();
        return true;
    }

    // Jhat = cols(A(Rhat,:)) \ J into w.buf; returns |Jhat| or -1 on overflow.
    // The rows of Rhat are dealt out to the team's ranks, as many passes as
    // |Rhat| (<= c <= 32) needs on a team of 16.
    __device__ int new_columns(int nh) {
        const int me = team.rank();
        int tot = 0;
        for (int t0 = 0; t0 < nh; t0 += Team::SIZE) {
            const int t = t0 + me;
            int len = 0;
            int64_t st = 0;
            if (t < nh) {
                st = A.row_ptr[w.Rhat[t]];
                len = (int)(A.row_ptr[w.Rhat[t] + 1] - st);
            }
            int part;
            const int off = tot + team.scan(len, &part);
            if (next_pow2(tot + part) > cap.scap) return -1;
            for (int e = 0; e < len; e += 4) {
                int32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = (e + u < len) ? A.col_idx[st + e + u] : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (e + u < len) w.buf[off + e + u] = v[u];
            }
            tot += part;
        }
        team.sync();
        team_sort_i32(team, w.buf, tot);
        int nu = team_unique_i32(team, w.buf, tot, w.buf2);
        int base = 0;
        for (int i0 = 0; i0 < nu; i0 += Team::SIZE) {
            int i = i0 + me;
            int f = (i < nu) && (find_J(w.buf2[i]) < 0);
            int t2;
            int pos = team.scan(f, &t2);
            if (f) w.buf[base + pos] = w.buf2[i];
            base += t2;
        }
        team.sync();
        return base;
    }

    // J = J u Jhat (both sorted, disjoint) by merge ranks
    __device__ bool merge_J(int nj) {
        const int me = team.rank();
        if (p + nj > cap.pcap) return false;
        for (int a = me; a < p; a += Team::SIZE) w.Jn[a + lower_bound_i32(w.buf, nj, w.J[a])] = w.J[a];
        for (int b = me; b < nj; b += Team::SIZE) w.Jn[b + lower_bound_i32(w.J, p, w.buf[b])] = w.buf[b];
        team.sync();
        p += nj;
        for (int a = me; a < p; a += Team::SIZE) w.J[a] = w.Jn[a];
        team.sync();
        return true;
    }

    // algorithmic bytes of columns entering J for the first time: 12 per
    // nonzero + 16 of pointers (a column dropped earlier was charged then)
    __device__ void note_bytes_columns(int from, int count, const int32_t *list) {
        long long b = 0;
        for (int t = from + team.rank(); t < from + count; t += Team::SIZE) {
            int32_t j = list[t];
            if (find_i32(w.D, nD, j) < 0) b += 12 * (A.col_ptr[j + 1] - A.col_ptr[j]) + 16;
        }
        c_bytes += team.sum(b);
    }

    // ---- frozen pattern (refit, backward) ----

    // J = Jk (sorted, length pk): false if it does not fit this bin
    __device__ bool load_pattern(const int32_t *Jk, int pk) {
        p = pk; q = 0; s = 0; nR = 0; l = 0; nD = 0; q0 = 0; p0 = 0; rank_flag = 0; rho = 0.0;
        if constexpr (!is_lane_team<Team>::value) fact_valid = false;
        c_qr = c_res = c_ref = c_ref64 = c_bytes = c_sel = 0;
        c_solves = c_drops = c_pmax = c_qmax = 0;
        if (pk > cap.pcap || pk < 1) return false;
        for (int c = team.rank(); c < pk; c += Team::SIZE) w.J[c] = Jk[c];
        team.sync();
        return true;
    }

    // out[i] = sum_c A(I_i, J_c) zc[c] over the rows of I, in double
    __device__ void rows_times(const double *zc, double *out) {
        for (int i = team.rank(); i < q; i += Team::SIZE) {
            const int32_t row = w.I[i];
            const int64_t e0 = A.row_ptr[row], e1 = A.row_ptr[row + 1];
            double acc = 0.0;
            for (int64_t e = e0; e < e1; ++e) {
                const int c = find_J(A.col_idx[e]);
                if (c >= 0) acc = fma(A.val[e], zc[c], acc);
            }
            out[i] = acc;
        }
        team.sync();
    }

    // out[c] = sum_i A(I_i, J_c) v[i] over the columns of J, in double
    __device__ void cols_times(const double *v, double *out) {
        for (int c = team.rank(); c < p; c += Team::SIZE) {
            const int32_t j = w.J[c];
            double acc = 0.0;
            for (int64_t e = A.col_ptr[j]; e < A.col_ptr[j + 1]; ++e)
                acc = fma(A.cval[e], v[find_i32(w.I, q, A.row_idx[e])], acc);
            out[c] = acc;
        }
        team.sync();
    }

    // rhs[0..p) <- (R^T R)^{-1} rhs[0..p) with R from the last solve
    __device__ void normal_solve(T small) {
        const int me = team.rank();
        for (int i = 0; i < p; ++i) {  // R^T y = rhs (forward, column-oriented)
            T d = w.B[(int64_t)i * q + i];
            T yi = (fabs(d) <= small) ? T(0) : w.rhs[i] / d;
            team.sync();
            for (int c = i + 1 + me; c < p; c += Team::SIZE) w.rhs[c] -= w.B[(int64_t)c * q + i] * yi;
            if (me == 0) w.rhs[i] = yi;
            team.sync();
        }
        if constexpr (is_lane_team<Team>::value) back_substitute_team(team, w.B, q, p, w.rhs, small);
        else back_substitute_blocked(team, w.B, q, p, w.rhs, small);
    }

    // Refit: solve on the loaded pattern, then the residual.  Returns false on
    // overflow.
    __device__ bool refit() {
        if (!solve(false)) return false;
        residual();
        return true;
    }

    // Adjoint of the frozen-pattern solve of column k (see rsai_backward):
    //   x = m_k(J_k), r = B x - e_k(I_k), z = (B^T B)^{-1} g (one FP64
    //   refinement step in FP32_REFINE), w = B z;  writes r, w over I_k and
    //   alpha = -z + 2 gr x, x over J_k.
    __device__ bool adjoint(const Frozen &F) {
        const int me = team.rank();
        if (!solve(false)) return false;
        residual();
        const int64_t mo = F.Mcolptr[k];
        for (int c = me; c < p; c += Team::SIZE) w.z[c] = F.grad_M[F.Mcsc_to_csr[mo + c]];
        team.sync();
        const T small = small_last;
        for (int c = me; c < p; c += Team::SIZE) w.rhs[c] = (T)w.z[c];
        team.sync();
        normal_solve(small);
        if (P.precision == RSAI_FP32_REFINE) {
            // one refinement step in double: z = z0 + (R^T R)^{-1} (g - B^T B z0);
            // g stays in z, z0 goes to buf, B z0 to wv, B^T B z0 to buf2
            double *z0 = reinterpret_cast<double *>(w.buf);
            double *u = reinterpret_cast<double *>(w.buf2);
            for (int c = me; c < p; c += Team::SIZE) z0[c] = (double)w.rhs[c];
            team.sync();
            rows_times(z0, w.wv);
            cols_times(w.wv, u);
            for (int c = me; c < p; c += Team::SIZE) w.rhs[c] = (T)(w.z[c] - u[c]);
            team.sync();
            normal_solve(small);
            for (int c = me; c < p; c += Team::SIZE) w.z[c] = z0[c] + (double)w.rhs[c];
            team.sync();
        } else {
            for (int c = me; c < p; c += Team::SIZE) w.z[c] = (double)w.rhs[c];
            team.sync();
        }
        rows_times(w.z, w.wv);
        const double gr = F.grad_rho2 ? F.grad_rho2[k] : 0.0;
        const int64_t qo = F.qoff[k];
        int pk = lower_bound_i32(w.I, q, k);
        bool has_k = pk < q && w.I[pk] == k;
        for (int i = me; i < q; i += Team::SIZE) {
            const int si = (has_k || i < pk) ? i : i + 1;
            F.poolI[qo + i] = w.I[i];
            F.poolR[qo + i] = w.r[si];
            F.poolW[qo + i] = w.wv[i];
        }
        for (int c = me; c < p; c += Team::SIZE) {
            const double x = w.m[c];
            F.alphaM[mo + c] = -w.z[c] + 2.0 * gr * x;
            F.xM[mo + c] = x;
        }
        team.sync();
        return true;
    }

    // First solve, J = {k} (Eq. 2.3 with p = 1): I = rows of A(:,k), which the
    // CSC keeps ascending, and m_kk = a_kk / ||a_k||^2 in double (the closed
    // form of the 1-column LS problem; no sort, tile or QR needed).
    __device__ bool initial_solve() {
        const int me = team.rank();
        const int64_t e0 = A.col_ptr[k];
        const int len = (int)(A.col_ptr[k + 1] - e0);
        if (len > cap.qcap) return false;
        double nn = 0.0;
        int kpos = -1;
        for (int i = me; i < len; i += Team::SIZE) {
            const int32_t r = A.row_idx[e0 + i];
            const double a = A.cval[e0 + i];
            w.I[i] = r;
            nn = fma(a, a, nn);
            if (r == k) kpos = i;
        }
        nn = team.sum(nn);
        // a_kk found by its position (an integer reduction), not summed in double
        kpos = team.maxv(kpos);
        const double akk = kpos >= 0 ? A.cval[e0 + kpos] : 0.0;
        q = len;
        build_jhash();
        if (me == 0) w.m[0] = (nn > 0.0) ? akk / nn : 0.0;
        rank_flag = (nn > 0.0) ? 0 : 1;
        c_qr += solve_flops(0, 0, q, 1);
        q0 = q;
        p0 = 1;
        c_solves += 1;
        c_pmax = max(c_pmax, 1);
        c_qmax = max(c_qmax, q);
        team.sync();
        return true;
    }

    __device__ int run() {
        const int me = team.rank();
        p = 1; q = 0; s = 0; nR = 0; l = 0; nD = 0; q0 = 0; p0 = 0; rank_flag = 0; rho = 0.0;
        if constexpr (!is_lane_team<Team>::value) fact_valid = false;
        c_qr = c_res = c_ref = c_ref64 = c_bytes = c_sel = 0;
        c_solves = c_drops = c_pmax = c_qmax = 0;
        if (me == 0) w.J[0] = k;
        team.sync();
        if (P.init_a) {
            // Algorithm 1 started from the initial pattern of A, solved by the
            // general path below
            long long b = 0;
            const int len = pattern_of_column(team, A.col_ptr, A.row_idx, k, cap.pcap, w.J, &b);
            if (len < 0) return COL_OVERFLOW;
            p = len;
            c_bytes += b;
        } else {
            c_bytes += 12 * (A.col_ptr[k + 1] - A.col_ptr[k]) + 16;
        }
        // One solve site: the first pass of every round solves on the new J
        // (appended to the last factor after the first round), the second
        // re-solves after a drop (Eq. 4.3); then the residual (Eq. 2.4).
        bool append = false, first = true;
        for (;;) {
            for (int pass = 0; pass < 2; ++pass) {
                // one call site of solve() (it is large and inlined): the
                // closed form covers the first solve of J = {k} only
                if (first && !P.init_a) {
                    if (!initial_solve()) return COL_OVERFLOW;
                } else if (!solve(append)) {
                    return COL_OVERFLOW;
                }
                first = false;
                append = false;
                if (pass == 1) break;
                const int dr = drop();
                if (dr < 0) return COL_OVERFLOW;
                if (dr == 0) break;
            }
            residual();
            bool grown = false;
            while (!grown && rho > P.eps && l < P.l_max) {
                if (P.spai) {
                    const SpaiPick pk = spai_select(team, A, P.c, P.tie_band, cap.scap, w.S, w.r, s, jset(), w.buf,
                                                    w.buf2, w.sc, w.Rhat);
                    c_bytes += pk.bytes;
                    c_sel += pk.sel;
                    const int na = pk.na;
                    if (na < 0) return COL_OVERFLOW;
                    if (na == 0) break;  // no candidate: nothing can be added later either
                    ++l;
                    note_bytes_columns(0, na, w.buf);
                    if (!merge_J(na)) return COL_OVERFLOW;
                    grown = true;
                    continue;
                }
                int nh = dominant_rows();
                if (nh == 0) break;
                if (!add_to_R(nh)) return COL_OVERFLOW;
                {
                    long long b = 0;
                    for (int t = me; t < nh; t += Team::SIZE) b += 4 * (A.row_ptr[w.Rhat[t] + 1] - A.row_ptr[w.Rhat[t]]) + 16;
                    c_bytes += team.sum(b);
                }
                int nj = new_columns(nh);
                if (nj < 0) return COL_OVERFLOW;
                ++l;
                if (nj == 0) continue;  // empty Jhat: back to the loop test (Algorithm 1)
                note_bytes_columns(0, nj, w.buf);
                if (!merge_J(nj)) return COL_OVERFLOW;
                grown = true;
            }
            if (!grown) break;
            append = true;
        }
        c_bytes += 36LL * p;
        return COL_DONE;
    }
};

}  // namespace rsai
