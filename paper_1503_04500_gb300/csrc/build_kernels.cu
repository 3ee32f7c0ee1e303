// build_kernels.cu -- the size bins of the RSAI(tol) column algorithm and
// their launchers (input checks, ||A||_1, statistics and the assembly of M
// are in setup_kernels.cu).
//
// Bins (one persistent launch each, columns pulled from an atomic queue; the
// columns are independent, Section 2 Eq. 2.2):
//   H  half a warp per column, two columns per warp, workspace in shared
//      memory (the smallest LS problems: |I| <= 48, |J| <= 16, e.g. 3-D
//      7-point stencils)
//   W  one warp per column, workspace in shared memory (small LS problems,
//      e.g. stencil matrices: |I| <= 64, |J| <= 32)
//   W2 the same kernel with |I| <= 128 (fewer warps per SM)
//   C  one CTA per column, workspace in shared memory (up to ~200 KB)
//   G  one CTA per column, workspace in a global-memory slab per CTA (the
//      long tail of matrices with dense rows, Section 4 "row irregular")
// A column that outgrows a bin is pushed to the next bin's queue and
// restarted there from J = {k}; the result is the same column of M.
#include "kernels.h"

namespace rsai {

// ---------------------------------------------------------------------------
// the bins

template <class Team, typename T>
__device__ void emit_or_forward(const Team &team, Column<Team, T> &col, int st, const ColQueue &Q,
                                const ColOut &O, bool last_bin, int bin) {
    const int me = team.rank();
    const int32_t k = col.k;
    Work<T> &w = col.w;
    if (st == COL_OVERFLOW) {
        if (!last_bin) {
            if (me == 0) {
                uint32_t pos = atomicAdd(Q.ovf_count, 1u);
                if ((int64_t)pos < Q.ovf_cap) Q.ovf_cols[pos] = k;
                else set_error(O.err, RSAI_ERR_WORKSPACE);
            }
        } else if (me == 0) {
            O.col_off[k] = 0;
            O.col_len[k] = 0;
            O.rho[k] = NAN;
            O.loops[k] = 0;
            O.flags[k] = RSAI_COL_FAILED;
            w.ctr[CTR_FAILED] += 1;
            set_error(O.err, RSAI_ERR_WORKSPACE);
        }
        team.sync();
        return;
    }
    const int p = col.p;
    unsigned long long off = 0;
    if (me == 0) off = atomicAdd(O.pool_top, (unsigned long long)p);
    off = team.bcast(off, 0);
    if ((int64_t)(off + p) > O.pool_cap) {
        if (me == 0) {
            O.col_off[k] = 0;
            O.col_len[k] = 0;
            O.rho[k] = NAN;
            O.flags[k] = RSAI_COL_FAILED;
            w.ctr[CTR_FAILED] += 1;
            set_error(O.err, RSAI_ERR_WORKSPACE);
        }
        team.sync();
        return;
    }
    int fin = 1;
    for (int c = me; c < p; c += Team::SIZE) {
        O.pool_rows[off + c] = w.J[c];
        O.pool_vals[off + c] = w.m[c];
        fin &= finite_bits(w.m[c]) ? 1 : 0;
    }
    fin = team.sum(1 - fin) == 0 && finite_bits(col.rho);
    if (me == 0) {
        int flags = (col.rho <= col.P.eps ? RSAI_COL_CONVERGED : 0) | (col.rank_flag ? RSAI_COL_RANK : 0) |
                    (fin ? 0 : RSAI_COL_NONFINITE);
        O.col_off[k] = (int64_t)off;
        O.col_len[k] = p;
        O.col_q[k] = col.q;
        O.rho[k] = col.rho;
        O.loops[k] = col.l;
        O.flags[k] = flags;
        w.ctr[CTR_QR] += col.c_qr;
        w.ctr[CTR_RES] += col.c_res;
        w.ctr[CTR_REFINE] += col.c_ref;
        w.ctr[CTR_REFINE64] += col.c_ref64;
        w.ctr[CTR_BYTES] += col.c_bytes;
        w.ctr[CTR_SELECT] += col.c_sel;
        w.ctr[CTR_LOOPS] += col.l;
        w.ctr[CTR_SOLVES] += col.c_solves;
        w.ctr[CTR_DROPS] += col.c_drops;
        w.ctr[CTR_PMAX] = max(w.ctr[CTR_PMAX], (long long)col.c_pmax);
        w.ctr[CTR_QMAX] = max(w.ctr[CTR_QMAX], (long long)col.c_qmax);
        w.ctr[CTR_COLS] += 1;
        w.ctr[CTR_RANK] += col.rank_flag ? 1 : 0;
        w.ctr[CTR_NONFINITE] += fin ? 0 : 1;
    }
    team.sync();
    (void)bin;
}

// A frozen-pattern column that does not fit this bin: forward or fail
__device__ __forceinline__ void forward_frozen(int me, const ColQueue &Q, const ColOut &O, int32_t k,
                                               bool last_bin, long long *ctr) {
    if (me != 0) return;
    if (!last_bin) {
        uint32_t pos = atomicAdd(Q.ovf_count, 1u);
        if ((int64_t)pos < Q.ovf_cap) Q.ovf_cols[pos] = k;
        else set_error(O.err, RSAI_ERR_WORKSPACE);
    } else {
        ctr[CTR_FAILED] += 1;
        set_error(O.err, RSAI_ERR_WORKSPACE);
    }
}

template <int MODE, class Team, typename T>
__device__ void run_queue(const Team &team, Work<T> &w, const DevA &A, const DevParams &P, const Caps &cap,
                          const ColQueue &Q, const ColOut &O, const Frozen &F, unsigned long long *gctr,
                          bool last_bin, int bin) {
    const int me = team.rank();
    for (int i = me; i < CTR_COUNT; i += Team::SIZE) w.ctr[i] = 0;
    team.sync();
    const int64_t nq = Q.count ? (int64_t)(*(volatile const uint32_t *)Q.count) : Q.n;
    // Half-warp teams: the two halves of a warp start their columns together
    // (one vote of the whole warp per column), so that similar columns run in
    // step and each instruction serves both; a half whose queue is empty sits
    // the round out.  The loop ends only when neither half has a column, so
    // every lane of the warp reaches each whole-warp vote and synchronisation.
    constexpr bool paired = std::is_same<Team, HalfTeam>::value;
    for (;;) {
        uint32_t idx = 0;
        if (me == 0) idx = atomicAdd(Q.next, 1u);
        idx = team.bcast(idx, 0);
        const bool have = (int64_t)idx < nq;
        if constexpr (paired) {
            if (!__any_sync(0xffffffffu, have)) break;
        } else {
            if (!have) break;
        }
        if (have) {
            const int32_t k = Q.cols ? Q.cols[idx] : (int32_t)idx;
            Column<Team, T> col(team, A, P, cap, w, k);
            if constexpr (MODE == MODE_BUILD) {
                int st = col.run();
                emit_or_forward(team, col, st, Q, O, last_bin, bin);
            } else {
                const int64_t mo = F.Mcolptr[k];
                const int pk = (int)(F.Mcolptr[k + 1] - mo);
                bool ok = col.load_pattern(F.Mrows + mo, pk);
                if (ok) {
                    if constexpr (MODE == MODE_REFIT) ok = col.refit();
                    else ok = col.adjoint(F);
                }
                if (!ok) {
                    forward_frozen(me, Q, O, k, last_bin, w.ctr);
                } else {
                    if constexpr (MODE == MODE_REFIT) {
                        for (int c = me; c < pk; c += Team::SIZE) F.Mval_csr[F.Mcsc_to_csr[mo + c]] = w.m[c];
                        if (me == 0) F.rho2[k] = col.rho * col.rho;
                    }
                    if (me == 0) w.ctr[CTR_COLS] += 1;
                }
                team.sync();
            }
        }
        if constexpr (paired) __syncwarp();
    }
    team.sync();
    if (me == 0) {
        for (int i = 0; i < CTR_COUNT; ++i) {
            if (i == CTR_PMAX || i == CTR_QMAX)
                atomicMax(&gctr[i], (unsigned long long)w.ctr[i]);
            else if (w.ctr[i] != 0)
                atomicAdd(&gctr[i], (unsigned long long)w.ctr[i]);
        }
        if (w.ctr[CTR_COLS] != 0) atomicAdd(&gctr[CTR_COUNT + bin], (unsigned long long)w.ctr[CTR_COLS]);
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256, (sizeof(T) == 8 ? 1 : 2))
    k_bin_warp(DevA A, DevParams P, Caps cap, ColQueue Q, ColOut O, Frozen F, unsigned long long *gctr, int last_bin) {
    extern __shared__ __align__(16) char smem[];
    const int wid = threadIdx.x >> 5;
    Work<T> w;
    w.carve(smem + (size_t)wid * Work<T>::bytes(cap), cap);
    WarpTeam team;
    run_queue<MODE>(team, w, A, P, cap, Q, O, F, gctr, last_bin != 0, 0);
}

// Bin H: every half warp is a team with its own workspace and its own column
template <typename T, int MODE>
__global__ void __launch_bounds__(256, (sizeof(T) == 8 ? 1 : 2))
    k_bin_half(DevA A, DevParams P, Caps cap, ColQueue Q, ColOut O, Frozen F, unsigned long long *gctr, int last_bin) {
    extern __shared__ __align__(16) char smem[];
    const int tid = threadIdx.x >> 4;
    Work<T> w;
    w.carve(smem + (size_t)tid * Work<T>::bytes(cap), cap);
    HalfTeam team;
    run_queue<MODE>(team, w, A, P, cap, Q, O, F, gctr, last_bin != 0, kBinHalf);
}

template <typename T, int NT, int MODE>
__global__ void __launch_bounds__(NT, 1)
    k_bin_block(DevA A, DevParams P, Caps cap, ColQueue Q, ColOut O, Frozen F, unsigned long long *gctr,
                int last_bin, char *gwork, size_t gstride, int bin) {
    extern __shared__ __align__(16) char smem[];
    __shared__ unsigned long long red[NT / 32 + 1];
    __shared__ int redi[NT / 32 + 1];
    Work<T> w;
    if (gwork) {
        w.carve(gwork + (size_t)blockIdx.x * gstride, cap);
        w.stage = smem;  // shared memory is free for panel staging
    } else {
        w.carve(smem, cap);
    }
    BlockTeam<NT> team{red, redi};
    run_queue<MODE>(team, w, A, P, cap, Q, O, F, gctr, last_bin != 0, bin);
}

// ---------------------------------------------------------------------------
// host-side launchers

template <typename T>
size_t warp_bin_smem(const Caps &c, int warps) { return (size_t)warps * Work<T>::bytes(c); }

template <typename T>
size_t half_bin_smem(const Caps &c, int warps) { return (size_t)(2 * warps) * Work<T>::bytes(c); }

template <typename T>
size_t work_bytes(const Caps &c) { return Work<T>::bytes(c); }

template size_t work_bytes<float>(const Caps &);
template size_t work_bytes<double>(const Caps &);

// Lets `fn` take up to the device's opt-in shared memory per block, less its
// static shared memory.  The limit is raised to that largest value instead of
// to each launch's size, so that every launch recorded in a CUDA graph stays
// within the function's limit whatever was launched (or planned) after it.
template <typename F> static void allow_full_smem(F fn) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, fn);  // static + dynamic must not exceed the opt-in limit
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <typename T, int MODE>
static cudaError_t launch_warp_t(int grid, int warps, const DevA &A, const DevParams &P, const Caps &cap,
                                 const ColQueue &Q, const ColOut &O, const Frozen &F, unsigned long long *gctr,
                                 bool last, cudaStream_t st) {
    size_t smem = warp_bin_smem<T>(cap, warps);
    allow_full_smem(k_bin_warp<T, MODE>);
    k_bin_warp<T, MODE><<<grid, warps * 32, smem, st>>>(A, P, cap, Q, O, F, gctr, last ? 1 : 0);
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t launch_half_t(int grid, int warps, const DevA &A, const DevParams &P, const Caps &cap,
                                 const ColQueue &Q, const ColOut &O, const Frozen &F, unsigned long long *gctr,
                                 bool last, cudaStream_t st) {
    size_t smem = half_bin_smem<T>(cap, warps);
    allow_full_smem(k_bin_half<T, MODE>);
    k_bin_half<T, MODE><<<grid, warps * 32, smem, st>>>(A, P, cap, Q, O, F, gctr, last ? 1 : 0);
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t launch_block_t(int grid, const DevA &A, const DevParams &P, const Caps &cap, const ColQueue &Q,
                                  const ColOut &O, const Frozen &F, unsigned long long *gctr, bool last, char *gwork,
                                  size_t gstride, int bin, cudaStream_t st) {
    size_t smem = gwork ? (size_t)cap.stage_bytes : Work<T>::bytes(cap);
    allow_full_smem(k_bin_block<T, kBlockThreads, MODE>);
    k_bin_block<T, kBlockThreads, MODE><<<grid, kBlockThreads, smem, st>>>(A, P, cap, Q, O, F, gctr, last ? 1 : 0,
                                                                          gwork, gstride, bin);
    return cudaGetLastError();
}

cudaError_t launch_bin_warp(int mode, bool fp32, int grid, int warps, const DevA &A, const DevParams &P,
                            const Caps &cap, const ColQueue &Q, const ColOut &O, const Frozen &F,
                            unsigned long long *gctr, bool last, cudaStream_t st) {
    if (fp32) {
        if (mode == MODE_BUILD) return launch_warp_t<float, MODE_BUILD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
        if (mode == MODE_REFIT) return launch_warp_t<float, MODE_REFIT>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
        return launch_warp_t<float, MODE_BACKWARD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
    }
    if (mode == MODE_BUILD) return launch_warp_t<double, MODE_BUILD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
    if (mode == MODE_REFIT) return launch_warp_t<double, MODE_REFIT>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
    return launch_warp_t<double, MODE_BACKWARD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
}

cudaError_t launch_bin_half(int mode, bool fp32, int grid, int warps, const DevA &A, const DevParams &P,
                            const Caps &cap, const ColQueue &Q, const ColOut &O, const Frozen &F,
                            unsigned long long *gctr, bool last, cudaStream_t st) {
    if (fp32) {
        if (mode == MODE_BUILD) return launch_half_t<float, MODE_BUILD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
        if (mode == MODE_REFIT) return launch_half_t<float, MODE_REFIT>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
        return launch_half_t<float, MODE_BACKWARD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
    }
    if (mode == MODE_BUILD) return launch_half_t<double, MODE_BUILD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
    if (mode == MODE_REFIT) return launch_half_t<double, MODE_REFIT>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
    return launch_half_t<double, MODE_BACKWARD>(grid, warps, A, P, cap, Q, O, F, gctr, last, st);
}

cudaError_t launch_bin_block(int mode, bool fp32, int grid, const DevA &A, const DevParams &P, const Caps &cap,
                             const ColQueue &Q, const ColOut &O, const Frozen &F, unsigned long long *gctr,
                             bool last, char *gwork, size_t gstride, int bin, cudaStream_t st) {
#define RSAI_LB(TT, MM) launch_block_t<TT, MM>(grid, A, P, cap, Q, O, F, gctr, last, gwork, gstride, bin, st)
    if (fp32) {
        if (mode == MODE_BUILD) return RSAI_LB(float, MODE_BUILD);
        if (mode == MODE_REFIT) return RSAI_LB(float, MODE_REFIT);
        return RSAI_LB(float, MODE_BACKWARD);
    }
    if (mode == MODE_BUILD) return RSAI_LB(double, MODE_BUILD);
    if (mode == MODE_REFIT) return RSAI_LB(double, MODE_REFIT);
    return RSAI_LB(double, MODE_BACKWARD);
#undef RSAI_LB
}


int occupancy_bin_warp(bool fp32, int warps, const Caps &cap) {
    int nb = 0;
    size_t smem = fp32 ? warp_bin_smem<float>(cap, warps) : warp_bin_smem<double>(cap, warps);
    if (fp32) {
        allow_full_smem(k_bin_warp<float, MODE_BUILD>);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bin_warp<float, MODE_BUILD>, warps * 32, smem);
    } else {
        allow_full_smem(k_bin_warp<double, MODE_BUILD>);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bin_warp<double, MODE_BUILD>, warps * 32, smem);
    }
    return nb;
}

int occupancy_bin_half(bool fp32, int warps, const Caps &cap) {
    int nb = 0;
    size_t smem = fp32 ? half_bin_smem<float>(cap, warps) : half_bin_smem<double>(cap, warps);
    if (fp32) {
        allow_full_smem(k_bin_half<float, MODE_BUILD>);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bin_half<float, MODE_BUILD>, warps * 32, smem);
    } else {
        allow_full_smem(k_bin_half<double, MODE_BUILD>);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bin_half<double, MODE_BUILD>, warps * 32, smem);
    }
    return nb;
}

int occupancy_bin_block(bool fp32, const Caps &cap, bool global_work) {
    int nb = 0;
    size_t smem = global_work ? 0 : (fp32 ? Work<float>::bytes(cap) : Work<double>::bytes(cap));
    if (fp32) {
        allow_full_smem(k_bin_block<float, kBlockThreads, MODE_BUILD>);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bin_block<float, kBlockThreads, MODE_BUILD>,
                                                      kBlockThreads, smem);
    } else {
        allow_full_smem(k_bin_block<double, kBlockThreads, MODE_BUILD>);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bin_block<double, kBlockThreads, MODE_BUILD>,
                                                      kBlockThreads, smem);
    }
    return nb;
}

}  // namespace rsai
