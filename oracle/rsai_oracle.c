/*
 * rsai_oracle.c -- plain FP64 CPU oracle of RSAI(tol) (Jia & Kang,
 * "A residual based sparse approximate inverse preconditioning procedure for
 * large sparse linear systems").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.  It is written to be read
 * against the paper, not to be fast: every LS problem is refactored from
 * scratch by a textbook Householder QR, sets are sorted arrays, and the loop
 * follows Algorithm 1 in the paper's order.
 *
 * What it computes, per column k (Section 2 Eq. 2.2-2.4, Section 3 Algorithm 1,
 * Section 4 Eq. 4.3; or, with select_mode SPAI, the selection of Section 2
 * Eqs. 2.5-2.7 in place of the dominant rows):
 *   J = J0(k), R = {}, l = 0                         (initial pattern)
 *     J0(k) = {k} (the pattern of I, the paper's usual choice) or the
 *     pattern of column k of A (init_mode 1)
 *   Solve(J); Drop(J); r = A m - e_k; rho = ||r||    (first solve, Eq. 4.3)
 *   while rho > eps and l < l_max                    (loop test)
 *     L = {i in S : |r_i| > band};  Cand = L \ R     (dominant indices, Eq. 3.2)
 *     if Cand empty: stop (r = 0 to working precision)
 *     Rhat = top-c of Cand by (|r_i| desc, i asc) with tie band; R += Rhat
 *     Jhat = cols(A(Rhat,:)) \ J                     (new columns)
 *     l = l + 1; if Jhat empty: continue             (empty Jhat)
 *     J += Jhat; Solve(J); Drop(J); r, rho           (update of m_k, Eq. 4.3)
 *   SPAI selection (select_mode 1) replaces the three selection lines:
 *     L = {i in S : |r_i| > band}                    (Eq. 2.5: rows where r != 0)
 *     N = nonzero columns of A(L,:); Jhat = N \ J     (candidates, Eq. 2.5)
 *     if Jhat empty: stop
 *     rho_j^2 = ||r||^2 - (r^T A e_j)^2 / ||A e_j||^2 (Eq. 2.7, from Eq. 2.6)
 *     take the c candidates with the smallest rho_j, i.e. the largest
 *     s_j = (r^T A e_j)^2 / ||A e_j||^2, by (s_j desc, j asc) with a tie band
 *     of tie_band * ||r||^2 (s_j <= ||r||^2); l = l + 1
 *
 * Readings of points the paper leaves open (each is restated in the design
 * notes of the repository):
 *   - Solve(J): I = rows of A(:,J) (Section 2), B = A(I,J) rows ascending in I,
 *     columns ascending in J, e = e_k(I); Householder QR without pivoting,
 *     v = x + sign(x1)||x|| e1 with sign(0) = +1; m = R^{-1} (Q^T e)(1:p).
 *     The paper updates the previous QR (Section 3); in exact arithmetic the
 *     LS solution is unique, so refactoring gives the same m.
 *   - Drop(J): threshold tau (NONE: no dropping; ADAPTIVE: eps/(p ||A||_1),
 *     Eq. 4.3 with nnz(m_k) = p = |J| before dropping; FIXED: tol/||A||_1).
 *     D = {j : |m_j| <= tau}; if D = J keep the largest |m_j| (lowest j on a
 *     tie); if D is not empty, J = J \ D and Solve(J) once more.  A single drop
 *     pass follows every solve, so the emitted m is the exact LS minimiser on
 *     its emitted pattern.
 *   - The residual lives on S = I u {k} (r(k) = -1 when k is not in I).
 *   - Ties: with v the c-th largest |r_i| of Cand and b = tie_band*||r||_inf,
 *     take every i with |r_i| > v + b, then fill up to c from
 *     {i : v - b <= |r_i| <= v + b} by lowest index; "r_i != 0" means |r_i| > b.
 *   - The choice of dominant indices always excludes R (not only on a
 *     repeat); loops whose Jhat is empty still count toward l_max (Algorithm 1
 *     raises l before it returns to its loop test).
 *   - Rank: if |R_jj| <= q*u*||B||_F the column is flagged RANK and that
 *     component of m is set to zero.
 *   - SPAI: no set of excluded rows (every row with r_i != 0 feeds the
 *     candidates each loop); a loop with no candidate left ends the column
 *     without counting (it could add nothing later either); candidates with
 *     s_j = 0 (no improvement) may still be taken when fewer than c do better.
 *
 * Algorithmic work counters (the method's own work, with the paper's QR
 * update rather than this file's refactoring; Section 3 "update ... as in
 * Grote97/Jia09"):
 *   solve on (q,p) appended to a previous factorisation (q0,p0):
 *     4 (p-p0) sum_{j<p0} (q0-j)  +  sum_{j=p0}^{p-1} (q-j) (2 + 4 (p-j))  +  p^2
 *   a solve after a drop, and the first solve, use p0 = 0 (no previous factor);
 *   residual: 2 nnz(A(:,J)) + 2 |S|.
 *   SPAI selection: 4 nnz(A e_j) + 3 per candidate j per loop (its dot
 *   product with r, its squared norm, Eq. 2.7); bytes 4 nnz(A(i,:)) + 16 per
 *   row of L and 12 nnz(A e_j) + 16 per candidate, each loop.
 *   bytes: 12 nnz(A(:,j)) + 16 once for every column j that ever enters J_k
 *          (a column dropped and later re-entered is not counted again: the
 *          method needs each entry of A(:,j) read once per column k),
 *          4 nnz(A(i,:)) + 16 for every dominant row i, 36 per emitted entry
 *          (12 to emit it, 24 to move it once more into CSR).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { DROP_NONE = 0, DROP_ADAPTIVE = 1, DROP_FIXED = 2 };
enum { SELECT_RSAI = 0, SELECT_SPAI = 1 };
enum { FLAG_CONVERGED = 1, FLAG_RANK = 2, FLAG_NONFINITE = 4 };

typedef struct {
    int64_t n;
    const int64_t *row_ptr; const int32_t *col_idx; const double *val;  /* CSR */
    const int64_t *col_ptr; const int32_t *row_idx; const double *cval; /* CSC */
} omat;

typedef struct {
    int32_t c, l_max, drop_mode, init_mode;  /* init_mode: 0 = pattern of I, 1 = pattern of A */
    double eps, tol, tie_band, norm1;
    int32_t select_mode;                     /* SELECT_RSAI (dominant rows) or SELECT_SPAI */
} oparams;

/* one finished column of M */
typedef struct {
    int32_t p;
    int32_t *J;
    double *m;
    double rho;
    int32_t loops, flags, solves, drops;
    int32_t p_max, q_max; /* largest LS problem met */
    double qr_flops, res_flops, bytes, sel_flops;
} ocol;

typedef struct {
    int64_t ncols;
    ocol *cols;
} oresult;

/* ---------- growable scratch ---------- */
typedef struct {
    int32_t *I; int64_t capI;
    int32_t *S; int64_t capS;
    int32_t *tmp; int64_t capT;
    double *B; int64_t capB;
    double *Bcopy; int64_t capBc;
    double *e; int64_t cape;
    double *r; int64_t capr;
    double *w; int64_t capw;
} ows;

static void *grow(void *p, int64_t *cap, int64_t need, size_t el) {
    if (need <= *cap) return p;
    int64_t nc = *cap ? *cap : 64;
    while (nc < need) nc *= 2;
    p = realloc(p, (size_t)nc * el);
    if (!p) abort();
    *cap = nc;
    return p;
}

static void ows_free(ows *w) {
    free(w->I); free(w->S); free(w->tmp); free(w->B); free(w->Bcopy);
    free(w->e); free(w->r); free(w->w);
    memset(w, 0, sizeof(*w));
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* sort + unique in place, returns new length */
static int64_t sort_unique(int32_t *a, int64_t len) {
    if (len == 0) return 0;
    qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t o = 1;
    for (int64_t i = 1; i < len; ++i)
        if (a[i] != a[o - 1]) a[o++] = a[i];
    return o;
}

/* position of v in sorted a[0..len), or -1 */
static int64_t find(const int32_t *a, int64_t len, int32_t v) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (lo < len && a[lo] == v) ? lo : -1;
}

/* ||A||_1 = max_j sum_i |a_ij| (Eq. 4.3) */
double ro_norm1(int64_t n, const int64_t *col_ptr, const double *cval) {
    double best = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) s += fabs(cval[e]);
        if (s > best) best = s;
    }
    return best;
}

/* I = sorted union of the row indices of A(:,J) (Section 2: nonzero rows). */
static int64_t rows_of(const omat *A, const int32_t *J, int p, ows *w) {
    int64_t tot = 0;
    for (int c = 0; c < p; ++c) tot += A->col_ptr[J[c] + 1] - A->col_ptr[J[c]];
    w->I = grow(w->I, &w->capI, tot + 1, sizeof(int32_t));
    int64_t t = 0;
    for (int c = 0; c < p; ++c)
        for (int64_t e = A->col_ptr[J[c]]; e < A->col_ptr[J[c] + 1]; ++e) w->I[t++] = A->row_idx[e];
    return sort_unique(w->I, t);
}

/* B = A(I,J), dense column-major q x p. */
static void gather(const omat *A, const int32_t *J, int p, const int32_t *I, int64_t q, double *B) {
    memset(B, 0, sizeof(double) * (size_t)(q * p));
    for (int c = 0; c < p; ++c)
        for (int64_t e = A->col_ptr[J[c]]; e < A->col_ptr[J[c] + 1]; ++e)
            B[c * q + find(I, q, A->row_idx[e])] = A->cval[e];
}

/*
 * Householder QR of B (q x p, column-major, in place) applied to the right-hand
 * side e; then back substitution.  After the call B holds R in its upper
 * triangle and the reflectors below it (v_j with its head stored in vhead[j]).
 * Returns 1 if a diagonal of R is negligible (rank flag).
 */
static int householder_solve(double *B, int64_t q, int p, double *e, double *x, double *vhead) {
    double fro = 0.0;
    for (int64_t i = 0; i < q * p; ++i) fro += B[i] * B[i];
    fro = sqrt(fro);
    const double small = (double)q * 2.220446049250313e-16 * fro;
    int rank = 0;
    for (int j = 0; j < p; ++j) {
        double *col = B + (int64_t)j * q;
        double sigma = 0.0;
        for (int64_t i = j; i < q; ++i) sigma += col[i] * col[i];
        double nrm = sqrt(sigma);
        double x0 = col[j];
        double alpha = (x0 >= 0.0) ? -nrm : nrm;  /* sign(0) = +1 */
        double v0 = x0 - alpha;
        double vtv = sigma - x0 * x0 + v0 * v0;
        vhead[j] = v0;
        if (vtv > 0.0) {
            /* H = I - 2 v v^T / v^T v applied to the trailing columns and to e */
            for (int cc = j + 1; cc <= p; ++cc) {
                double *t = (cc < p) ? B + (int64_t)cc * q : e;
                double s = v0 * t[j];
                for (int64_t i = j + 1; i < q; ++i) s += col[i] * t[i];
                double f = 2.0 * s / vtv;
                t[j] -= f * v0;
                for (int64_t i = j + 1; i < q; ++i) t[i] -= f * col[i];
            }
        }
        col[j] = alpha; /* R_jj */
        if (fabs(alpha) <= small) rank = 1;
    }
    for (int i = p - 1; i >= 0; --i) {
        double s = e[i];
        for (int cc = i + 1; cc < p; ++cc) s -= B[(int64_t)cc * q + i] * x[cc];
        double d = B[(int64_t)i * q + i];
        x[i] = (fabs(d) <= small) ? 0.0 : s / d;
    }
    return rank;
}

/* Solve the reduced LS problem (Eq. 2.3) on pattern J; returns q. */
static int64_t ls_solve(const omat *A, int64_t k, const int32_t *J, int p, ows *w, double *x, int *rank) {
    int64_t q = rows_of(A, J, p, w);
    w->B = grow(w->B, &w->capB, q * p + 1, sizeof(double));
    w->e = grow(w->e, &w->cape, q + 1, sizeof(double));
    w->w = grow(w->w, &w->capw, p + 1, sizeof(double));
    gather(A, J, p, w->I, q, w->B);
    memset(w->e, 0, sizeof(double) * (size_t)q);
    int64_t pk = find(w->I, q, (int32_t)k);
    if (pk >= 0) w->e[pk] = 1.0;
    if (q < p) { /* more unknowns than equations: cannot happen for nonsingular A */
        for (int c = 0; c < p; ++c) x[c] = 0.0;
        *rank = 1;
        return q;
    }
    *rank |= householder_solve(w->B, q, p, w->e, x, w->w);
    return q;
}

/* r = A(:,J) m - e_k on S = I u {k} (Eq. 2.4); returns |S|, rho = ||r||. */
static int64_t residual(const omat *A, int64_t k, const int32_t *J, int p, const double *m,
                        ows *w, double *rho, double *nnzJ) {
    int64_t q = rows_of(A, J, p, w);
    w->S = grow(w->S, &w->capS, q + 1, sizeof(int32_t));
    memcpy(w->S, w->I, sizeof(int32_t) * (size_t)q);
    int64_t s = q;
    if (find(w->S, s, (int32_t)k) < 0) { w->S[s++] = (int32_t)k; s = sort_unique(w->S, s); }
    w->r = grow(w->r, &w->capr, s + 1, sizeof(double));
    memset(w->r, 0, sizeof(double) * (size_t)s);
    double cnt = 0.0;
    for (int c = 0; c < p; ++c)
        for (int64_t e = A->col_ptr[J[c]]; e < A->col_ptr[J[c] + 1]; ++e) {
            w->r[find(w->S, s, A->row_idx[e])] += A->cval[e] * m[c];
            cnt += 1.0;
        }
    w->r[find(w->S, s, (int32_t)k)] -= 1.0;
    double ss = 0.0;
    for (int64_t i = 0; i < s; ++i) ss += w->r[i] * w->r[i];
    *rho = sqrt(ss);
    *nnzJ = cnt;
    return s;
}

static double solve_flops(int64_t q0, int p0, int64_t q, int p) {
    double f = 0.0;
    for (int j = 0; j < p0; ++j) f += 4.0 * (double)(p - p0) * (double)(q0 - j);
    for (int j = p0; j < p; ++j) f += (double)(q - j) * (2.0 + 4.0 * (double)(p - j));
    return f + (double)p * (double)p;
}

typedef struct { double a; int32_t i; } keyed;

static int cmp_dom(const void *x, const void *y) {
    const keyed *u = x, *v = y;
    if (u->a > v->a) return -1;
    if (u->a < v->a) return 1;
    return (u->i > v->i) - (u->i < v->i);
}

static int cmp_idx(const void *x, const void *y) {
    const keyed *u = x, *v = y;
    return (u->i > v->i) - (u->i < v->i);
}

/* One column of RSAI(tol): Algorithm 1 with the dropping of Eq. 4.3. */
static void rsai_column(const omat *A, const oparams *P, int64_t k, ocol *out, ows *w) {
    int64_t n = A->n;
    int64_t capJ = 16, capR = 16;
    int32_t *J = malloc(sizeof(int32_t) * capJ);
    int32_t *Rset = malloc(sizeof(int32_t) * capR);
    int64_t capSeen = 16;
    int64_t nSeen = 0;
    int32_t *seen = malloc(sizeof(int32_t) * capSeen); /* every column that has entered J, sorted */
    double *m = malloc(sizeof(double) * capJ);
    int p = 1, nR = 0, l = 0, rank = 0, solves = 0, drops = 0;
    int64_t q = 0, q0 = 0;
    int p0 = 0, pmax = 1;
    int64_t qmax = 0;
    double qr_flops = 0.0, res_flops = 0.0, bytes = 0.0, rho = 0.0, nnzJ = 0.0, sel_flops = 0.0;
    J[0] = (int32_t)k;
    if (P->init_mode == 1) {
        /* Algorithm 1 started from the initial pattern of A: J = rows of A(:,k) */
        int64_t len = A->col_ptr[k + 1] - A->col_ptr[k];
        if (len > 0) {
            J = grow(J, &capJ, len, sizeof(int32_t));
            m = realloc(m, sizeof(double) * (size_t)capJ);
            for (int64_t e = 0; e < len; ++e) J[e] = A->row_idx[A->col_ptr[k] + e];
            p = (int)len;
            pmax = p;
        }
    }

    /* bytes of a column of A the first time it enters J */
#define NOTE_COLUMN(j)                                                              \
    do {                                                                            \
        int32_t jj_ = (j);                                                          \
        if (find(seen, nSeen, jj_) < 0) {                                           \
            seen = grow(seen, &capSeen, nSeen + 1, sizeof(int32_t));                \
            seen[nSeen++] = jj_;                                                    \
            qsort(seen, (size_t)nSeen, sizeof(int32_t), cmp_i32);                   \
            bytes += 12.0 * (double)(A->col_ptr[jj_ + 1] - A->col_ptr[jj_]) + 16.0; \
        }                                                                           \
    } while (0)

    /* Solve on J, counting work; appended = 1 if J extends the last solved J. */
#define SOLVE(appended)                                                              \
    do {                                                                             \
        rank = 0;                                                                    \
        q = ls_solve(A, k, J, p, w, m, &rank);                                       \
        qr_flops += (appended) ? solve_flops(q0, p0, q, p) : solve_flops(0, 0, q, p); \
        q0 = q; p0 = p; ++solves;                                                    \
        if (p > pmax) pmax = p;                                                      \
        if (q > qmax) qmax = q;                                                      \
    } while (0)

    /* Eq. 4.3 drop pass followed by one re-solve. */
#define DROP()                                                                        \
    do {                                                                              \
        if (P->drop_mode != DROP_NONE) {                                              \
            double tau = (P->drop_mode == DROP_ADAPTIVE) ? P->eps / ((double)p * P->norm1) \
                                                         : P->tol / P->norm1;          \
            int keep = 0, best = 0;                                                   \
            for (int c = 0; c < p; ++c) {                                             \
                if (fabs(m[c]) > tau) ++keep;                                         \
                if (fabs(m[c]) > fabs(m[best])) best = c;                             \
            }                                                                         \
            if (keep < p) {                                                           \
                int o = 0;                                                            \
                if (keep == 0) { J[0] = J[best]; o = 1; }                             \
                else for (int c = 0; c < p; ++c) if (fabs(m[c]) > tau) J[o++] = J[c]; \
                if (o < p) { p = o; ++drops; SOLVE(0); }                              \
            }                                                                         \
        }                                                                             \
    } while (0)

    for (int c = 0; c < p; ++c) NOTE_COLUMN(J[c]);
    SOLVE(0);
    DROP();
    int64_t s = residual(A, k, J, p, m, w, &rho, &nnzJ);
    res_flops += 2.0 * nnzJ + 2.0 * (double)s;

    while (rho > P->eps && l < P->l_max) {
        if (P->select_mode == SELECT_SPAI) {
            /* L = rows of S where r != 0 (beyond the band), Eq. 2.5 */
            double rinf = 0.0, rr = 0.0;
            for (int64_t i = 0; i < s; ++i) {
                if (fabs(w->r[i]) > rinf) rinf = fabs(w->r[i]);
                rr += w->r[i] * w->r[i];
            }
            double band = P->tie_band * rinf;
            int64_t tot = 0, nL = 0;
            for (int64_t i = 0; i < s; ++i)
                if (fabs(w->r[i]) > band) {
                    int32_t row = w->S[i];
                    tot += A->row_ptr[row + 1] - A->row_ptr[row];
                    bytes += 4.0 * (double)(A->row_ptr[row + 1] - A->row_ptr[row]) + 16.0;
                    ++nL;
                }
            if (nL == 0) break;
            /* N = nonzero columns of A(L,:); Jhat = N \ J */
            w->tmp = grow(w->tmp, &w->capT, tot + 1, sizeof(int32_t));
            int64_t nj = 0;
            for (int64_t i = 0; i < s; ++i)
                if (fabs(w->r[i]) > band) {
                    int32_t row = w->S[i];
                    for (int64_t e = A->row_ptr[row]; e < A->row_ptr[row + 1]; ++e)
                        if (find(J, p, A->col_idx[e]) < 0) w->tmp[nj++] = A->col_idx[e];
                }
            nj = sort_unique(w->tmp, nj);
            if (nj == 0) break; /* no candidate: nothing can be added */
            /* s_j = (r^T A e_j)^2 / ||A e_j||^2 (Eq. 2.7: rho_j^2 = ||r||^2 - s_j) */
            keyed *cand = malloc(sizeof(keyed) * (size_t)nj);
            for (int64_t t = 0; t < nj; ++t) {
                int32_t j = w->tmp[t];
                double dot = 0.0, nrm = 0.0;
                for (int64_t e = A->col_ptr[j]; e < A->col_ptr[j + 1]; ++e) {
                    int64_t pos = find(w->S, s, A->row_idx[e]);
                    if (pos >= 0) dot += w->r[pos] * A->cval[e];
                    nrm += A->cval[e] * A->cval[e];
                }
                double len = (double)(A->col_ptr[j + 1] - A->col_ptr[j]);
                sel_flops += 4.0 * len + 3.0;
                bytes += 12.0 * len + 16.0;
                cand[t].a = (nrm > 0.0) ? dot * dot / nrm : 0.0;
                cand[t].i = j;
            }
            /* the c largest s_j, ties by lowest j within tie_band * ||r||^2 */
            int c = P->c < 64 ? P->c : 64;
            int32_t add[64];
            int na = 0;
            if (nj <= c) {
                for (int64_t t = 0; t < nj; ++t) add[na++] = cand[t].i;
            } else {
                double sband = P->tie_band * rr;
                qsort(cand, (size_t)nj, sizeof(keyed), cmp_dom);
                double v = cand[c - 1].a;
                for (int64_t t = 0; t < nj; ++t) if (cand[t].a > v + sband) add[na++] = cand[t].i;
                keyed *tie = malloc(sizeof(keyed) * (size_t)nj);
                int64_t nt = 0;
                for (int64_t t = 0; t < nj; ++t)
                    if (cand[t].a >= v - sband && cand[t].a <= v + sband) tie[nt++] = cand[t];
                qsort(tie, (size_t)nt, sizeof(keyed), cmp_idx);
                for (int64_t t = 0; t < nt && na < c; ++t) add[na++] = tie[t].i;
                free(tie);
            }
            free(cand);
            ++l;
            J = grow(J, &capJ, p + na, sizeof(int32_t));
            m = realloc(m, sizeof(double) * (size_t)capJ);
            for (int t = 0; t < na; ++t) { J[p + t] = add[t]; NOTE_COLUMN(add[t]); }
            p += na;
            qsort(J, (size_t)p, sizeof(int32_t), cmp_i32);
            SOLVE(1);
            DROP();
            s = residual(A, k, J, p, m, w, &rho, &nnzJ);
            res_flops += 2.0 * nnzJ + 2.0 * (double)s;
            continue;
        }
        /* dominant rows among L \ R (Algorithm 1, Eq. 3.2) */
        double rinf = 0.0;
        for (int64_t i = 0; i < s; ++i) if (fabs(w->r[i]) > rinf) rinf = fabs(w->r[i]);
        double band = P->tie_band * rinf;
        keyed *cand = malloc(sizeof(keyed) * (size_t)(s + 1));
        int64_t nc = 0;
        for (int64_t i = 0; i < s; ++i) {
            double a = fabs(w->r[i]);
            if (a > band && find(Rset, nR, w->S[i]) < 0) { cand[nc].a = a; cand[nc].i = w->S[i]; ++nc; }
        }
        if (nc == 0) { free(cand); break; }
        int32_t Rhat[64];
        int nh = 0;
        int c = P->c < 64 ? P->c : 64;
        if (nc <= c) {
            for (int64_t t = 0; t < nc; ++t) Rhat[nh++] = cand[t].i;
        } else {
            qsort(cand, (size_t)nc, sizeof(keyed), cmp_dom);
            double v = cand[c - 1].a;
            double hi = v + band, lo = v - band;
            /* above the band: certainly among the top c; inside [lo, hi]: a tie */
            for (int64_t t = 0; t < nc; ++t) if (cand[t].a > hi) Rhat[nh++] = cand[t].i;
            int64_t nt = 0;
            keyed *tie = malloc(sizeof(keyed) * (size_t)nc);
            for (int64_t t = 0; t < nc; ++t)
                if (cand[t].a >= lo && cand[t].a <= hi) tie[nt++] = cand[t];
            qsort(tie, (size_t)nt, sizeof(keyed), cmp_idx);
            for (int64_t t = 0; t < nt && nh < c; ++t) Rhat[nh++] = tie[t].i;
            free(tie);
        }
        free(cand);
        /* R = R u Rhat (kept sorted) */
        for (int t = 0; t < nh; ++t) {
            Rset = grow(Rset, &capR, nR + 1, sizeof(int32_t));
            Rset[nR++] = Rhat[t];
            bytes += 4.0 * (double)(A->row_ptr[Rhat[t] + 1] - A->row_ptr[Rhat[t]]) + 16.0;
        }
        nR = (int)sort_unique(Rset, nR);
        /* new columns: Jhat = cols(A(Rhat,:)) \ J */
        int64_t tot = 0;
        for (int t = 0; t < nh; ++t) tot += A->row_ptr[Rhat[t] + 1] - A->row_ptr[Rhat[t]];
        w->tmp = grow(w->tmp, &w->capT, tot + 1, sizeof(int32_t));
        int64_t nj = 0;
        for (int t = 0; t < nh; ++t)
            for (int64_t e = A->row_ptr[Rhat[t]]; e < A->row_ptr[Rhat[t] + 1]; ++e) {
                int32_t j = A->col_idx[e];
                if (find(J, p, j) < 0) w->tmp[nj++] = j;
            }
        nj = sort_unique(w->tmp, nj);
        /* l = l + 1; an empty Jhat goes back to the loop test */
        ++l;
        if (nj == 0) continue;
        /* J = J u Jhat (sorted), update the LS solution, drop, residual */
        J = grow(J, &capJ, p + nj, sizeof(int32_t));
        m = realloc(m, sizeof(double) * (size_t)capJ);
        for (int64_t t = 0; t < nj; ++t) { J[p + t] = w->tmp[t]; NOTE_COLUMN(w->tmp[t]); }
        p += (int)nj;
        qsort(J, (size_t)p, sizeof(int32_t), cmp_i32);
        SOLVE(1);
        DROP();
        s = residual(A, k, J, p, m, w, &rho, &nnzJ);
        res_flops += 2.0 * nnzJ + 2.0 * (double)s;
    }
#undef NOTE_COLUMN
#undef SOLVE
#undef DROP
    int finite = isfinite(rho);
    for (int c = 0; c < p; ++c) finite &= isfinite(m[c]);
    bytes += 36.0 * (double)p;
    out->p = p;
    out->J = J;
    out->m = m;
    out->rho = rho;
    out->loops = l;
    out->flags = (rho <= P->eps ? FLAG_CONVERGED : 0) | (rank ? FLAG_RANK : 0) | (finite ? 0 : FLAG_NONFINITE);
    out->solves = solves;
    out->drops = drops;
    out->p_max = pmax;
    out->q_max = (int32_t)qmax;
    out->qr_flops = qr_flops;
    out->res_flops = res_flops;
    out->bytes = bytes;
    out->sel_flops = sel_flops;
    free(Rset);
    free(seen);
    (void)n;
}

/*
 * Build the columns cols[0..ncols) of M (all n columns if cols is NULL).
 * Returns an opaque result; read it with ro_nnz / ro_export, free with ro_free.
 */
void *ro_build(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
               const int64_t *col_ptr, const int32_t *row_idx, const double *cval,
               int32_t c, int32_t l_max, double eps, int32_t drop_mode, double tol, double tie_band,
               const int64_t *cols, int64_t ncols, int32_t nthreads, int32_t init_mode, int32_t select_mode) {
    omat A = {n, row_ptr, col_idx, val, col_ptr, row_idx, cval};
    oparams P = {c, l_max, drop_mode, init_mode, eps, tol, tie_band, ro_norm1(n, col_ptr, cval), select_mode};
    oresult *res = calloc(1, sizeof(oresult));
    if (!cols) ncols = n;
    res->ncols = ncols;
    res->cols = calloc((size_t)(ncols ? ncols : 1), sizeof(ocol));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        ows w;
        memset(&w, 0, sizeof(w));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t t = 0; t < ncols; ++t)
            rsai_column(&A, &P, cols ? cols[t] : t, &res->cols[t], &w);
        ows_free(&w);
    }
    (void)nthreads;
    return res;
}

int64_t ro_nnz(const void *h) {
    const oresult *r = h;
    int64_t s = 0;
    for (int64_t t = 0; t < r->ncols; ++t) s += r->cols[t].p;
    return s;
}

/* Column-wise (CSC-like) export; any output pointer may be NULL. */
void ro_export(const void *h, int64_t *colptr, int32_t *rows, double *vals, double *rho,
               int32_t *loops, int32_t *flags, double *counters /* ncols x 9 */) {
    const oresult *r = h;
    int64_t off = 0;
    for (int64_t t = 0; t < r->ncols; ++t) {
        const ocol *c = &r->cols[t];
        if (colptr) colptr[t] = off;
        for (int i = 0; i < c->p; ++i) {
            if (rows) rows[off + i] = c->J[i];
            if (vals) vals[off + i] = c->m[i];
        }
        off += c->p;
        if (rho) rho[t] = c->rho;
        if (loops) loops[t] = c->loops;
        if (flags) flags[t] = c->flags;
        if (counters) {
            double *o = counters + 9 * t;
            o[0] = c->qr_flops; o[1] = c->res_flops; o[2] = c->bytes; o[3] = c->solves;
            o[4] = c->drops; o[5] = c->p_max; o[6] = c->q_max; o[7] = c->p; o[8] = c->sel_flops;
        }
    }
    if (colptr) colptr[r->ncols] = off;
}

void ro_free(void *h) {
    oresult *r = h;
    if (!r) return;
    for (int64_t t = 0; t < r->ncols; ++t) { free(r->cols[t].J); free(r->cols[t].m); }
    free(r->cols);
    free(r);
}

/*
 * Frozen-pattern re-solve: for each column k with pattern J_k (CSC-like
 * Mcolptr/Mrows, rows ascending), m_k = argmin ||A(:,J_k) x - e_k|| (Eq. 2.3)
 * and rho2[k] = ||r_k||^2 (Eq. 2.4).  No dropping, no pattern change.
 */
void ro_refit(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
              const int64_t *col_ptr, const int32_t *row_idx, const double *cval,
              const int64_t *Mcolptr, const int32_t *Mrows, double *Mval, double *rho2,
              int32_t nthreads) {
    omat A = {n, row_ptr, col_idx, val, col_ptr, row_idx, cval};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        ows w;
        memset(&w, 0, sizeof(w));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t k = 0; k < n; ++k) {
            int p = (int)(Mcolptr[k + 1] - Mcolptr[k]);
            const int32_t *J = Mrows + Mcolptr[k];
            double *x = Mval + Mcolptr[k];
            int rank = 0;
            double rho, cnt;
            ls_solve(&A, k, J, p, &w, x, &rank);
            residual(&A, k, J, p, x, &w, &rho, &cnt);
            rho2[k] = rho * rho;
        }
        ows_free(&w);
    }
    (void)nthreads;
}

/*
 * Adjoint of the frozen-pattern solve.  For every column k with B = A(I_k,J_k),
 * x = m_k(J_k), r = B x - e_k(I_k), and a loss L(M, rho^2) with
 * gm = dL/dm_k(J_k) and gr = dL/d(rho_k^2):
 *   from B^T B x = B^T e:   dx = (B^T B)^{-1} (-dB^T r - B^T dB x)
 *   from rho^2 = ||r||^2 and B^T r = 0:   d rho^2 = 2 r^T dB x
 * so, with z = (B^T B)^{-1} gm = R^{-1} R^{-T} gm,
 *   dL/dB = -r z^T - (B z) x^T + 2 gr r x^T,
 * and dL/dA(i,j) sums that over all columns k whose I_k x J_k holds (i,j).
 * grad_val is in CSR order and is overwritten.  Serial over k, so the sum order
 * is fixed.
 */
void ro_backward(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                 const int64_t *col_ptr, const int32_t *row_idx, const double *cval,
                 const int64_t *Mcolptr, const int32_t *Mrows, const double *grad_m,
                 const double *grad_rho2, double *grad_val) {
    omat A = {n, row_ptr, col_idx, val, col_ptr, row_idx, cval};
    ows w;
    memset(&w, 0, sizeof(w));
    memset(grad_val, 0, sizeof(double) * (size_t)row_ptr[n]);
    double *x = NULL, *z = NULL, *y = NULL, *rr = NULL, *bz = NULL;
    int64_t capx = 0, capz = 0, capy = 0, caprr = 0, capbz = 0;
    for (int64_t k = 0; k < n; ++k) {
        int p = (int)(Mcolptr[k + 1] - Mcolptr[k]);
        const int32_t *J = Mrows + Mcolptr[k];
        const double *gm = grad_m + Mcolptr[k];
        double gr = grad_rho2 ? grad_rho2[k] : 0.0;
        x = grow(x, &capx, p + 1, sizeof(double));
        z = grow(z, &capz, p + 1, sizeof(double));
        y = grow(y, &capy, p + 1, sizeof(double));
        int rank = 0;
        int64_t q = ls_solve(&A, k, J, p, &w, x, &rank);
        /* w.B now holds R (upper triangle); rebuild B itself for r and B z */
        w.Bcopy = grow(w.Bcopy, &w.capBc, q * p + 1, sizeof(double));
        gather(&A, J, p, w.I, q, w.Bcopy);
        const double *R = w.B;
        /* R^T y = gm (forward), R z = y (backward) */
        for (int i = 0; i < p; ++i) {
            double s = gm[i];
            for (int cc = 0; cc < i; ++cc) s -= R[(int64_t)i * q + cc] * y[cc];
            y[i] = s / R[(int64_t)i * q + i];
        }
        for (int i = p - 1; i >= 0; --i) {
            double s = y[i];
            for (int cc = i + 1; cc < p; ++cc) s -= R[(int64_t)cc * q + i] * z[cc];
            z[i] = s / R[(int64_t)i * q + i];
        }
        rr = grow(rr, &caprr, q + 1, sizeof(double));
        bz = grow(bz, &capbz, q + 1, sizeof(double));
        int64_t pk = find(w.I, q, (int32_t)k);
        for (int64_t i = 0; i < q; ++i) {
            double s = (i == pk) ? -1.0 : 0.0, t = 0.0;
            for (int cc = 0; cc < p; ++cc) {
                s += w.Bcopy[(int64_t)cc * q + i] * x[cc];
                t += w.Bcopy[(int64_t)cc * q + i] * z[cc];
            }
            rr[i] = s;
            bz[i] = t;
        }
        for (int cc = 0; cc < p; ++cc) {
            int32_t j = J[cc];
            for (int64_t e = A.col_ptr[j]; e < A.col_ptr[j + 1]; ++e) {
                int32_t i = A.row_idx[e];
                int64_t pi = find(w.I, q, i);
                double g = -rr[pi] * z[cc] - bz[pi] * x[cc] + 2.0 * gr * rr[pi] * x[cc];
                /* CSR position of (i, j) */
                int64_t lo = A.row_ptr[i], len = A.row_ptr[i + 1] - lo;
                int64_t off = find(A.col_idx + lo, len, j);
                grad_val[lo + off] += g;
            }
        }
    }
    free(x); free(z); free(y); free(rr); free(bz);
    ows_free(&w);
}
