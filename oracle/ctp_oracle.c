/*
 * ctp_oracle.c -- plain, slow CPU FP64 oracle for compressed threshold pivoting
 * (Hogg & Scott, "Compressed threshold pivoting for sparse symmetric indefinite
 * systems", arXiv 1305.2353).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or constant generator with
 * the CUDA library, and it never calls into it.
 *
 * Style: single thread, natural loop orders, no blocking, compiled with
 * -ffp-contract=off so that every multiply and add is rounded separately --
 * except the trailing update of Listing 1's working matrix, where each
 * a(i,k) - l(i) a(k,q) (or + for the worst-case rows) is one explicit fma()
 * (reading Q18 below).
 * Columns and A11 rows are moved physically, exactly as the paper's listing
 * describes ("permute m to position nelim+1"), with a stable shift.
 *
 * Data convention for a supernode (Section 1, eq. (1.1)): A is n x p,
 * column-major with leading dimension lda >= n; rows 0..p-1 are A11 (only the
 * lower triangle is read), rows p..n-1 are A21.
 *
 * Readings of the paper that the listing leaves open (they are listed, with
 * their justification, in the design notes):
 *   Q1  first sweep starts with the second column as candidate; a rejected
 *       candidate stays in place and m moves on; when m passes the last
 *       column a new sweep starts at the first uneliminated column if the
 *       previous sweep accepted anything, otherwise the factorization stops.
 *   Q2  accepted pivots move to the front by a stable shift; the next
 *       candidate is the column that followed m.
 *   Q3  test_2x2 scales by max(|a_tt|, |a_tm|, |a_mm|).
 *   Q4  the 2x2 candidate is rejected iff |detpiv| <= max(small, |detpiv0|/2,
 *       |detpiv1|/2).
 *   Q5  growth test of eq. (2.2): |D^-1| (maxt, maxm)^T <= (1/u, 1/u)^T.
 *   Q7  zero-pivot test scans every uneliminated entry of column m.
 *   Q8  t is the lowest-index maximiser; no 2x2 attempt when m is the first
 *       uneliminated column.
 *   Q9  column maxima run over all uneliminated A11 rows and all outer rows
 *       (A21 rows for TPP, C rows for compressed pivoting), excluding t, m.
 *   Q10 strict update of C (eq. (4.3), Lemma 5.1, proof of Theorem 5.2):
 *       c(j,k) += chat(j,q) |a(k,q)|, chat = c |D_q^-1|.
 *   Q11 relaxed: ties go to the lowest row; columns left after every A21 row
 *       is flagged get a zero row of C.
 *   Q13 Solve is L21 = (A21 P^T)(D11 L11^T)^-1; rows of A21 never move.
 *   Q21 single-row compression (Section 4.1, closing remark): eq. (4.1) with
 *       the one set J = all rows of A21, so C is one row of column maxima,
 *       updated by the worst-case rule eq. (4.3).
 *   Q18 IEEE FP64, round to nearest even.  The paper fixes no rounding order.
 *       The multipliers l(i) = a(i,q)/d (and [a(i,t) a(i,m)] D^-1) are rounded
 *       per operation; each update a(i,k) -= l(i) a(k,q) of the working matrix
 *       (A11 lower triangle, mirrored, and the outer rows) rounds once, as a
 *       fused multiply-add, the 2x2 terms in the order t, then m.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* pivoting methods */
#define ORC_STRICT 0
#define ORC_RELAXED 1
#define ORC_TPP 2
#define ORC_RESTRICTED 3
#define ORC_SINGLE_ROW 4

/* per-position pivot kinds */
#define PIV_1X1 1
#define PIV_2X2_FIRST 2
#define PIV_2X2_SECOND 0
#define PIV_ZERO (-1)
#define PIV_DELAYED 3

/* update rule for outer rows */
#define UPD_NORMAL 0 /* eq. (4.2): signed update, as for rows of A */
#define UPD_ABS 1    /* eq. (4.3): worst-case update of the strict C */

/* decision-log kinds */
#define LOG_ZERO 0     /* lhs = column max, rhs = small; zero pivot iff lhs < rhs  */
#define LOG_2X2_MAX 1  /* lhs = max |D entry|, rhs = small; reject iff lhs < rhs  */
#define LOG_2X2_DET 2  /* lhs = |detpiv|, rhs = max(small,|d0|/2,|d1|/2); reject iff lhs <= rhs */
#define LOG_2X2_TINY 3 /* lhs = max(maxm,maxt), rhs = small; accept iff lhs < rhs */
#define LOG_2X2_GROW 4 /* lhs = max of |D^-1|(maxt,maxm), rhs = 1/u; accept iff lhs <= rhs */
#define LOG_1X1 5      /* lhs = |a_mm|, rhs = u*maxm; accept iff lhs >= rhs */

typedef struct {
    int32_t kind;
    int32_t m, t; /* original column indices (t = -1 when unused) */
    int32_t outcome;
    double lhs, rhs;
} orc_log_entry;

typedef struct {
    int64_t tests_1x1, tests_2x2, accepted_1x1, accepted_2x2, zero_pivots, sweeps;
    /* operation counters following the counting rules of Appendix A */
    int64_t ops_colmax, ops_test, ops_apply, ops_update;
} orc_stats;

typedef struct {
    int p;        /* columns; rows 0..p-1 of w hold A11 in full symmetric form */
    int rt;       /* outer rows p..p+rt-1: tested and updated with mode `tmode` */
    int rs;       /* shadow rows p+rt..p+rt+rs-1: updated normally, never tested */
    int tmode;    /* UPD_NORMAL or UPD_ABS for the tested outer rows */
    int64_t ldw;
    double *w;
    int *perm;    /* perm[pos] = original column */
    int *piv;
    double *D;    /* D[2k] = D(k,k), D[2k+1] = D(k+1,k) for the first of a 2x2 */
    double u, small;
    orc_log_entry *log;
    int log_cap, log_len;
    orc_stats *st;
} work_t;

#define W(i, j) (wk->w[(int64_t)(j) * wk->ldw + (i)])

static void log_push(work_t *wk, int kind, int m, int t, double lhs, double rhs, int outcome) {
    if (wk->log && wk->log_len < wk->log_cap) {
        orc_log_entry *e = &wk->log[wk->log_len];
        e->kind = kind;
        e->m = m;
        e->t = t;
        e->lhs = lhs;
        e->rhs = rhs;
        e->outcome = outcome;
    }
    wk->log_len++;
}

/* Stable move of column `from` (and, for A11, row `from`) to position `to`
 * (to <= from); positions to..from-1 shift right by one. */
static void move_to(work_t *wk, int from, int to) {
    int nrow = wk->p + wk->rt + wk->rs;
    if (from == to) return;
    for (int i = 0; i < nrow; i++) {
        double x = W(i, from);
        for (int c = from; c > to; c--) W(i, c) = W(i, c - 1);
        W(i, to) = x;
    }
    for (int c = 0; c < wk->p; c++) {
        double x = W(from, c);
        for (int r = from; r > to; r--) W(r, c) = W(r - 1, c);
        W(to, c) = x;
    }
    int pm = wk->perm[from];
    for (int c = from; c > to; c--) wk->perm[c] = wk->perm[c - 1];
    wk->perm[to] = pm;
}

/* max |a(i,col)| over uneliminated A11 rows i >= nelim (positions), skipping
 * positions x1 and x2 (-1 = none), and over the tested outer rows. */
static double col_max(work_t *wk, int nelim, int col, int x1, int x2) {
    double mx = 0.0;
    for (int i = nelim; i < wk->p; i++) {
        if (i == x1 || i == x2) continue;
        double v = fabs(W(i, col));
        if (v > mx) mx = v;
    }
    for (int i = wk->p; i < wk->p + wk->rt; i++) {
        double v = fabs(W(i, col));
        if (v > mx) mx = v;
    }
    return mx;
}

/* test_2x2 of Listing 1 with readings Q3, Q4, Q5.  a_tt, a_tm, a_mm are the
 * entries of the candidate block; returns 1 to accept. */
static int test_2x2(work_t *wk, int m_orig, int t_orig, double a_tt, double a_tm, double a_mm,
                    double maxt, double maxm) {
    double amax = fmax(fabs(a_tt), fmax(fabs(a_tm), fabs(a_mm)));
    if (amax < wk->small) {
        log_push(wk, LOG_2X2_MAX, m_orig, t_orig, amax, wk->small, 0);
        return 0;
    }
    double detscale = 1.0 / amax;
    double detpiv1 = (a_tm * detscale) * a_tm;
    double detpiv0 = a_mm * detscale * a_tt;
    double detpiv = detpiv0 - detpiv1;
    double guard = fmax(wk->small, fmax(fabs(detpiv0) / 2, fabs(detpiv1) / 2));
    if (fabs(detpiv) <= guard) {
        log_push(wk, LOG_2X2_DET, m_orig, t_orig, fabs(detpiv), guard, 0);
        return 0;
    }
    log_push(wk, LOG_2X2_DET, m_orig, t_orig, fabs(detpiv), guard, 1);
    double mxx = fmax(maxm, maxt);
    if (mxx < wk->small) {
        log_push(wk, LOG_2X2_TINY, m_orig, t_orig, mxx, wk->small, 1);
        return 1;
    }
    /* D = [[a_tt, a_tm], [a_tm, a_mm]] in (t, m) order,
       |D^-1| = (detscale/|detpiv|) [[|a_mm|, |a_tm|], [|a_tm|, |a_tt|]]   (eq. (2.2)) */
    double gt = (fabs(a_mm) * maxt + fabs(a_tm) * maxm) * detscale / fabs(detpiv);
    double gm = (fabs(a_tm) * maxt + fabs(a_tt) * maxm) * detscale / fabs(detpiv);
    double g = fmax(gt, gm);
    int ok = (gt <= 1.0 / wk->u) && (gm <= 1.0 / wk->u);
    log_push(wk, LOG_2X2_GROW, m_orig, t_orig, g, 1.0 / wk->u, ok);
    return ok;
}

/* Eliminate a 1x1 pivot at position q (already moved there). */
static void pivot_1x1(work_t *wk, int q, double *lcol) {
    int p = wk->p, nrow = p + wk->rt + wk->rs;
    double d = W(q, q);
    wk->piv[q] = PIV_1X1;
    wk->D[2 * q] = d;
    wk->D[2 * q + 1] = 0.0;
    /* multipliers l(i,q) = a(i,q)/d for every row below the pivot (normal rows),
       chat(j,q) = c(j,q)/|d| for abs rows (eq. (4.3)) */
    for (int i = q + 1; i < nrow; i++) {
        int is_abs = (wk->tmode == UPD_ABS) && i >= p && i < p + wk->rt;
        lcol[i] = is_abs ? W(i, q) / fabs(d) : W(i, q) / d;
    }
    /* trailing update (right-looking) */
    for (int k = q + 1; k < p; k++) {
        double akq = W(k, q);
        for (int i = k; i < p; i++) W(i, k) = fma(-lcol[i], akq, W(i, k)); /* A11 lower incl. diagonal */
        for (int i = k + 1; i < p; i++) W(k, i) = W(i, k);                 /* keep symmetric copy */
        for (int i = p; i < nrow; i++) {
            int is_abs = (wk->tmode == UPD_ABS) && i < p + wk->rt;
            if (is_abs)
                W(i, k) = fma(lcol[i], fabs(akq), W(i, k));
            else
                W(i, k) = fma(-lcol[i], akq, W(i, k));
        }
        if (wk->st) wk->st->ops_update += (p - k) + (nrow - p);
    }
    for (int i = q + 1; i < nrow; i++) W(i, q) = lcol[i];
    if (wk->st) wk->st->ops_apply += nrow - q - 1;
}

/* Eliminate a 2x2 pivot at positions q, q+1 (t then m, already moved). */
static void pivot_2x2(work_t *wk, int q, double *l0, double *l1) {
    int p = wk->p, nrow = p + wk->rt + wk->rs;
    double a = W(q, q), b = W(q + 1, q), c = W(q + 1, q + 1);
    double amax = fmax(fabs(a), fmax(fabs(b), fabs(c)));
    double detscale = 1.0 / amax;
    double detpiv = c * detscale * a - (b * detscale) * b;
    /* D^-1 = (detscale/detpiv) [[c, -b], [-b, a]] */
    double i11 = (c * detscale) / detpiv;
    double i21 = (-b * detscale) / detpiv;
    double i22 = (a * detscale) / detpiv;
    wk->piv[q] = PIV_2X2_FIRST;
    wk->piv[q + 1] = PIV_2X2_SECOND;
    wk->D[2 * q] = a;
    wk->D[2 * q + 1] = b;
    wk->D[2 * q + 2] = c;
    wk->D[2 * q + 3] = 0.0;
    for (int i = q + 2; i < nrow; i++) {
        double x = W(i, q), y = W(i, q + 1);
        int is_abs = (wk->tmode == UPD_ABS) && i >= p && i < p + wk->rt;
        if (is_abs) {
            l0[i] = x * fabs(i11) + y * fabs(i21);
            l1[i] = x * fabs(i21) + y * fabs(i22);
        } else {
            l0[i] = x * i11 + y * i21;
            l1[i] = x * i21 + y * i22;
        }
    }
    for (int k = q + 2; k < p; k++) {
        double akq = W(k, q), akq1 = W(k, q + 1);
        for (int i = k; i < p; i++) W(i, k) = fma(-l1[i], akq1, fma(-l0[i], akq, W(i, k)));
        for (int i = k + 1; i < p; i++) W(k, i) = W(i, k);
        for (int i = p; i < nrow; i++) {
            int is_abs = (wk->tmode == UPD_ABS) && i < p + wk->rt;
            if (is_abs)
                W(i, k) = fma(l1[i], fabs(akq1), fma(l0[i], fabs(akq), W(i, k)));
            else
                W(i, k) = fma(-l1[i], akq1, fma(-l0[i], akq, W(i, k)));
        }
        if (wk->st) wk->st->ops_update += 2 * ((p - k) + (nrow - p));
    }
    for (int i = q + 2; i < nrow; i++) {
        W(i, q) = l0[i];
        W(i, q + 1) = l1[i];
    }
    if (wk->st) wk->st->ops_apply += 4 * (nrow - q - 2);
}

/* Zero pivot at position q: D = 0, L column = 0, no update (Listing 1, Q7). */
static void pivot_zero(work_t *wk, int q) {
    int nrow = wk->p + wk->rt + wk->rs;
    wk->piv[q] = PIV_ZERO;
    wk->D[2 * q] = 0.0;
    wk->D[2 * q + 1] = 0.0;
    for (int i = q + 1; i < nrow; i++) W(i, q) = 0.0;
}

/* Listing 1 (Section 2) on the working matrix, with readings Q1-Q10.
 * stop_nelim >= 0 stops as soon as nelim >= stop_nelim (used only by the
 * invariant tests that look at intermediate stages).  Returns nelim. */
static int listing1(work_t *wk, int stop_nelim) {
    int p = wk->p, nrow = p + wk->rt + wk->rs;
    double *l0 = (double *)calloc((size_t)nrow + 1, sizeof(double));
    double *l1 = (double *)calloc((size_t)nrow + 1, sizeof(double));
    for (int k = 0; k < p; k++) wk->piv[k] = PIV_DELAYED;
    for (int k = 0; k < 2 * p; k++) wk->D[k] = 0.0;
    int nelim = 0;
    int m = (p >= 2) ? 1 : 0; /* Listing 1 starts with m = 2 (1-based) */
    int accepted_in_sweep = 0;
    if (wk->st) wk->st->sweeps = 1;
    while (nelim < p) {
        if (stop_nelim >= 0 && nelim >= stop_nelim) break;
        if (m >= p) {
            if (!accepted_in_sweep) break; /* no elimination possible any more */
            accepted_in_sweep = 0;
            m = nelim; /* new sweep from the first uneliminated column */
            if (wk->st) wk->st->sweeps++;
            continue;
        }
        int m_orig = wk->perm[m];
        /* special 1x1 case: the whole uneliminated column is below small */
        double cmax = col_max(wk, nelim, m, -1, -1);
        if (cmax < wk->small) {
            log_push(wk, LOG_ZERO, m_orig, -1, cmax, wk->small, 1);
            move_to(wk, m, nelim);
            pivot_zero(wk, nelim);
            nelim++;
            if (wk->st) wk->st->zero_pivots++;
            accepted_in_sweep = 1;
            m++;
            continue;
        }
        log_push(wk, LOG_ZERO, m_orig, -1, cmax, wk->small, 0);
        if (m > nelim) {
            /* t: column of the largest |a(m, nelim:m-1)|, lowest index on ties */
            int t = nelim;
            double best = fabs(W(m, nelim));
            for (int j = nelim + 1; j < m; j++) {
                double v = fabs(W(m, j));
                if (v > best) {
                    best = v;
                    t = j;
                }
            }
            double maxt = col_max(wk, nelim, t, t, m);
            double maxm = col_max(wk, nelim, m, t, m);
            if (wk->st) {
                wk->st->tests_2x2++;
                wk->st->ops_colmax += 2 * ((int64_t)(p - nelim - 2) + wk->rt - 1);
                wk->st->ops_test += 18;
            }
            if (test_2x2(wk, m_orig, wk->perm[t], W(t, t), W(m, t), W(m, m), maxt, maxm)) {
                move_to(wk, t, nelim);     /* t < m: m stays at position m */
                move_to(wk, m, nelim + 1); /* stable shift of the rejected columns */
                pivot_2x2(wk, nelim, l0, l1);
                nelim += 2;
                if (wk->st) wk->st->accepted_2x2++;
                accepted_in_sweep = 1;
                m++; /* the column that followed m is still at position m+1 */
                continue;
            }
        }
        /* failed as 2x2 (or no partner): try as 1x1 */
        double maxm1 = col_max(wk, nelim, m, m, -1);
        double lhs = fabs(W(m, m)), rhs = wk->u * maxm1;
        if (wk->st) wk->st->tests_1x1++;
        if (lhs >= rhs) {
            log_push(wk, LOG_1X1, m_orig, -1, lhs, rhs, 1);
            move_to(wk, m, nelim);
            pivot_1x1(wk, nelim, l0);
            nelim++;
            if (wk->st) wk->st->accepted_1x1++;
            accepted_in_sweep = 1;
            m++;
            continue;
        }
        log_push(wk, LOG_1X1, m_orig, -1, lhs, rhs, 0);
        m++; /* candidate rejected: it stays in place */
    }
    free(l0);
    free(l1);
    return nelim;
}

/* ------------------------------------------------------------------------- */
/* Compression of A21 (Section 4.1 and Section 4.2).                          */

/* Strict compression, eq. (4.1): J(i) = argmax_k |a21(i,k)| (lowest k on ties),
 * c(j,k) = max over rows i with J(i) = j of |a21(i,k)|, 0 if there is none.
 * C is p x p column-major (ldc >= p).  J (length m) may be NULL. */
int orc_compress_strict(int m, int p, const double *A21, int64_t lda, double *C, int64_t ldc,
                        int32_t *J) {
    if (m < 0 || p < 1 || lda < m || ldc < p) return ORC_EINVAL;
    for (int k = 0; k < p; k++)
        for (int j = 0; j < p; j++) C[(int64_t)k * ldc + j] = 0.0;
    for (int i = 0; i < m; i++) {
        int arg = 0;
        double best = fabs(A21[i]);
        for (int k = 1; k < p; k++) {
            double v = fabs(A21[(int64_t)k * lda + i]);
            if (v > best) {
                best = v;
                arg = k;
            }
        }
        if (J) J[i] = arg;
        for (int k = 0; k < p; k++) {
            double v = fabs(A21[(int64_t)k * lda + i]);
            if (v > C[(int64_t)k * ldc + arg]) C[(int64_t)k * ldc + arg] = v;
        }
    }
    return ORC_OK;
}

/* Relaxed compression (Section 4.2): for j = 1..p, the unflagged row holding the
 * largest |a21(i,j)| (lowest i on ties) is flagged and copied, with its signs,
 * into row j of C.  rows[j] = chosen A21 row, or -1 when every row was already
 * flagged (C row j is then zero). */
int orc_compress_relaxed(int m, int p, const double *A21, int64_t lda, double *C, int64_t ldc,
                         int32_t *rows) {
    if (m < 0 || p < 1 || lda < m || ldc < p) return ORC_EINVAL;
    char *flag = (char *)calloc((size_t)m + 1, 1);
    if (!flag) return ORC_ENOMEM;
    for (int j = 0; j < p; j++) {
        int arg = -1;
        double best = -1.0;
        for (int i = 0; i < m; i++) {
            if (flag[i]) continue;
            double v = fabs(A21[(int64_t)j * lda + i]);
            if (v > best) {
                best = v;
                arg = i;
            }
        }
        if (rows) rows[j] = arg;
        for (int k = 0; k < p; k++) C[(int64_t)k * ldc + j] = (arg >= 0) ? A21[(int64_t)k * lda + arg] : 0.0;
        if (arg >= 0) flag[arg] = 1;
    }
    free(flag);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Listing 1 on a caller-built working matrix (exposed for invariant tests).  */
/* W is (p+rt+rs) x p column-major; rows 0..p-1 must hold A11 in full
 * symmetric form.  perm[] is filled with 0..p-1 on entry. */
int orc_listing1(int p, int rt, int rs, int tmode, double *Wm, int64_t ldw, double u, double small,
                 int stop_nelim, int32_t *perm, int32_t *piv, double *D, int32_t *nelim,
                 orc_stats *st, orc_log_entry *log, int log_cap, int32_t *log_len) {
    if (p < 1 || rt < 0 || rs < 0 || ldw < p + rt + rs || !(u > 0.0) || u > 0.5) return ORC_EINVAL;
    work_t wk;
    memset(&wk, 0, sizeof(wk));
    wk.p = p;
    wk.rt = rt;
    wk.rs = rs;
    wk.tmode = tmode;
    wk.ldw = ldw;
    wk.w = Wm;
    int *pm = (int *)malloc(sizeof(int) * (size_t)p);
    int *pv = (int *)malloc(sizeof(int) * (size_t)p);
    for (int k = 0; k < p; k++) pm[k] = k;
    wk.perm = pm;
    wk.piv = pv;
    wk.D = D;
    wk.u = u;
    wk.small = small;
    wk.log = log;
    wk.log_cap = log_cap;
    wk.st = st;
    if (st) memset(st, 0, sizeof(*st));
    int e = listing1(&wk, stop_nelim);
    for (int k = 0; k < p; k++) {
        perm[k] = pm[k];
        piv[k] = pv[k];
    }
    *nelim = e;
    if (log_len) *log_len = wk.log_len;
    free(pm);
    free(pv);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Solve (Section 1 task list, Figure 4.1 (d),(e)): apply the pivots chosen on
 * [A11; C] to A21 in one pass.  X = A21 P^T (rows never move).  With L11 the
 * unit lower factor of the e eliminated positions, L_d its rows for the
 * delayed positions and D11 block diagonal:
 *   Y   = X_e L11^{-T}        (forward substitution, column by column)
 *   L21 = Y D11^{-1}          (1x1 and 2x2 blocks; zero pivots give 0)
 *   R   = X_d - Y L_d^T       (update of the delayed columns)
 * Wf is the factored p x p block (positions), as left by Listing 1. */
static void apply_solve(int m, int p, int e, const double *Wf, int64_t ldw, const int *perm,
                        const int *piv, const double *D, double *A21, int64_t lda) {
    double *x = (double *)malloc(sizeof(double) * (size_t)p);
    double *y = (double *)malloc(sizeof(double) * (size_t)p);
#define LF(i, j) Wf[(int64_t)(j) * ldw + (i)]
    for (int i = 0; i < m; i++) {
        for (int k = 0; k < p; k++) x[k] = A21[(int64_t)perm[k] * lda + i];
        /* forward substitution with the unit lower L11; inside a 2x2 block the
           (q+1, q) slot holds D, and L there is 0 */
        for (int j = 0; j < e; j++) {
            double s = x[j];
            for (int k = 0; k < j; k++) {
                double ljk = (piv[k] == PIV_2X2_FIRST && j == k + 1) ? 0.0 : LF(j, k);
                s -= y[k] * ljk;
            }
            y[j] = s;
        }
        /* delayed columns */
        for (int k = e; k < p; k++) {
            double s = x[k];
            for (int j = 0; j < e; j++) s -= y[j] * LF(k, j);
            A21[(int64_t)k * lda + i] = s;
        }
        /* L21 = Y D11^{-1} */
        for (int j = 0; j < e; j++) {
            if (piv[j] == PIV_1X1) {
                A21[(int64_t)j * lda + i] = y[j] / D[2 * j];
            } else if (piv[j] == PIV_ZERO) {
                A21[(int64_t)j * lda + i] = 0.0;
            } else if (piv[j] == PIV_2X2_FIRST) {
                double a = D[2 * j], b = D[2 * j + 1], c = D[2 * j + 2];
                double amax = fmax(fabs(a), fmax(fabs(b), fabs(c)));
                double detscale = 1.0 / amax;
                double detpiv = c * detscale * a - (b * detscale) * b;
                double i11 = (c * detscale) / detpiv;
                double i21 = (-b * detscale) / detpiv;
                double i22 = (a * detscale) / detpiv;
                A21[(int64_t)j * lda + i] = y[j] * i11 + y[j + 1] * i21;
                A21[(int64_t)(j + 1) * lda + i] = y[j] * i21 + y[j + 1] * i22;
            }
        }
    }
#undef LF
    free(x);
    free(y);
}

/* Full supernode: compression (strict / relaxed / single-row), Listing 1 on
 * [A11; C] (or on [A11; A21] for TPP, on A11 alone for restricted pivoting),
 * then Solve and the delayed-column update.  A is overwritten in place:
 *   rows 0..p-1, lower triangle, in pivot order: L11 (unit diagonal implied),
 *     D on the diagonal and in the (q+1,q) slot of each 2x2 block, L_d in the
 *     delayed rows, and the updated delayed block;
 *   rows p..n-1: L21 in the first e columns, updated delayed columns after.
 * C_out (p x p, may be NULL) receives the compressed matrix before factoring. */
int orc_factor(int n, int p, double *A, int64_t lda, int method, double u, double small,
               int32_t *perm, int32_t *piv, double *D, int32_t *nelim, double *C_out,
               orc_stats *st, orc_log_entry *log, int log_cap, int32_t *log_len) {
    if (p < 1 || n < p || lda < n || !(u > 0.0) || u > 0.5) return ORC_EINVAL;
    if (method < 0 || method > 4) return ORC_EINVAL;
    int m = n - p;
    int rt = (method == ORC_TPP) ? m : (method == ORC_RESTRICTED ? 0 : (method == ORC_SINGLE_ROW ? 1 : p));
    int64_t ldw = p + rt;
    double *Wm = (double *)calloc((size_t)ldw * (size_t)p, sizeof(double));
    if (!Wm) return ORC_ENOMEM;
    /* A11 in full symmetric form from its lower triangle */
    for (int j = 0; j < p; j++)
        for (int i = j; i < p; i++) {
            Wm[(int64_t)j * ldw + i] = A[(int64_t)j * lda + i];
            Wm[(int64_t)i * ldw + j] = A[(int64_t)j * lda + i];
        }
    if (method == ORC_TPP) {
        for (int j = 0; j < p; j++)
            for (int i = 0; i < m; i++) Wm[(int64_t)j * ldw + p + i] = A[(int64_t)j * lda + p + i];
    } else if (method == ORC_STRICT) {
        orc_compress_strict(m, p, A + p, lda, Wm + p, ldw, NULL);
    } else if (method == ORC_RELAXED) {
        orc_compress_relaxed(m, p, A + p, lda, Wm + p, ldw, NULL);
    } else if (method == ORC_SINGLE_ROW) {
        /* eq. (4.1) with one set J = {1, ..., n-p}: C is the single row of
           column maxima c(k) = max_i |a21(i,k)| (0 when A21 has no rows) */
        for (int k = 0; k < p; k++) {
            double c = 0.0;
            for (int i = 0; i < m; i++) c = fmax(c, fabs(A[(int64_t)k * lda + p + i]));
            Wm[(int64_t)k * ldw + p] = c;
        }
    }
    if (C_out) {
        for (int j = 0; j < p; j++)
            for (int i = 0; i < p; i++)
                C_out[(int64_t)j * p + i] = (method == ORC_STRICT || method == ORC_RELAXED ||
                                             (method == ORC_SINGLE_ROW && i == 0))
                                                ? Wm[(int64_t)j * ldw + p + i]
                                                : 0.0;
    }
    int rc = orc_listing1(p, rt, 0, (method == ORC_STRICT || method == ORC_SINGLE_ROW) ? UPD_ABS : UPD_NORMAL,
                          Wm, ldw, u, small, -1,
                          perm, piv, D, nelim, st, log, log_cap, log_len);
    if (rc != ORC_OK) {
        free(Wm);
        return rc;
    }
    int e = *nelim;
    /* A11 block, lower triangle, in pivot order */
    for (int j = 0; j < p; j++)
        for (int i = j; i < p; i++) A[(int64_t)j * lda + i] = Wm[(int64_t)j * ldw + i];
    if (method == ORC_TPP) {
        for (int j = 0; j < p; j++)
            for (int i = 0; i < m; i++) A[(int64_t)j * lda + p + i] = Wm[(int64_t)j * ldw + p + i];
    } else {
        apply_solve(m, p, e, Wm, ldw, perm, piv, D, A + p, lda);
    }
    free(Wm);
    return ORC_OK;
}

/* Form (Section 1 task list): S = L21 D11 L21^T, lower triangle only.
 * L21 is m x e (column-major, ldl), S is m x m (column-major, lds). */
int orc_form(int m, int e, const double *L21, int64_t ldl, const int32_t *piv, const double *D,
             double *S, int64_t lds) {
    if (m < 0 || e < 0 || ldl < m || lds < m) return ORC_EINVAL;
    double *Wd = (double *)calloc((size_t)m * (size_t)(e > 0 ? e : 1), sizeof(double));
    if (!Wd) return ORC_ENOMEM;
    /* W21 = L21 D11 */
    for (int k = 0; k < e; k++) {
        if (piv[k] == PIV_1X1) {
            for (int i = 0; i < m; i++) Wd[(int64_t)k * m + i] = L21[(int64_t)k * ldl + i] * D[2 * k];
        } else if (piv[k] == PIV_2X2_FIRST) {
            double a = D[2 * k], b = D[2 * k + 1], c = D[2 * k + 2];
            for (int i = 0; i < m; i++) {
                double x = L21[(int64_t)k * ldl + i], y = L21[(int64_t)(k + 1) * ldl + i];
                Wd[(int64_t)k * m + i] = x * a + y * b;
                Wd[(int64_t)(k + 1) * m + i] = x * b + y * c;
            }
        }
        /* zero pivots and second columns of 2x2 blocks: handled above or zero */
    }
    for (int j = 0; j < m; j++)
        for (int i = j; i < m; i++) {
            double s = 0.0;
            for (int k = 0; k < e; k++) s += Wd[(int64_t)k * m + i] * L21[(int64_t)k * ldl + j];
            S[(int64_t)j * lds + i] = s;
        }
    free(Wd);
    return ORC_OK;
}

/* Selected entries of S = L21 D11 L21^T (for parity checks on sizes where the
 * whole S is out of reach of this code): val[t] = S(ii[t], jj[t]). */
int orc_form_entries(int m, int e, const double *L21, int64_t ldl, const int32_t *piv,
                     const double *D, int count, const int64_t *ii, const int64_t *jj, double *val) {
    if (m < 0 || e < 0 || ldl < m) return ORC_EINVAL;
    for (int t = 0; t < count; t++) {
        int64_t i = ii[t], j = jj[t];
        double s = 0.0;
        for (int k = 0; k < e; k++) {
            double wik;
            if (piv[k] == PIV_1X1) {
                wik = L21[(int64_t)k * ldl + i] * D[2 * k];
            } else if (piv[k] == PIV_2X2_FIRST) {
                wik = L21[(int64_t)k * ldl + i] * D[2 * k] + L21[(int64_t)(k + 1) * ldl + i] * D[2 * k + 1];
            } else if (piv[k] == PIV_2X2_SECOND) {
                wik = L21[(int64_t)(k - 1) * ldl + i] * D[2 * (k - 1) + 1] + L21[(int64_t)k * ldl + i] * D[2 * k];
            } else {
                wik = 0.0;
            }
            s += wik * L21[(int64_t)k * ldl + j];
        }
        val[t] = s;
    }
    return ORC_OK;
}


/* Factorization with a prescribed pivot sequence in natural order (no tests):
 * piv_in[k] = PIV_1X1 or PIV_2X2_FIRST/PIV_2X2_SECOND for k = 0..e-1, normal
 * right-looking update of every row (the classical LDL^T recurrence used in
 * the proofs of Section 5).  A (n x p, A11 lower read) is overwritten with the
 * same layout as orc_factor; D receives the pivot blocks. */
int orc_ldlt_fixed(int n, int p, double *A, int64_t lda, int e, const int32_t *piv_in, double *D) {
    if (p < 1 || n < p || lda < n || e < 0 || e > p) return ORC_EINVAL;
    int64_t ldw = n;
    double *Wm = (double *)calloc((size_t)n * (size_t)p, sizeof(double));
    double *l0 = (double *)calloc((size_t)n + 1, sizeof(double));
    double *l1 = (double *)calloc((size_t)n + 1, sizeof(double));
    int *pm = (int *)malloc(sizeof(int) * (size_t)p);
    int *pv = (int *)malloc(sizeof(int) * (size_t)p);
    for (int j = 0; j < p; j++) {
        pm[j] = j;
        pv[j] = PIV_DELAYED;
        for (int i = j; i < p; i++) {
            Wm[(int64_t)j * ldw + i] = A[(int64_t)j * lda + i];
            Wm[(int64_t)i * ldw + j] = A[(int64_t)j * lda + i];
        }
        for (int i = p; i < n; i++) Wm[(int64_t)j * ldw + i] = A[(int64_t)j * lda + i];
    }
    for (int k = 0; k < 2 * p; k++) D[k] = 0.0;
    work_t wk;
    memset(&wk, 0, sizeof(wk));
    wk.p = p;
    wk.rt = n - p;
    wk.tmode = UPD_NORMAL;
    wk.ldw = ldw;
    wk.w = Wm;
    wk.perm = pm;
    wk.piv = pv;
    wk.D = D;
    wk.u = 0.5;
    wk.small = 0.0;
    int q = 0;
    while (q < e) {
        if (piv_in[q] == PIV_2X2_FIRST && q + 1 < e) {
            pivot_2x2(&wk, q, l0, l1);
            q += 2;
        } else {
            pivot_1x1(&wk, q, l0);
            q += 1;
        }
    }
    for (int j = 0; j < p; j++) {
        for (int i = j; i < p; i++) A[(int64_t)j * lda + i] = Wm[(int64_t)j * ldw + i];
        for (int i = p; i < n; i++) A[(int64_t)j * lda + i] = Wm[(int64_t)j * ldw + i];
    }
    free(Wm);
    free(l0);
    free(l1);
    free(pm);
    free(pv);
    return ORC_OK;
}

int orc_abi_version(void) { return 1; }
