/*
 * rorbk_oracle.c -- plain, slow, FP64 CPU restatement of ROR-BK.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the CUDA
 * solver.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or helper with
 * the CUDA path, and nothing in the product path calls it.
 *
 * Source: Kar & Venkatapathi, "A fast solver for ill-conditioned linear
 * systems using randomized stable solutions of its blocks" (arXiv 2510.02156).
 *   - Algorithm 1 (ROR-BK): setup steps (uniform contiguous aggregation,
 *     centroids, C, P) and the iteration (3 sampled regularised block
 *     updates, full residual, convergence test, residual top-K dynamic block).
 *   - Section 2, the formula for P_t: Pbar_t = exp(-2 sum_j C(t,j) / n).
 *   - Section 2, the definition of C(i,j) = |<Abar_i,Abar_j>|/(|Abar_i||Abar_j|)
 *     with the centroid being the plain sum of the block's rows.
 *   - Section 3.1: the static blocks' (A_t A_t^T + mu I)^{-1} are computed
 *     once and stored; the update is x += A_t^T W_t (b_t - A_t x).
 *   - Eq. (3) / Lemma 1 / Theorem 1 are pinned by the tests, not used here.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - partition: block t holds rows [off_t, off_{t+1}) with
 *     off_t = t*floor(m/k) + min(t, m mod k)  (the first m mod k blocks get
 *     one extra row; every block has >= floor(m/k) rows as Section 2 asks);
 *   - C(t,t) = 1; C(t,j) = 0 for j != t if either centroid is zero;
 *   - the sampler is a Philox4x64-10 counter stream (Salmon et al., SC'11):
 *     key = (seed, system_id), counter = (iteration, l, 0, 0), word 0,
 *     u = (w >> 11) * 2^-53, tau = min{ t : u * cdf[k-1] < cdf[t] } with the
 *     cdf summed sequentially in FP64 from Pbar (the normalisation of P is
 *     folded into u * cdf[k-1]);
 *   - convergence: ||b - A x|| / ||b|| <= tol, tested after the static updates
 *     and before the dynamic one, as Algorithm 1 orders it; ||b|| = 0 returns
 *     x = 0 after zero iterations;
 *   - top-K: the K = floor(m/k) rows with the largest |r_i| (the same order as
 *     r_i^2), ties to the lower row index, returned in ascending row order;
 *   - the dynamic block uses r_I from the full residual (x has not changed
 *     since it was formed, so b_I - A_I x = r_I);
 *   - static operators W_t are formed lazily on the first draw of block t and
 *     then kept (the paper forms them once and stores them; forming them on
 *     first use gives the same numbers);
 *   - W_t = L^{-T} L^{-1} with L = chol(A_t A_t^T + mu I).
 *
 * Rounding: every multiply-add a*b + c is one IEEE 754 fusedMultiplyAdd
 * (C99 fma), rounded once; plain sums and quotients round as written.
 *
 * Fixed summation orders (so that each number has one definition):
 *   - row dot products run over a CSR row in stored (ascending column) order,
 *     a dense row in column order;
 *   - (A_B^T y)_c sums over the block's rows in ascending order into a zeroed
 *     vector delta, and then x_c += delta_c;
 *   - Gram entries G_ij = sum_c A_ic A_jc in ascending column order;
 *   - y = W r sums over ascending columns of W;
 *   - norms are sequential sums of squares.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* Matrix view: CSR (int64 row pointers, int32 columns, FP64 values) or dense
 * row-major FP64.  FP32-defined systems are passed widened to FP64, which is
 * exact. */
typedef struct {
    int64_t m, n;
    int32_t is_dense;
    int32_t pad_;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *val;
    const double *dense;
    int64_t ld;
} orc_matrix;

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOT_SPD (-4)
#define ORC_ERR_OOM (-3)

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  One round maps (X0,X1,X2,X3) with key (K0,K1)
 * to (hi(M1*X2)^X1^K0, lo(M1*X2), hi(M0*X0)^X3^K1, lo(M0*X0)); the key is
 * bumped by the Weyl constants between rounds. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        uint64_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, the block partition: uniform contiguous aggregation into k blocks. */
int orc_partition(int64_t m, int64_t k, int64_t *off)
{
    if (k < 1 || k > m) return ORC_ERR_ARG;
    int64_t q = m / k, rem = m % k;
    for (int64_t t = 0; t <= k; ++t)
        off[t] = t * q + (t < rem ? t : rem);
    return ORC_OK;
}

/* Row helpers.  dot = sum_c A_ic x_c in stored order. */
static double row_dot(const orc_matrix *A, int64_t i, const double *x)
{
    double s = 0.0;
    if (A->is_dense) {
        const double *a = A->dense + i * A->ld;
        for (int64_t c = 0; c < A->n; ++c) s = fma(a[c], x[c], s);
    } else {
        for (int64_t p = A->row_ptr[i]; p < A->row_ptr[i + 1]; ++p)
            s = fma(A->val[p], x[A->col_idx[p]], s);
    }
    return s;
}

/* Gram entry <A_i, A_j> in ascending column order. */
static double row_row_dot(const orc_matrix *A, int64_t i, int64_t j)
{
    double s = 0.0;
    if (A->is_dense) {
        const double *a = A->dense + i * A->ld, *b = A->dense + j * A->ld;
        for (int64_t c = 0; c < A->n; ++c) s = fma(a[c], b[c], s);
        return s;
    }
    int64_t p = A->row_ptr[i], pe = A->row_ptr[i + 1];
    int64_t q = A->row_ptr[j], qe = A->row_ptr[j + 1];
    while (p < pe && q < qe) {
        int32_t cp = A->col_idx[p], cq = A->col_idx[q];
        if (cp == cq) { s = fma(A->val[p], A->val[q], s); ++p; ++q; }
        else if (cp < cq) ++p;
        else ++q;
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1's set-up and the Section 2 definitions: centroids
 * Abar_t = sum of the block's rows, C(i,j) = |<Abar_i,Abar_j>|/(|Abar_i||Abar_j|).
 * Outputs the row sums sum_j C(t,j) (always) and the full k x k matrix C when
 * C != NULL.  Each centroid is kept as a sorted (column, value) list; the
 * Gram matrix Abar Abar^T is formed as a sum over columns c (ascending) of
 * the outer products of column c of Abar^T: G(i,j) = sum_c Abar_ic Abar_jc. */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int orc_orthogonality(const orc_matrix *A, int64_t k, const int64_t *off,
                      double *C, double *C_rowsum)
{
    int64_t n = A->n;
    int st = ORC_ERR_OOM;
    double *acc = (double *)calloc((size_t)n, sizeof(double));
    unsigned char *seen = (unsigned char *)calloc((size_t)n, 1);
    int64_t *cptr = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    int64_t *colcnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t cap = 1024, used = 0;
    int32_t *ccol = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    double *cval = (double *)malloc((size_t)cap * sizeof(double));
    int32_t *cb = NULL;
    double *cv = NULL, *G = NULL;
    int64_t *fill = NULL;
    if (!acc || !seen || !cptr || !colcnt || !ccol || !cval) goto out;

    /* centroids: sum of the block's rows (rows ascending) */
    for (int64_t t = 0; t < k; ++t) {
        int64_t need = used + (A->is_dense ? n : 0);
        if (!A->is_dense)
            for (int64_t i = off[t]; i < off[t + 1]; ++i)
                need += A->row_ptr[i + 1] - A->row_ptr[i];
        if (need > cap) {
            while (cap < need) cap *= 2;
            int32_t *nc = (int32_t *)realloc(ccol, (size_t)cap * sizeof(int32_t));
            if (!nc) goto out;
            ccol = nc;
            double *nv = (double *)realloc(cval, (size_t)cap * sizeof(double));
            if (!nv) goto out;
            cval = nv;
        }
        int64_t len = 0;
        for (int64_t i = off[t]; i < off[t + 1]; ++i) {
            if (A->is_dense) {
                for (int64_t c = 0; c < n; ++c) acc[c] += A->dense[i * A->ld + c];
                continue;
            }
            for (int64_t p = A->row_ptr[i]; p < A->row_ptr[i + 1]; ++p) {
                int32_t c = A->col_idx[p];
                acc[c] += A->val[p];
                if (!seen[c]) { seen[c] = 1; ccol[used + len++] = c; }
            }
        }
        if (A->is_dense) {
            for (int64_t c = 0; c < n; ++c) ccol[used + c] = (int32_t)c;
            len = n;
        } else {
            qsort(ccol + used, (size_t)len, sizeof(int32_t), cmp_i32);
        }
        for (int64_t a = 0; a < len; ++a) {
            int32_t c = ccol[used + a];
            cval[used + a] = acc[c];
            acc[c] = 0.0;
            seen[c] = 0;
            colcnt[c + 1]++;
        }
        used += len;
        cptr[t + 1] = used;
    }

    /* column lists of Abar (blocks in ascending order), then the Gram */
    for (int64_t c = 0; c < n; ++c) colcnt[c + 1] += colcnt[c];
    cb = (int32_t *)malloc((size_t)(used ? used : 1) * sizeof(int32_t));
    cv = (double *)malloc((size_t)(used ? used : 1) * sizeof(double));
    fill = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    G = (double *)calloc((size_t)k * (size_t)k, sizeof(double));
    if (!cb || !cv || !fill || !G) goto out;
    for (int64_t c = 0; c < n; ++c) fill[c] = colcnt[c];
    for (int64_t t = 0; t < k; ++t)
        for (int64_t a = cptr[t]; a < cptr[t + 1]; ++a) {
            int64_t pos = fill[ccol[a]]++;
            cb[pos] = (int32_t)t;
            cv[pos] = cval[a];
        }
    for (int64_t c = 0; c < n; ++c)
        for (int64_t a = colcnt[c]; a < colcnt[c + 1]; ++a)
            for (int64_t b2 = colcnt[c]; b2 < colcnt[c + 1]; ++b2)
                G[(int64_t)cb[a] * k + cb[b2]] = fma(cv[a], cv[b2], G[(int64_t)cb[a] * k + cb[b2]]);

    for (int64_t i = 0; i < k; ++i) {
        double rsum = 0.0;
        double ni = sqrt(G[i * k + i]);
        for (int64_t j = 0; j < k; ++j) {
            double nj = sqrt(G[j * k + j]);
            double cij;
            if (i == j) cij = 1.0;
            else if (ni == 0.0 || nj == 0.0) cij = 0.0;
            else cij = fabs(G[i * k + j]) / (ni * nj);
            if (C) C[i * k + j] = cij;
            rsum += cij;
        }
        C_rowsum[i] = rsum;
    }
    st = ORC_OK;
out:
    free(acc); free(seen); free(cptr); free(colcnt); free(ccol); free(cval);
    free(cb); free(cv); free(fill); free(G);
    return st;
}

/* Algorithm 1's proposal / Section 2: Pbar_t = exp(-2 sum_j C(t,j) / n),
 * P = Pbar / sum(Pbar).  Also the sequential FP64 prefix sum cdf_t. */
void orc_proposal(const double *C_rowsum, int64_t k, int64_t n, double *Pbar,
                  double *P, double *cdf)
{
    double s = 0.0;
    for (int64_t t = 0; t < k; ++t) {
        Pbar[t] = exp(-2.0 * C_rowsum[t] / (double)n);
        s += Pbar[t];
        cdf[t] = s;
    }
    if (P) for (int64_t t = 0; t < k; ++t) P[t] = Pbar[t] / s;
}

/* Draw tau for (iteration it, static update l). */
int64_t orc_sample(const double *cdf, int64_t k, uint64_t seed, uint64_t sysid,
                   int64_t it, int64_t l)
{
    uint64_t ctr[4] = {(uint64_t)it, (uint64_t)l, 0, 0}, key[2] = {seed, sysid}, w[4];
    orc_philox4x64_10(ctr, key, w);
    double u = (double)(w[0] >> 11) * 0x1.0p-53;
    double target = u * cdf[k - 1];
    for (int64_t t = 0; t < k; ++t)
        if (target < cdf[t]) return t;
    return k - 1;
}

/* ------------------------------------------------------------------------ */
/* Host threads.  The residual's rows and the top-K scan are split into
 * contiguous row ranges over the host cores; each row's arithmetic and every
 * result are the same as with one thread (rows are independent, the sum of
 * squares stays one sequential chain, and the top-K set is unique).
 * ORC_THREADS overrides the count; inputs under 65536 rows use one thread. */
int orc_thread_count(int64_t rows)
{
    if (rows < 65536) return 1;
    const char *e = getenv("ORC_THREADS");
    long t = e ? atol(e) : sysconf(_SC_NPROCESSORS_ONLN);
    if (t < 1) t = 1;
    if (t > 256) t = 256;
    return (int)t;
}

typedef struct {
    const orc_matrix *A;
    const double *b, *x;
    double *r;
    int64_t i0, i1;
} residual_job;

static void *residual_rows(void *arg)
{
    residual_job *j = (residual_job *)arg;
    for (int64_t i = j->i0; i < j->i1; ++i) j->r[i] = j->b[i] - row_dot(j->A, i, j->x);
    return NULL;
}

/* Algorithm 1: r = b - A x and ||r||^2 (sequential sum). */
double orc_residual(const orc_matrix *A, const double *b, const double *x, double *r)
{
    const int T = orc_thread_count(A->m);
    residual_job jobs[256];
    pthread_t th[256];
    int started[256];
    for (int t = 0; t < T; ++t) {
        jobs[t].A = A; jobs[t].b = b; jobs[t].x = x; jobs[t].r = r;
        jobs[t].i0 = A->m * t / T;
        jobs[t].i1 = A->m * (t + 1) / T;
        started[t] = t > 0 && pthread_create(&th[t], NULL, residual_rows, &jobs[t]) == 0;
    }
    for (int t = 0; t < T; ++t)
        if (!started[t]) residual_rows(&jobs[t]);
    for (int t = 1; t < T; ++t)
        if (started[t]) pthread_join(th[t], NULL);
    double rr = 0.0;
    for (int64_t i = 0; i < A->m; ++i) rr = fma(r[i], r[i], rr);
    return rr;
}

/* Algorithm 1 (residual-based dynamic aggregation): indices of the K largest
 * |r_i| (ties to the lower index), written in ascending order.  A bounded
 * min-heap keyed on (|r|, -index) keeps the current best K.  With several
 * threads each keeps the best K of its row range and the ranges' survivors
 * are offered to one heap: the K best under this strict order are unique, so
 * the set is the one-thread set. */
static int heap_less(double ka, int64_t ia, double kb, int64_t ib)
{   /* "a ranks below b": smaller key, or equal key and larger index */
    return ka < kb || (ka == kb && ia > ib);
}

typedef struct {
    double *hk;
    int64_t *hi;
    int64_t size, K;
} topk_heap;

static void heap_offer(topk_heap *h, double key, int64_t i)
{
    double *hk = h->hk;
    int64_t *hi = h->hi;
    const int64_t K = h->K;
    if (h->size < K) {
        int64_t c = h->size++;
        hk[c] = key; hi[c] = i;
        while (c > 0) {
            int64_t p = (c - 1) / 2;
            if (heap_less(hk[c], hi[c], hk[p], hi[p])) {
                double tk = hk[c]; hk[c] = hk[p]; hk[p] = tk;
                int64_t ti = hi[c]; hi[c] = hi[p]; hi[p] = ti;
                c = p;
            } else break;
        }
    } else if (heap_less(hk[0], hi[0], key, i)) {
        hk[0] = key; hi[0] = i;
        int64_t c = 0;
        for (;;) {
            int64_t a = 2 * c + 1, b2 = a + 1, s = c;
            if (a < K && heap_less(hk[a], hi[a], hk[s], hi[s])) s = a;
            if (b2 < K && heap_less(hk[b2], hi[b2], hk[s], hi[s])) s = b2;
            if (s == c) break;
            double tk = hk[c]; hk[c] = hk[s]; hk[s] = tk;
            int64_t ti = hi[c]; hi[c] = hi[s]; hi[s] = ti;
            c = s;
        }
    }
}

typedef struct {
    const double *r;
    int64_t i0, i1;
    topk_heap h;
} topk_job;

static void *topk_rows(void *arg)
{
    topk_job *j = (topk_job *)arg;
    for (int64_t i = j->i0; i < j->i1; ++i) heap_offer(&j->h, fabs(j->r[i]), i);
    return NULL;
}

int orc_topk(const double *r, int64_t m, int64_t K, int64_t *I)
{
    if (K < 0 || K > m) return ORC_ERR_ARG;
    if (K == 0) return ORC_OK;
    const int T = orc_thread_count(m);
    double *hk = (double *)malloc((size_t)(T + 1) * K * sizeof(double));
    int64_t *hi = (int64_t *)malloc((size_t)(T + 1) * K * sizeof(int64_t));
    if (!hk || !hi) { free(hk); free(hi); return ORC_ERR_OOM; }
    topk_job jobs[256];
    pthread_t th[256];
    int started[256];
    for (int t = 0; t < T; ++t) {
        jobs[t].r = r;
        jobs[t].i0 = m * t / T;
        jobs[t].i1 = m * (t + 1) / T;
        jobs[t].h.hk = hk + (int64_t)(t + 1) * K;
        jobs[t].h.hi = hi + (int64_t)(t + 1) * K;
        jobs[t].h.size = 0;
        jobs[t].h.K = K;
        started[t] = T > 1 && t > 0 && pthread_create(&th[t], NULL, topk_rows, &jobs[t]) == 0;
    }
    for (int t = 0; t < T; ++t)
        if (!started[t]) topk_rows(&jobs[t]);
    for (int t = 1; t < T; ++t)
        if (started[t]) pthread_join(th[t], NULL);
    topk_heap best = {hk, hi, 0, K};
    if (T == 1) {
        best = jobs[0].h;
    } else {
        for (int t = 0; t < T; ++t)
            for (int64_t a = 0; a < jobs[t].h.size; ++a) heap_offer(&best, jobs[t].h.hk[a], jobs[t].h.hi[a]);
    }
    /* ascending row order (insertion sort of K indices) */
    for (int64_t a = 0; a < K; ++a) I[a] = best.hi[a];
    for (int64_t a = 1; a < K; ++a) {
        int64_t v = I[a], b2 = a - 1;
        while (b2 >= 0 && I[b2] > v) { I[b2 + 1] = I[b2]; --b2; }
        I[b2 + 1] = v;
    }
    free(hk); free(hi);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense SPD helpers on an s x s row-major array. */

/* G = A_B A_B^T + mu I for the rows listed in rows[0..s). */
void orc_block_gram(const orc_matrix *A, const int64_t *rows, int64_t s,
                    double mu, double *G)
{
    for (int64_t a = 0; a < s; ++a)
        for (int64_t b2 = 0; b2 <= a; ++b2) {
            double g = row_row_dot(A, rows[a], rows[b2]);
            if (a == b2) g += mu;
            G[a * s + b2] = g;
            G[b2 * s + a] = g;
        }
}

/* Cholesky G = L L^T in place (lower triangle; the strict upper triangle is
 * zeroed).  Textbook column-by-column (Cholesky-Banachiewicz-free, i.e. the
 * right-looking outer-product form):
 *   for j: L_jj = sqrt(G_jj); L_ij = G_ij / L_jj (i > j);
 *          G_ab -= L_aj L_bj for a >= b > j.  */
int orc_cholesky(double *G, int64_t s)
{
    for (int64_t j = 0; j < s; ++j) {
        double d = G[j * s + j];
        if (!(d > 0.0)) return ORC_ERR_NOT_SPD;
        double l = sqrt(d);
        G[j * s + j] = l;
        for (int64_t i = j + 1; i < s; ++i) G[i * s + j] /= l;
        for (int64_t a = j + 1; a < s; ++a) {
            double la = G[a * s + j];
            for (int64_t b2 = j + 1; b2 <= a; ++b2)
                G[a * s + b2] = fma(-la, G[b2 * s + j], G[a * s + b2]);
        }
    }
    for (int64_t a = 0; a < s; ++a)
        for (int64_t b2 = a + 1; b2 < s; ++b2) G[a * s + b2] = 0.0;
    return ORC_OK;
}

/* y = (L L^T)^{-1} r by two triangular solves in column (saxpy) order:
 *   forward : y = r; for j = 0..s-1: y_j /= L_jj; y_i -= L_ij y_j (i > j);
 *   backward: for j = s-1..0: y_j /= L_jj; y_i -= L_ji y_j (i < j).
 * (Each y_i therefore receives its subtractions in ascending j on the way
 * forward and in descending j on the way back.) */
void orc_chol_solve(const double *L, int64_t s, const double *r, double *y)
{
    for (int64_t i = 0; i < s; ++i) y[i] = r[i];
    for (int64_t j = 0; j < s; ++j) {
        y[j] = y[j] / L[j * s + j];
        for (int64_t i = j + 1; i < s; ++i) y[i] = fma(-L[i * s + j], y[j], y[i]);
    }
    for (int64_t j = s - 1; j >= 0; --j) {
        y[j] = y[j] / L[j * s + j];
        for (int64_t i = 0; i < j; ++i) y[i] = fma(-L[j * s + i], y[j], y[i]);
    }
}

/* W = (L L^T)^{-1} = L^{-T} L^{-1}.  Linv by columns: Linv_jj = 1/L_jj,
 * Linv_ij = -(sum_{c=j}^{i-1} L_ic Linv_cj) / L_ii; then
 * W_ij = sum_{c >= max(i,j)} Linv_ci Linv_cj (c ascending). */
int orc_spd_inverse(const double *L, int64_t s, double *W)
{
    double *Li = (double *)calloc((size_t)(s * s), sizeof(double));
    if (!Li) return ORC_ERR_OOM;
    for (int64_t j = 0; j < s; ++j) {
        Li[j * s + j] = 1.0 / L[j * s + j];
        for (int64_t i = j + 1; i < s; ++i) {
            double acc = 0.0;
            for (int64_t c = j; c < i; ++c) acc = fma(L[i * s + c], Li[c * s + j], acc);
            Li[i * s + j] = -acc / L[i * s + i];
        }
    }
    for (int64_t i = 0; i < s; ++i)
        for (int64_t j = 0; j <= i; ++j) {
            double acc = 0.0;
            for (int64_t c = i; c < s; ++c) acc = fma(Li[c * s + i], Li[c * s + j], acc);
            W[i * s + j] = acc;
            W[j * s + i] = acc;
        }
    free(Li);
    return ORC_OK;
}

/* x += A_B^T y for the rows rows[0..s): delta_c = sum over rows ascending of
 * A_rc y_r (accumulated into the zeroed scratch delta[n]), then x_c += delta_c
 * for every column the block touches; delta is re-zeroed on exit. */
static void scatter_update(const orc_matrix *A, const int64_t *rows, int64_t s,
                           const double *y, double *x, double *delta)
{
    if (A->is_dense) {
        for (int64_t a = 0; a < s; ++a) {
            const double *ar = A->dense + rows[a] * A->ld;
            for (int64_t c = 0; c < A->n; ++c) delta[c] = fma(ar[c], y[a], delta[c]);
        }
        for (int64_t c = 0; c < A->n; ++c) { x[c] += delta[c]; delta[c] = 0.0; }
        return;
    }
    for (int64_t a = 0; a < s; ++a)
        for (int64_t p = A->row_ptr[rows[a]]; p < A->row_ptr[rows[a] + 1]; ++p)
            delta[A->col_idx[p]] = fma(A->val[p], y[a], delta[A->col_idx[p]]);
    /* a column shared by several rows is applied on its first visit; later
     * visits add the re-zeroed delta_c = 0, which leaves x_c unchanged */
    for (int64_t a = 0; a < s; ++a)
        for (int64_t p = A->row_ptr[rows[a]]; p < A->row_ptr[rows[a] + 1]; ++p) {
            int32_t c = A->col_idx[p];
            x[c] += delta[c];
            delta[c] = 0.0;
        }
}

/* The paper's update (Algorithm 1, Eq. in Lemma 2's proof) with a stored
 * inverse (Section 3.1): r_B = b_B - A_B x; y = W r_B; x += A_B^T y.
 * W is s x s row-major; y[i] = sum_j W_ij r_j in ascending j. */
void orc_update_with_inverse(const orc_matrix *A, const int64_t *rows, int64_t s,
                             const double *W, const double *b, double *x,
                             double *scratch_n, double *work_2s)
{
    double *rB = work_2s, *y = work_2s + s;
    for (int64_t a = 0; a < s; ++a) rB[a] = b[rows[a]] - row_dot(A, rows[a], x);
    for (int64_t a = 0; a < s; ++a) {
        double acc = 0.0;
        for (int64_t c = 0; c < s; ++c) acc = fma(W[a * s + c], rB[c], acc);
        y[a] = acc;
    }
    scatter_update(A, rows, s, y, x, scratch_n);
}

/* The dynamic-block update: G = A_I A_I^T + mu I, L = chol(G),
 * y = G^{-1} rI (two triangular solves), x += A_I^T y. */
int orc_update_with_cholesky(const orc_matrix *A, const int64_t *rows, int64_t s,
                             double mu, const double *rI, double *x,
                             double *scratch_n)
{
    double *G = (double *)malloc((size_t)(s * s) * sizeof(double));
    double *y = (double *)malloc((size_t)(s ? s : 1) * sizeof(double));
    if (!G || !y) { free(G); free(y); return ORC_ERR_OOM; }
    orc_block_gram(A, rows, s, mu, G);
    int st = orc_cholesky(G, s);
    if (st == ORC_OK) {
        orc_chol_solve(G, s, rI, y);
        scatter_update(A, rows, s, y, x, scratch_n);
    }
    free(G); free(y);
    return st;
}

/* Static operator W_t for block t (Section 3.1): chol then explicit inverse. */
int orc_static_operator(const orc_matrix *A, const int64_t *off, int64_t t,
                        double mu, double *W)
{
    int64_t s = off[t + 1] - off[t];
    int64_t *rows = (int64_t *)malloc((size_t)(s ? s : 1) * sizeof(int64_t));
    double *G = (double *)malloc((size_t)(s > 0 ? s * s : 1) * sizeof(double));
    if (!rows || !G) { free(rows); free(G); return ORC_ERR_OOM; }
    for (int64_t a = 0; a < s; ++a) rows[a] = off[t] + a;
    orc_block_gram(A, rows, s, mu, G);
    int st = orc_cholesky(G, s);
    if (st == ORC_OK) st = orc_spd_inverse(G, s, W);
    free(rows); free(G);
    return st;
}

/* ------------------------------------------------------------------------ */
/* The s >= n form (Lemma 1 and Section 3.1).  By Lemma 1,
 *   x + A_B^T (A_B A_B^T + mu I)^{-1} (b_B - A_B x)
 *     = x + (A_B^T A_B + mu I)^{-1} A_B^T (b_B - A_B x),
 * and Section 3.1 stores the n x n inverse on the right when the block has at
 * least as many rows as A has columns (s >= n).  The same reading is applied
 * to the dynamic block when K >= n.  Entries that are not stored count as
 * zero in the column sums below (a fused multiply-add by 0 leaves a finite
 * running sum unchanged, so this equals summing over the stored entries). */

/* The listed rows as a dense s x n row-major array. */
static void dense_rows(const orc_matrix *A, const int64_t *rows, int64_t s, double *D)
{
    const int64_t n = A->n;
    memset(D, 0, (size_t)(s * n) * sizeof(double));
    for (int64_t a = 0; a < s; ++a) {
        if (A->is_dense) {
            memcpy(D + a * n, A->dense + rows[a] * A->ld, (size_t)n * sizeof(double));
        } else {
            for (int64_t p = A->row_ptr[rows[a]]; p < A->row_ptr[rows[a] + 1]; ++p)
                D[a * n + A->col_idx[p]] = A->val[p];
        }
    }
}

/* G = A_B^T A_B + mu I (n x n row-major): G_cd = sum over the rows a in the
 * listed order of a_ac a_ad, a chain of fused multiply-adds from 0, then mu
 * added on the diagonal. */
int orc_column_gram(const orc_matrix *A, const int64_t *rows, int64_t s, double mu, double *G)
{
    const int64_t n = A->n;
    double *D = (double *)malloc((size_t)((s ? s : 1) * n) * sizeof(double));
    if (!D) return ORC_ERR_OOM;
    dense_rows(A, rows, s, D);
    for (int64_t c = 0; c < n; ++c)
        for (int64_t d = 0; d <= c; ++d) {
            double g = 0.0;
            for (int64_t a = 0; a < s; ++a) g = fma(D[a * n + c], D[a * n + d], g);
            if (c == d) g += mu;
            G[c * n + d] = g;
            G[d * n + c] = g;
        }
    free(D);
    return ORC_OK;
}

/* h = A_B^T v: h_c = sum over the rows a in the listed order of a_ac v_a (a
 * chain of fused multiply-adds from 0). */
static int column_sums(const orc_matrix *A, const int64_t *rows, int64_t s, const double *v, double *h)
{
    const int64_t n = A->n;
    double *D = (double *)malloc((size_t)((s ? s : 1) * n) * sizeof(double));
    if (!D) return ORC_ERR_OOM;
    dense_rows(A, rows, s, D);
    for (int64_t c = 0; c < n; ++c) {
        double g = 0.0;
        for (int64_t a = 0; a < s; ++a) g = fma(D[a * n + c], v[a], g);
        h[c] = g;
    }
    free(D);
    return ORC_OK;
}

/* V_t = (A_t^T A_t + mu I)^{-1} (n x n) for static block t: the column Gram,
 * its Cholesky factor, then the explicit inverse as for W_t. */
int orc_column_operator(const orc_matrix *A, const int64_t *off, int64_t t, double mu, double *V)
{
    const int64_t s = off[t + 1] - off[t], n = A->n;
    int64_t *rows = (int64_t *)malloc((size_t)(s ? s : 1) * sizeof(int64_t));
    double *G = (double *)malloc((size_t)(n * n) * sizeof(double));
    if (!rows || !G) { free(rows); free(G); return ORC_ERR_OOM; }
    for (int64_t a = 0; a < s; ++a) rows[a] = off[t] + a;
    int st = orc_column_gram(A, rows, s, mu, G);
    if (st == ORC_OK) st = orc_cholesky(G, n);
    if (st == ORC_OK) st = orc_spd_inverse(G, n, V);
    free(rows); free(G);
    return st;
}

/* x += V A_B^T (b_B - A_B x) with a stored V (n x n): r_B as in the s < n
 * form, g = A_B^T r_B (column sums above), y_c = sum over d ascending of
 * V_cd g_d (a chain from 0), then x_c += y_c for every column c. */
int orc_update_woodbury(const orc_matrix *A, const int64_t *rows, int64_t s, const double *V,
                        const double *b, double *x)
{
    const int64_t n = A->n;
    double *rB = (double *)malloc((size_t)(s ? s : 1) * sizeof(double));
    double *g = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    int st = (rB && g && y) ? ORC_OK : ORC_ERR_OOM;
    if (st == ORC_OK) {
        for (int64_t a = 0; a < s; ++a) rB[a] = b[rows[a]] - row_dot(A, rows[a], x);
        st = column_sums(A, rows, s, rB, g);
    }
    if (st == ORC_OK) {
        for (int64_t c = 0; c < n; ++c) {
            double acc = 0.0;
            for (int64_t d = 0; d < n; ++d) acc = fma(V[c * n + d], g[d], acc);
            y[c] = acc;
        }
        for (int64_t c = 0; c < n; ++c) x[c] += y[c];
    }
    free(rB); free(g); free(y);
    return st;
}

/* The dynamic block when K >= n: G = A_I^T A_I + mu I, L = chol(G),
 * h = A_I^T r_I, y = (L L^T)^{-1} h by the two triangular solves of
 * orc_chol_solve, then x_c += y_c for every column c. */
int orc_update_woodbury_cholesky(const orc_matrix *A, const int64_t *rows, int64_t K, double mu,
                                 const double *rI, double *x)
{
    const int64_t n = A->n;
    double *G = (double *)malloc((size_t)(n * n) * sizeof(double));
    double *h = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    int st = (G && h && y) ? ORC_OK : ORC_ERR_OOM;
    if (st == ORC_OK) st = orc_column_gram(A, rows, K, mu, G);
    if (st == ORC_OK) st = orc_cholesky(G, n);
    if (st == ORC_OK) st = column_sums(A, rows, K, rI, h);
    if (st == ORC_OK) {
        orc_chol_solve(G, n, h, y);
        for (int64_t c = 0; c < n; ++c) x[c] += y[c];
    }
    free(G); free(h); free(y);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, the whole solve.
 *   inputs : A, k blocks (uniform partition), mu, b, x0 (NULL -> 0), tol,
 *            maxit, seed, sysid, n_static (3 in the paper), start_iter (the
 *            counter offset of the first iteration, so a solve can resume).
 *   outputs: x, *iters, *rrn.
 *   traces (each may be NULL):
 *     tr_tau [maxit * n_static]  sampled blocks
 *     tr_rrn [maxit]             RRN after the static updates of iteration j
 *     tr_I   [maxit * K]         dynamic index sets (ascending)
 *     tr_x   [maxit * n]         x at the end of each iteration (after the
 *                                dynamic update; on the converging iteration,
 *                                x after the static updates)
 * Returns ORC_OK when converged, ORC_NOT_CONVERGED at maxit, or an error. */
/* ------------------------------------------------------------------------ */
/* Algorithm 2 (Appendix, initial solution): y = the sum of a set of rows of A
 * (here rows first .. first+count-1, each column summed over the rows in
 * ascending order), b~ = A y, x0 = (<b, b~> / ||b~||^2) y.  x0 lies in
 * range(A^T) and ||b - A x0|| <= ||b|| (the Remark after Algorithm 2).  The
 * two inner products are summed in index order.  Returns ORC_ERR_ARG for an
 * empty or out-of-range set or b~ = 0. */
int orc_initial_solution(const orc_matrix *A, int64_t first, int64_t count,
                         const double *b, double *x0)
{
    int64_t m = A->m, n = A->n;
    if (count < 1 || first < 0 || first + count > m) return ORC_ERR_ARG;
    double *bt = (double *)malloc((size_t)m * sizeof(double));
    double *zero = (double *)calloc((size_t)m, sizeof(double));
    if (!bt || !zero) { free(bt); free(zero); return ORC_ERR_OOM; }
    for (int64_t c = 0; c < n; ++c) x0[c] = 0.0;
    for (int64_t i = first; i < first + count; ++i) {
        if (A->is_dense) {
            const double *a = A->dense + i * A->ld;
            for (int64_t c = 0; c < n; ++c) x0[c] = x0[c] + a[c];
        } else {
            for (int64_t p = A->row_ptr[i]; p < A->row_ptr[i + 1]; ++p)
                x0[A->col_idx[p]] = x0[A->col_idx[p]] + A->val[p];
        }
    }
    orc_residual(A, zero, x0, bt);              /* bt = 0 - A y */
    double bb = 0.0, tt = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double v = -bt[i];                       /* b~ = A y */
        bb = fma(b[i], v, bb);
        tt = fma(v, v, tt);
    }
    free(bt); free(zero);
    if (!(tt > 0.0)) return ORC_ERR_ARG;
    double alpha = bb / tt;
    for (int64_t c = 0; c < n; ++c) x0[c] = alpha * x0[c];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The residual-weighted proposal (not in the paper: its P is static, Algorithm
 * 1's proposal).  Block t is drawn with weight w_t = Pbar_t * rho_t, where rho_t is
 * the squared norm of the residual on block t's rows: one fused chain over the
 * rows in ascending order.  The draws use the running sum of the weights,
 * cdf_t = w_0 + ... + w_t, summed in block order as P's running sum is. */
void orc_block_norms(const double *r, const int64_t *off, int64_t k, double *rho)
{
    for (int64_t t = 0; t < k; ++t) {
        double s = 0.0;
        for (int64_t i = off[t]; i < off[t + 1]; ++i) s = fma(r[i], r[i], s);
        rho[t] = s;
    }
}

/* Returns the total weight (cdf[k-1]). */
double orc_weighted_cdf(const double *Pbar, const double *rho, int64_t k, double *cdf)
{
    double s = 0.0;
    for (int64_t t = 0; t < k; ++t) {
        const double w = Pbar[t] * rho[t];
        s = s + w;
        cdf[t] = s;
    }
    return cdf[k - 1];
}

int orc_solve(const orc_matrix *A, int64_t k, double mu, const double *b,
              const double *x0, double *x, double tol, int64_t maxit,
              uint64_t seed, uint64_t sysid, int64_t n_static, int64_t start_iter,
              int dist_mode, const int64_t *force_tau,
              int64_t *iters, double *rrn_out,
              int64_t *tr_tau, double *tr_rrn, int64_t *tr_I, double *tr_x)
{
    int64_t m = A->m, n = A->n;
    if (k < 1 || k > m || n_static < 0) return ORC_ERR_ARG;
    int64_t K = m / k;
    int64_t *off = (int64_t *)malloc((size_t)(k + 1) * sizeof(int64_t));
    double *rs = (double *)malloc((size_t)k * sizeof(double));
    double *Pbar = (double *)malloc((size_t)k * sizeof(double));
    double *cdf = (double *)malloc((size_t)k * sizeof(double));
    double *r = (double *)malloc((size_t)m * sizeof(double));
    double *delta = (double *)calloc((size_t)n, sizeof(double));
    double **Wcache = (double **)calloc((size_t)k, sizeof(double *));
    int64_t *I = (int64_t *)malloc((size_t)(K ? K : 1) * sizeof(int64_t));
    double *rI = (double *)malloc((size_t)(K ? K : 1) * sizeof(double));
    int64_t smax = m / k + 1;
    int64_t *rows = (int64_t *)malloc((size_t)smax * sizeof(int64_t));
    double *work = (double *)malloc((size_t)(2 * smax) * sizeof(double));
    double *rho = (double *)malloc((size_t)k * sizeof(double));
    double *wcdf = (double *)malloc((size_t)k * sizeof(double));
    const double *dcdf = NULL;      /* the cdf the next draws use */
    int st = ORC_OK;
    if (!off || !rs || !Pbar || !cdf || !r || !delta || !Wcache || !I || !rI ||
        !rows || !work || !rho || !wcdf) { st = ORC_ERR_OOM; goto done; }
    if (dist_mode != 0 && dist_mode != 1) { st = ORC_ERR_ARG; goto done; }

    orc_partition(m, k, off);
    st = orc_orthogonality(A, k, off, NULL, rs);
    if (st != ORC_OK) goto done;
    orc_proposal(rs, k, n, Pbar, NULL, cdf);

    for (int64_t c = 0; c < n; ++c) x[c] = x0 ? x0[c] : 0.0;
    double bb = 0.0;
    for (int64_t i = 0; i < m; ++i) bb += b[i] * b[i];
    double bnorm = sqrt(bb);
    *iters = 0;
    *rrn_out = 0.0;
    if (bnorm == 0.0) {
        for (int64_t c = 0; c < n; ++c) x[c] = 0.0;
        st = ORC_OK;
        goto done;
    }
    st = ORC_NOT_CONVERGED;
    dcdf = cdf;
    if (dist_mode == 1) {               /* weights from r = b - A x0 */
        orc_residual(A, b, x, r);
        orc_block_norms(r, off, k, rho);
        if (orc_weighted_cdf(Pbar, rho, k, wcdf) > 0.0) dcdf = wcdf;
    }
    for (int64_t j = 0; j < maxit; ++j) {
        for (int64_t l = 0; l < n_static; ++l) {
            int64_t tau = force_tau && force_tau[j * n_static + l] >= 0
                              ? force_tau[j * n_static + l]
                              : orc_sample(dcdf, k, seed, sysid, start_iter + j, l);
            if (tau < 0 || tau >= k) { st = ORC_ERR_ARG; goto done; }
            if (tr_tau) tr_tau[j * n_static + l] = tau;
            int64_t s = off[tau + 1] - off[tau];
            const int wood = s >= n;        /* the n x n form (Lemma 1, Section 3.1) */
            if (!Wcache[tau]) {
                const int64_t sz = wood ? n * n : s * s;
                Wcache[tau] = (double *)malloc((size_t)(sz ? sz : 1) * sizeof(double));
                if (!Wcache[tau]) { st = ORC_ERR_OOM; goto done; }
                int e = wood ? orc_column_operator(A, off, tau, mu, Wcache[tau])
                             : orc_static_operator(A, off, tau, mu, Wcache[tau]);
                if (e != ORC_OK) { st = e; goto done; }
            }
            for (int64_t a = 0; a < s; ++a) rows[a] = off[tau] + a;
            if (wood) {
                int e = orc_update_woodbury(A, rows, s, Wcache[tau], b, x);
                if (e != ORC_OK) { st = e; goto done; }
            } else {
                orc_update_with_inverse(A, rows, s, Wcache[tau], b, x, delta, work);
            }
        }
        double rr = orc_residual(A, b, x, r);
        double rrn = sqrt(rr) / bnorm;
        if (dist_mode == 1) {           /* weights of the next iteration */
            orc_block_norms(r, off, k, rho);
            dcdf = orc_weighted_cdf(Pbar, rho, k, wcdf) > 0.0 ? wcdf : cdf;
        }
        if (tr_rrn) tr_rrn[j] = rrn;
        *iters = j + 1;
        *rrn_out = rrn;
        if (rrn <= tol) {
            if (tr_x) memcpy(tr_x + j * n, x, (size_t)n * sizeof(double));
            st = ORC_OK;
            break;
        }
        orc_topk(r, m, K, I);
        if (tr_I) memcpy(tr_I + j * K, I, (size_t)K * sizeof(int64_t));
        for (int64_t a = 0; a < K; ++a) rI[a] = r[I[a]];
        int e = K >= n ? orc_update_woodbury_cholesky(A, I, K, mu, rI, x)
                       : orc_update_with_cholesky(A, I, K, mu, rI, x, delta);
        if (e != ORC_OK) { st = e; break; }
        if (tr_x) memcpy(tr_x + j * n, x, (size_t)n * sizeof(double));
    }
done:
    if (Wcache) for (int64_t t = 0; t < k; ++t) free(Wcache[t]);
    free(Wcache); free(off); free(rs); free(Pbar); free(cdf); free(r); free(delta);
    free(I); free(rI); free(rows); free(work); free(rho); free(wcdf);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (Appendix): flexible AB-GMRES with ROR-BK as the right
 * preconditioner.  x = x0 (0 if NULL), r0 = b - A x, beta = ||r0||,
 * v_1 = r0 / beta.  Outer step j: z_j = ROR-BK on A z = v_j from z = 0 until
 * ||v_j - A z|| <= eta ||v_j|| or lmax iterations (the Philox counter runs on
 * across the inner solves); w = A z_j; modified Gram-Schmidt against
 * v_1..v_j (h_ij = <w, v_i>, w -= h_ij v_i); h_{j+1,j} = ||w||,
 * v_{j+1} = w / h_{j+1,j}; Givens rotations keep the least-squares problem
 * min ||beta e1 - H y|| triangular, and |g_{j+1}| is its residual norm.  Stops
 * when |g_{j+1}| <= tol ||b||, at breakdown (h_{j+1,j} = 0) or after maxit
 * outer steps; then y from the triangle, x += Z y.  Inner products and norms
 * are fused chains in index order.  Outputs: outer and inner iteration counts,
 * the final ||b - A x|| / ||b||, the residual estimate after each outer step. */
static double dotv(const double *a, const double *b, int64_t m)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s = fma(a[i], b[i], s);
    return s;
}

int orc_fabgmres(const orc_matrix *A, int64_t k, double mu, const double *b,
                 const double *x0, double *x, double tol, int64_t maxit, double eta,
                 int64_t lmax, uint64_t seed, uint64_t sysid, int64_t n_static,
                 int64_t *outer_out, int64_t *inner_out, double *rrn_out, double *est_hist)
{
    int64_t m = A->m, n = A->n;
    if (maxit < 1 || lmax < 0 || !(eta >= 0) || !(tol >= 0)) return ORC_ERR_ARG;
    double *V = (double *)malloc((size_t)(maxit + 1) * m * sizeof(double));
    double *Z = (double *)malloc((size_t)maxit * n * sizeof(double));
    double *H = (double *)calloc((size_t)(maxit + 1) * maxit, sizeof(double));
    double *cs = (double *)malloc((size_t)maxit * sizeof(double));
    double *sn = (double *)malloc((size_t)maxit * sizeof(double));
    double *g = (double *)calloc((size_t)(maxit + 1), sizeof(double));
    double *y = (double *)malloc((size_t)maxit * sizeof(double));
    double *w = (double *)malloc((size_t)m * sizeof(double));
    double *zero = (double *)calloc((size_t)m, sizeof(double));
    int st = ORC_OK;
    if (!V || !Z || !H || !cs || !sn || !g || !y || !w || !zero) { st = ORC_ERR_OOM; goto done; }
    for (int64_t c = 0; c < n; ++c) x[c] = x0 ? x0[c] : 0.0;
    double bnorm = sqrt(dotv(b, b, m));
    *outer_out = 0; *inner_out = 0; *rrn_out = 0.0;
    if (bnorm == 0.0) { for (int64_t c = 0; c < n; ++c) x[c] = 0.0; goto done; }
    double beta = sqrt(orc_residual(A, b, x, w));
    if (beta == 0.0) goto done;
    for (int64_t i = 0; i < m; ++i) V[i] = w[i] / beta;
    g[0] = beta;
    int64_t J = 0, inner = 0;
    for (int64_t j = 0; j < maxit; ++j) {
        double *vj = V + j * m, *zj = Z + j * n;
        int64_t it = 0;
        double rr = 0.0;
        int e = orc_solve(A, k, mu, vj, NULL, zj, eta, lmax, seed, sysid, n_static, inner, 0, NULL,
                          &it, &rr, NULL, NULL, NULL, NULL);
        if (e < 0) { st = e; goto done; }
        inner += it;
        orc_residual(A, zero, zj, w);            /* w = -A z_j */
        for (int64_t i = 0; i < m; ++i) w[i] = -w[i];
        for (int64_t i = 0; i <= j; ++i) {
            const double *vi = V + i * m;
            double h = dotv(w, vi, m);
            H[i * maxit + j] = h;
            for (int64_t t = 0; t < m; ++t) w[t] = fma(-h, vi[t], w[t]);
        }
        double hn = sqrt(dotv(w, w, m));
        H[(j + 1) * maxit + j] = hn;
        if (hn > 0.0) for (int64_t t = 0; t < m; ++t) V[(j + 1) * m + t] = w[t] / hn;
        for (int64_t i = 0; i < j; ++i) {        /* earlier rotations on column j */
            double a0 = H[i * maxit + j], a1 = H[(i + 1) * maxit + j];
            H[i * maxit + j] = cs[i] * a0 + sn[i] * a1;
            H[(i + 1) * maxit + j] = -sn[i] * a0 + cs[i] * a1;
        }
        double a0 = H[j * maxit + j], a1 = H[(j + 1) * maxit + j];
        double d = sqrt(a0 * a0 + a1 * a1);
        cs[j] = a0 / d; sn[j] = a1 / d;
        H[j * maxit + j] = d; H[(j + 1) * maxit + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        J = j + 1;
        double est = fabs(g[j + 1]) / bnorm;
        if (est_hist) est_hist[j] = est;
        if (est <= tol || hn == 0.0) break;
    }
    for (int64_t i = J - 1; i >= 0; --i) {       /* R y = g */
        double s = g[i];
        for (int64_t l = i + 1; l < J; ++l) s = fma(-H[i * maxit + l], y[l], s);
        y[i] = s / H[i * maxit + i];
    }
    for (int64_t c = 0; c < n; ++c) {
        double u = 0.0;
        for (int64_t j = 0; j < J; ++j) u = fma(y[j], Z[j * n + c], u);
        x[c] = x[c] + u;
    }
    *outer_out = J;
    *inner_out = inner;
    *rrn_out = sqrt(orc_residual(A, b, x, w)) / bnorm;
    st = *rrn_out <= tol ? ORC_OK : ORC_NOT_CONVERGED;
done:
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(w); free(zero);
    return st;
}
