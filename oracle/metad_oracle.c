/*
 * FP64 CPU oracle for the per-step metadynamics bias path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA implementation.
 *
 * What it computes (GPU-MetaD, Methods "Metadynamics Method"):
 *   U_b = U_0 + V_b                                              (Eq. 1)
 *   V_b(s) = sum_tau V_b(s; s_tau, tau)                          (Eq. 2)
 *   V_b(s; s_tau, tau) = w_k exp(-(s - s_tau)^2 / (2 sigma^2))   (Eq. 3)
 * with the CVs s named in the paper's large-scale GaN runs (coordination
 * number, Section "B4-B1 phase transition in Large-scale systems") plus a
 * locally averaged Steinhardt Q6, the well-tempered height rule (named in
 * Section "Water dissociation on rutile (110) surface" and Fig. 3, formula
 * not printed), and bias forces F = -dV_b/dr obtained, as in the paper's
 * autograd (Section "Frameworks of GPU-MetaD"), by reverse-mode
 * differentiation, here written out by hand.
 *
 * Readings where the paper is silent (switch, CN mask, Q6 weights and
 * averaging, the well-tempered rule, the Hermite grid) are stated at each
 * function.  Everything is plain IEEE double, compiled -ffp-contract=off;
 * the per-atom loops are OpenMP-parallel but every sum over atoms or hills
 * runs serially in index order, so the result does not depend on the thread
 * count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_L 6
#define ORC_NM (2 * ORC_L + 1)
#define ORC_MAXCV 5 /* CN, Q6 and the three lattice parameters */

typedef struct {
    double box[3];
    double rc;
    double r0;
    int32_t sw_n;
    int32_t sw_m;
    int32_t stretch;        /* 1: shift/scale the switch to vanish at rc */
    int32_t cn_unlike_only; /* 1: CN counts unlike-species pairs only */
    int32_t n_cv;           /* 1: CN; 2: CN and averaged Q6 */
    int32_t pad;
} orc_params;

typedef struct {
    int32_t n[2];
    int32_t pad[2];
    double lo[2];
    double hi[2];
    double *data; /* [n0][n1][4]: V, dV/ds0, dV/ds1, d2V/ds0ds1 */
} orc_grid;

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ geometry
 * Minimum-image displacement d = x_j - x_i (FP64), one shift of +-L when
 * |d| > L/2.  Valid for coordinates wrapped into [0, L). */
static double mi(double d, double L)
{
    if (d > 0.5 * L)
        d -= L;
    else if (d < -0.5 * L)
        d += L;
    return d;
}

static void disp(const float *pos4, const double *box, int64_t i, int64_t j, double d[3])
{
    for (int a = 0; a < 3; ++a)
        d[a] = mi((double)pos4[4 * j + a] - (double)pos4[4 * i + a], box[a]);
}

/* r^2 = (dx*dx + dy*dy) + dz*dz, in this order, no fused multiply-add. */
static double r2_of(const double d[3])
{
    double s = d[0] * d[0] + d[1] * d[1];
    return s + d[2] * d[2];
}

/* ------------------------------------------------------------- neighbours
 * Pair set: unordered {i, j}, i != j, with r^2 < rc^2 (strict), rc^2 = rc*rc.
 * Output: pairs (i, j), i < j, ascending lexicographic order.  Returns the
 * pair count, or -(count) - 1 when cap is too small (nothing written past
 * cap). */
int64_t orc_pairs_brute(int32_t n, const float *pos4, const double *box, double rc,
                        int64_t *pairs, int64_t cap)
{
    double rc2 = rc * rc;
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double d[3];
            disp(pos4, box, i, j, d);
            if (r2_of(d) < rc2) {
                if (np < cap) {
                    pairs[2 * np] = i;
                    pairs[2 * np + 1] = j;
                }
                ++np;
            }
        }
    return np <= cap ? np : -np - 1;
}

typedef struct {
    int nc[3];
    int32_t *start; /* [ncell+1] */
    int32_t *atoms; /* [n] atom ids grouped by cell, ascending within a cell */
} cells_t;

static int cell_of(double x, double L, int nc)
{
    int c = (int)floor(x / L * nc);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

static int build_cells(int32_t n, const float *pos4, const double *box, double rc, cells_t *c)
{
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        int k = (int)floor(box[a] / rc);
        c->nc[a] = k < 1 ? 1 : k;
        ncell *= c->nc[a];
    }
    c->start = (int32_t *)calloc((size_t)ncell + 1, sizeof(int32_t));
    c->atoms = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!c->start || !c->atoms || !cid) {
        free(c->start); free(c->atoms); free(cid);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        int cx = cell_of(pos4[4 * i + 0], box[0], c->nc[0]);
        int cy = cell_of(pos4[4 * i + 1], box[1], c->nc[1]);
        int cz = cell_of(pos4[4 * i + 2], box[2], c->nc[2]);
        cid[i] = (int32_t)(((int64_t)cz * c->nc[1] + cy) * c->nc[0] + cx);
        c->start[cid[i] + 1]++;
    }
    for (int64_t k = 0; k < ncell; ++k) c->start[k + 1] += c->start[k];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    if (!fill) { free(c->start); free(c->atoms); free(cid); return -1; }
    memcpy(fill, c->start, sizeof(int32_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) c->atoms[fill[cid[i]]++] = (int32_t)i;
    free(fill);
    free(cid);
    return 0;
}

/* distinct cell offsets along one axis (fewer than 3 cells: no repeats) */
static int axis_offsets(int nc, int *off)
{
    if (nc >= 3) { off[0] = -1; off[1] = 0; off[2] = 1; return 3; }
    if (nc == 2) { off[0] = 0; off[1] = 1; return 2; }
    off[0] = 0;
    return 1;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Same pair set as orc_pairs_brute, found through a cell list (cell edge >=
 * rc, all 27 surrounding cells, each distinct cell once). */
int64_t orc_pairs_cells(int32_t n, const float *pos4, const double *box, double rc,
                        int64_t *pairs, int64_t cap, int nthreads)
{
    set_threads(nthreads);
    cells_t c;
    if (build_cells(n, pos4, box, rc, &c) != 0) return -1;
    double rc2 = rc * rc;
    int ox[3], oy[3], oz[3];
    int sx = axis_offsets(c.nc[0], ox), sy = axis_offsets(c.nc[1], oy), sz = axis_offsets(c.nc[2], oz);
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t **rows = (int32_t **)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t *));
    if (!cnt || !rows) { free(cnt); free(rows); free(c.start); free(c.atoms); return -1; }
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int cx = cell_of(pos4[4 * i + 0], box[0], c.nc[0]);
        int cy = cell_of(pos4[4 * i + 1], box[1], c.nc[1]);
        int cz = cell_of(pos4[4 * i + 2], box[2], c.nc[2]);
        int32_t buf_cap = 64, nb = 0;
        int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)buf_cap);
        for (int a = 0; a < sz; ++a)
            for (int b = 0; b < sy; ++b)
                for (int e = 0; e < sx; ++e) {
                    int zz = (cz + oz[a] + c.nc[2]) % c.nc[2];
                    int yy = (cy + oy[b] + c.nc[1]) % c.nc[1];
                    int xx = (cx + ox[e] + c.nc[0]) % c.nc[0];
                    int64_t k = ((int64_t)zz * c.nc[1] + yy) * c.nc[0] + xx;
                    for (int32_t t = c.start[k]; t < c.start[k + 1]; ++t) {
                        int64_t j = c.atoms[t];
                        if (j <= i) continue;
                        double d[3];
                        disp(pos4, box, i, j, d);
                        if (r2_of(d) < rc2) {
                            if (nb == buf_cap) {
                                buf_cap *= 2;
                                int32_t *nbuf = (int32_t *)realloc(buf, sizeof(int32_t) * (size_t)buf_cap);
                                if (!nbuf) { failed = 1; continue; }
                                buf = nbuf;
                            }
                            buf[nb++] = (int32_t)j;
                        }
                    }
                }
        qsort(buf, (size_t)nb, sizeof(int32_t), cmp_i32);
        rows[i] = buf;
        cnt[i + 1] = nb;
    }
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t t = 0; t < cnt[i + 1]; ++t) {
            if (np < cap) {
                pairs[2 * np] = i;
                pairs[2 * np + 1] = rows[i][t];
            }
            ++np;
        }
        free(rows[i]);
    }
    free(rows); free(cnt); free(c.start); free(c.atoms);
    if (failed) return -1;
    return np <= cap ? np : -np - 1;
}

/* ------------------------------------------------------------------ switch
 * Rational switch x = r/r0, s_raw = (1 - x^n)/(1 - x^m); near x = 1 the
 * first-order expansion (n/m)(1 + (n-m)(x-1)/2) replaces the 0/0.  With
 * stretch, s = (s_raw(r) - s_raw(rc)) / (1 - s_raw(rc)) for r < rc, else 0.
 * ds gets d s / d r. */
static void sw_raw(double r, double r0, int n, int m, double *f, double *df)
{
    double x = r / r0;
    if (fabs(x - 1.0) < 1e-6) {
        double e = x - 1.0;
        *f = ((double)n / m) * (1.0 + 0.5 * (n - m) * e);
        *df = ((double)n * (n - m) / (2.0 * m)) / r0;
        return;
    }
    double xn = pow(x, n), xm = pow(x, m);
    double num = 1.0 - xn, den = 1.0 - xm;
    *f = num / den;
    double dnum = -n * pow(x, n - 1), dden = -m * pow(x, m - 1);
    *df = ((dnum * den - num * dden) / (den * den)) / r0;
}

static void switch_fn(const orc_params *p, double r, double *s, double *ds)
{
    if (!(r < p->rc)) { *s = 0.0; *ds = 0.0; return; }
    double f, df;
    sw_raw(r, p->r0, p->sw_n, p->sw_m, &f, &df);
    if (p->stretch) {
        double fc, dfc;
        sw_raw(p->rc, p->r0, p->sw_n, p->sw_m, &fc, &dfc);
        *s = (f - fc) / (1.0 - fc);
        *ds = df / (1.0 - fc);
    } else {
        *s = f;
        *ds = df;
    }
}

void orc_switch(const orc_params *p, int32_t n, const double *r, double *s, double *ds)
{
    for (int32_t k = 0; k < n; ++k) switch_fn(p, r[k], &s[k], &ds[k]);
}

/* ------------------------------------------------------- spherical harmonics
 * Complex Y_l^m with the Condon-Shortley phase:
 *   Y_l^m(rhat) = K_lm P_l^m(cos theta) e^{i m phi},
 *   K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
 *   P_l^m(t) = (-1)^m (1-t^2)^{m/2} d^m P_l/dt^m,
 * written pole-free with t = z/r and u = (x+iy)/r = sin(theta) e^{i phi}:
 *   Y_l^m = K_lm (-1)^m [d^m P_l/dt^m](t) u^m   (m >= 0),
 *   Y_l^{-m} = (-1)^m conj(Y_l^m).
 * P_l comes from its explicit sum 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) t^(l-2k). */
static double fact(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

static double binom(int a, int b)
{
    return fact(a) / (fact(b) * fact(a - b));
}

typedef struct {
    double dcoef[ORC_L + 2][ORC_L + 1]; /* dcoef[k][p]: coefficient of t^p in d^k P_l/dt^k */
    double K[ORC_L + 1];
} ylm_tab;

static void ylm_init(ylm_tab *T)
{
    const int l = ORC_L;
    memset(T, 0, sizeof(*T));
    for (int k = 0; 2 * k <= l; ++k)
        T->dcoef[0][l - 2 * k] = ((k % 2) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l) / pow(2.0, l);
    for (int d = 1; d <= l + 1; ++d)
        for (int p = 0; p < l; ++p) T->dcoef[d][p] = T->dcoef[d - 1][p + 1] * (p + 1);
    for (int m = 0; m <= l; ++m)
        T->K[m] = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - m) / fact(l + m));
}

static double poly(const double *c, int deg, double t)
{
    double v = 0.0;
    for (int p = deg; p >= 0; --p) v = v * t + c[p];
    return v;
}

/* Y[mi] for m = mi - l, and (if g != NULL) g[mi][a] = dY/dd_a for the
 * unnormalised vector d. */
static void ylm_eval(const ylm_tab *T, const double d[3], double complex Y[ORC_NM],
                     double complex g[ORC_NM][3])
{
    const int l = ORC_L;
    double r = sqrt(r2_of(d));
    double uh[3] = {d[0] / r, d[1] / r, d[2] / r};
    double t = uh[2];
    double complex u = (d[0] + I * d[1]) / r;
    double complex upow[ORC_L + 1];
    upow[0] = 1.0;
    for (int m = 1; m <= l; ++m) upow[m] = upow[m - 1] * u;
    double dt[3], complex_dummy = 0.0;
    (void)complex_dummy;
    double complex du[3];
    for (int a = 0; a < 3; ++a) {
        dt[a] = ((a == 2 ? 1.0 : 0.0) - t * uh[a]) / r;
        du[a] = ((a == 0 ? 1.0 : 0.0) + (a == 1 ? I : 0.0) - u * uh[a]) / r;
    }
    for (int m = 0; m <= l; ++m) {
        double sgn = (m % 2) ? -1.0 : 1.0;
        double Pm = poly(T->dcoef[m], l - m, t);
        double Pm1 = (m < l) ? poly(T->dcoef[m + 1], l - m - 1, t) : 0.0;
        double complex y = T->K[m] * sgn * Pm * upow[m];
        Y[l + m] = y;
        if (m > 0) Y[l - m] = sgn * conj(y);
        if (g) {
            for (int a = 0; a < 3; ++a) {
                double complex gy = T->K[m] * sgn * (Pm1 * upow[m] * dt[a]);
                if (m > 0) gy += T->K[m] * sgn * (Pm * m * upow[m - 1] * du[a]);
                g[l + m][a] = gy;
                if (m > 0) g[l - m][a] = sgn * conj(gy);
            }
        }
    }
}

void orc_ylm(int32_t n, const double *dvec, double *Yre, double *Yim, double *gre, double *gim)
{
    ylm_tab T;
    ylm_init(&T);
    for (int32_t k = 0; k < n; ++k) {
        double complex Y[ORC_NM], g[ORC_NM][3];
        ylm_eval(&T, dvec + 3 * k, Y, g);
        for (int mi = 0; mi < ORC_NM; ++mi) {
            Yre[ORC_NM * k + mi] = creal(Y[mi]);
            Yim[ORC_NM * k + mi] = cimag(Y[mi]);
            if (gre)
                for (int a = 0; a < 3; ++a) {
                    gre[(ORC_NM * k + mi) * 3 + a] = creal(g[mi][a]);
                    gim[(ORC_NM * k + mi) * 3 + a] = cimag(g[mi][a]);
                }
        }
    }
}

/* ---------------------------------------------------------- neighbour rows
 * Symmetric adjacency (CSR) from the sorted pair list: row i lists every j
 * with {i, j} a pair, ascending. */
typedef struct {
    int32_t n;
    int64_t *off;
    int32_t *idx;
} adj_t;

static int adj_build(int32_t n, const int64_t *pairs, int64_t np, adj_t *A)
{
    A->n = n;
    A->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    A->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * np > 0 ? 2 * np : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!A->off || !A->idx || !fill) { free(A->off); free(A->idx); free(fill); return -1; }
    for (int64_t p = 0; p < np; ++p) { A->off[pairs[2 * p] + 1]++; A->off[pairs[2 * p + 1] + 1]++; }
    for (int64_t i = 0; i < n; ++i) A->off[i + 1] += A->off[i];
    memcpy(fill, A->off, sizeof(int64_t) * (size_t)n);
    for (int64_t p = 0; p < np; ++p) {
        int64_t i = pairs[2 * p], j = pairs[2 * p + 1];
        A->idx[fill[i]++] = (int32_t)j;
        A->idx[fill[j]++] = (int32_t)i;
    }
    free(fill);
    return 0;
}

static void adj_free(adj_t *A) { free(A->off); free(A->idx); }

static int make_adj(int32_t n, const float *pos4, const orc_params *p, adj_t *A, int nthreads)
{
    int64_t cap = (int64_t)n * 32 + 64;
    for (;;) {
        int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)cap);
        if (!pairs) return -1;
        int64_t np = orc_pairs_cells(n, pos4, p->box, p->rc, pairs, cap, nthreads);
        if (np < -1) { free(pairs); cap = -np - 1; continue; }
        if (np == -1) { free(pairs); return -1; }
        int rc = adj_build(n, pairs, np, A);
        free(pairs);
        return rc;
    }
}

/* ------------------------------------------------------------------ CVs
 * CN_i    = sum_{j in N(i)} s(r_ij) [unlike species, or all pairs]
 * s1      = (1/N) sum_i CN_i
 * w_ij    = s(r_ij)  (all species);  W_i = sum_j w_ij
 * q_m(i)  = sum_j w_ij Y_6^m(rhat_ij) / W_i   (0 when W_i = 0)
 * qb_m(i) = (q_m(i) + sum_j w_ij q_m(j)) / (1 + W_i)
 * qb6(i)  = sqrt(4 pi / 13 sum_m |qb_m(i)|^2)
 * s2      = (1/N) sum_i qb6(i)
 * State kept for the reverse pass lives in cvstate. */
typedef struct {
    int32_t n;
    adj_t A;
    double *w;          /* per directed entry */
    double *cn, *W, *qb6;
    double complex *q;  /* [n][13] */
    double complex *qb; /* [n][13] */
    double s[2];
} cvstate;

static void cv_free(cvstate *S)
{
    adj_free(&S->A);
    free(S->w); free(S->cn); free(S->W); free(S->qb6); free(S->q); free(S->qb);
}

static int cv_forward(int32_t n, const float *pos4, const orc_params *p, cvstate *S, int nthreads)
{
    memset(S, 0, sizeof(*S));
    S->n = n;
    set_threads(nthreads);
    if (make_adj(n, pos4, p, &S->A, nthreads) != 0) return -1;
    int64_t ne = S->A.off[n];
    S->w = (double *)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1));
    S->cn = (double *)calloc((size_t)n + 1, sizeof(double));
    S->W = (double *)calloc((size_t)n + 1, sizeof(double));
    S->qb6 = (double *)calloc((size_t)n + 1, sizeof(double));
    int q6 = p->n_cv >= 2;
    if (q6) {
        S->q = (double complex *)calloc((size_t)n * ORC_NM + 1, sizeof(double complex));
        S->qb = (double complex *)calloc((size_t)n * ORC_NM + 1, sizeof(double complex));
    }
    if (!S->w || !S->cn || !S->W || !S->qb6 || (q6 && (!S->q || !S->qb))) return -1;
    ylm_tab T;
    ylm_init(&T);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double cn = 0.0, W = 0.0;
        double complex Q[ORC_NM];
        for (int mi = 0; mi < ORC_NM; ++mi) Q[mi] = 0.0;
        for (int64_t e = S->A.off[i]; e < S->A.off[i + 1]; ++e) {
            int64_t j = S->A.idx[e];
            double d[3], s, ds;
            disp(pos4, p->box, i, j, d);
            switch_fn(p, sqrt(r2_of(d)), &s, &ds);
            S->w[e] = s;
            int unlike = pos4[4 * i + 3] != pos4[4 * j + 3];
            if (!p->cn_unlike_only || unlike) cn += s;
            W += s;
            if (q6) {
                double complex Y[ORC_NM];
                ylm_eval(&T, d, Y, NULL);
                for (int mi = 0; mi < ORC_NM; ++mi) Q[mi] += s * Y[mi];
            }
        }
        S->cn[i] = cn;
        S->W[i] = W;
        if (q6)
            for (int mi = 0; mi < ORC_NM; ++mi) S->q[i * ORC_NM + mi] = W > 0.0 ? Q[mi] / W : 0.0;
    }
    if (q6) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double complex A[ORC_NM];
            for (int mi = 0; mi < ORC_NM; ++mi) A[mi] = S->q[i * ORC_NM + mi];
            for (int64_t e = S->A.off[i]; e < S->A.off[i + 1]; ++e) {
                int64_t j = S->A.idx[e];
                for (int mi = 0; mi < ORC_NM; ++mi) A[mi] += S->w[e] * S->q[j * ORC_NM + mi];
            }
            double sq = 0.0;
            for (int mi = 0; mi < ORC_NM; ++mi) {
                S->qb[i * ORC_NM + mi] = A[mi] / (1.0 + S->W[i]);
                double complex z = S->qb[i * ORC_NM + mi];
                sq += creal(z) * creal(z) + cimag(z) * cimag(z);
            }
            S->qb6[i] = sqrt(4.0 * M_PI / 13.0 * sq);
        }
    }
    double a = 0.0, b = 0.0;
    for (int64_t i = 0; i < n; ++i) { a += S->cn[i]; b += S->qb6[i]; }
    S->s[0] = n > 0 ? a / n : 0.0;
    S->s[1] = n > 0 ? b / n : 0.0;
    return 0;
}

/* CVs of one frame; cn/qb6 (per atom, may be NULL) and s[n_cv]. */
int orc_cv(int32_t n, const float *pos4, const orc_params *p, double *s, double *cn, double *qb6, int nthreads)
{
    cvstate S;
    if (cv_forward(n, pos4, p, &S, nthreads) != 0) { cv_free(&S); return -1; }
    s[0] = S.s[0];
    if (p->n_cv >= 2) s[1] = S.s[1];
    if (cn) memcpy(cn, S.cn, sizeof(double) * (size_t)n);
    if (qb6) memcpy(qb6, S.qb6, sizeof(double) * (size_t)n);
    cv_free(&S);
    return 0;
}

/* ------------------------------------------------------------------ forces
 * F = -sum_d (dV/ds_d) ds_d/dr by reverse-mode differentiation of the CV
 * forward pass above, each step the adjoint of one forward line, taken in
 * reverse order.  Complex adjoints carry (dL/dRe, dL/dIm) as re + i im. */
static int cv_reverse(const float *pos4, const orc_params *p, const cvstate *S, const double *dVds,
                      double *F, double *vir)
{
    const int32_t n = S->n;
    const int q6 = p->n_cv >= 2;
    const double s1bar = dVds[0];
    const double s2bar = q6 ? dVds[1] : 0.0;
    double *Wbar = (double *)calloc((size_t)n + 1, sizeof(double));
    double complex *Abar = NULL, *Qbar = NULL;
    if (q6) {
        Abar = (double complex *)calloc((size_t)n * ORC_NM + 1, sizeof(double complex));
        Qbar = (double complex *)calloc((size_t)n * ORC_NM + 1, sizeof(double complex));
    }
    if (!Wbar || (q6 && (!Abar || !Qbar))) { free(Wbar); free(Abar); free(Qbar); return -1; }
    if (q6) {
        /* s2 = (1/N) sum qb6 ; qb6 = sqrt(4pi/13 sum |qb|^2) ; qb = A / (1 + W) */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double qb6bar = s2bar / n;
            double D = 1.0 + S->W[i], Dbar = 0.0;
            for (int mi = 0; mi < ORC_NM; ++mi) {
                double complex qb = S->qb[i * ORC_NM + mi];
                double complex qbbar = S->qb6[i] > 0.0 ? qb6bar * (4.0 * M_PI / 13.0) * qb / S->qb6[i] : 0.0;
                double complex abar = qbbar / D;
                Abar[i * ORC_NM + mi] = abar;
                Dbar -= creal(conj(abar) * qb);
            }
            Wbar[i] = Dbar;
        }
        /* A_m(i) = q_m(i) + sum_j w_ij q_m(j)  ->  qbar; q = Q / W -> Qbar, Wbar */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double complex qbar[ORC_NM];
            for (int mi = 0; mi < ORC_NM; ++mi) qbar[mi] = Abar[i * ORC_NM + mi];
            for (int64_t e = S->A.off[i]; e < S->A.off[i + 1]; ++e) {
                int64_t k = S->A.idx[e];
                for (int mi = 0; mi < ORC_NM; ++mi) qbar[mi] += S->w[e] * Abar[k * ORC_NM + mi];
            }
            double W = S->W[i];
            double wb = 0.0;
            for (int mi = 0; mi < ORC_NM; ++mi) {
                Qbar[i * ORC_NM + mi] = W > 0.0 ? qbar[mi] / W : 0.0;
                if (W > 0.0) wb -= creal(conj(qbar[mi]) * S->q[i * ORC_NM + mi]) / W;
            }
            Wbar[i] += wb;
        }
    }
    ylm_tab T;
    ylm_init(&T);
    /* per-atom shares of the virial sum_{directed entries} (dL/dd)_c d_c, added
     * in atom order afterwards */
    double *vi = vir ? (double *)calloc(3 * (size_t)n + 1, sizeof(double)) : NULL;
    if (vir && !vi) { free(Wbar); free(Abar); free(Qbar); return -1; }
    /* adjoint of one directed entry i -> j (d = r_j - r_i), returned as dL/dd */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double g[3] = {0.0, 0.0, 0.0};
        for (int64_t e = S->A.off[i]; e < S->A.off[i + 1]; ++e) {
            int64_t j = S->A.idx[e];
            for (int side = 0; side < 2; ++side) {
                /* side 0: entry i -> j ; side 1: entry j -> i (its d is -d_ij) */
                int64_t a = side == 0 ? i : j, b = side == 0 ? j : i;
                double d[3], s, ds;
                disp(pos4, p->box, a, b, d);
                double r = sqrt(r2_of(d));
                switch_fn(p, r, &s, &ds);
                int unlike = pos4[4 * a + 3] != pos4[4 * b + 3];
                double wbar = 0.0;
                if (!p->cn_unlike_only || unlike) wbar += s1bar / n;
                double dd[3] = {0.0, 0.0, 0.0};
                if (q6) {
                    wbar += Wbar[a];
                    double complex Y[ORC_NM], gy[ORC_NM][3];
                    ylm_eval(&T, d, Y, gy);
                    for (int mi = 0; mi < ORC_NM; ++mi) {
                        double complex Qb = Qbar[a * ORC_NM + mi];
                        wbar += creal(conj(Qb) * Y[mi]);
                        wbar += creal(conj(Abar[a * ORC_NM + mi]) * S->q[b * ORC_NM + mi]);
                        double complex ybar = s * Qb;
                        for (int c = 0; c < 3; ++c) dd[c] += creal(conj(ybar) * gy[mi][c]);
                    }
                }
                for (int c = 0; c < 3; ++c) dd[c] += wbar * ds * d[c] / r;
                /* d = r_b - r_a : dL/dr_a = -dd, dL/dr_b = +dd; keep atom i's share */
                for (int c = 0; c < 3; ++c) g[c] += (side == 0 ? -dd[c] : dd[c]);
                /* every directed entry is side 0 exactly once (from its own row) */
                if (vi && side == 0)
                    for (int c = 0; c < 3; ++c) vi[3 * i + c] += dd[c] * d[c];
            }
        }
        for (int c = 0; c < 3; ++c) F[3 * i + c] = -g[c];
    }
    if (vir) {
        vir[0] = vir[1] = vir[2] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) vir[c] += vi[3 * i + c];
        free(vi);
    }
    free(Wbar); free(Abar); free(Qbar);
    return 0;
}

/* Bias forces for given dV/ds; also returns s (and per-atom cn/qb6 if set). */
int orc_forces(int32_t n, const float *pos4, const orc_params *p, const double *dVds, double *F,
               double *s, int nthreads)
{
    cvstate S;
    if (cv_forward(n, pos4, p, &S, nthreads) != 0) { cv_free(&S); return -1; }
    if (s) { s[0] = S.s[0]; if (p->n_cv >= 2) s[1] = S.s[1]; }
    int rc = cv_reverse(pos4, p, &S, dVds, F, NULL);
    cv_free(&S);
    return rc;
}

/* -------------------------------------------------------------------- grid
 * Bicubic Hermite patch on a uniform node grid over [lo, hi] (n nodes per
 * axis, both ends included).  Nodes hold V, dV/dx, dV/dy, d2V/dxdy.  Outside
 * [lo, hi] in either axis the grid contributes nothing. */
static void hermite_basis(double t, double A[2], double B[2], double dA[2], double dB[2])
{
    double t2 = t * t, t3 = t2 * t;
    A[0] = 2.0 * t3 - 3.0 * t2 + 1.0;
    A[1] = -2.0 * t3 + 3.0 * t2;
    B[0] = t3 - 2.0 * t2 + t;
    B[1] = t3 - t2;
    dA[0] = 6.0 * t2 - 6.0 * t;
    dA[1] = -6.0 * t2 + 6.0 * t;
    dB[0] = 3.0 * t2 - 4.0 * t + 1.0;
    dB[1] = 3.0 * t2 - 2.0 * t;
}

static void grid_eval(const orc_grid *G, const double *s, double *V, double *dV)
{
    *V = 0.0; dV[0] = 0.0; dV[1] = 0.0;
    if (!G || !G->data) return;
    double h[2], t[2];
    int c[2];
    for (int a = 0; a < 2; ++a) {
        if (!(s[a] >= G->lo[a] && s[a] <= G->hi[a])) return;
        h[a] = (G->hi[a] - G->lo[a]) / (G->n[a] - 1);
        int k = (int)floor((s[a] - G->lo[a]) / h[a]);
        if (k > G->n[a] - 2) k = G->n[a] - 2;
        if (k < 0) k = 0;
        c[a] = k;
        t[a] = (s[a] - (G->lo[a] + k * h[a])) / h[a];
    }
    double Ax[2], Bx[2], dAx[2], dBx[2], Ay[2], By[2], dAy[2], dBy[2];
    hermite_basis(t[0], Ax, Bx, dAx, dBx);
    hermite_basis(t[1], Ay, By, dAy, dBy);
    double v = 0.0, gx = 0.0, gy = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double *nd = G->data + ((int64_t)(c[0] + a) * G->n[1] + (c[1] + b)) * 4;
            v += Ax[a] * Ay[b] * nd[0] + h[0] * Bx[a] * Ay[b] * nd[1] + h[1] * Ax[a] * By[b] * nd[2] +
                 h[0] * h[1] * Bx[a] * By[b] * nd[3];
            gx += (dAx[a] * Ay[b] * nd[0] + h[0] * dBx[a] * Ay[b] * nd[1] + h[1] * dAx[a] * By[b] * nd[2] +
                   h[0] * h[1] * dBx[a] * By[b] * nd[3]) / h[0];
            gy += (Ax[a] * dAy[b] * nd[0] + h[0] * Bx[a] * dAy[b] * nd[1] + h[1] * Ax[a] * dBy[b] * nd[2] +
                   h[0] * h[1] * Bx[a] * dBy[b] * nd[3]) / h[1];
        }
    *V = v; dV[0] = gx; dV[1] = gy;
}

/* Add hills to every node: exact Gaussian sums and analytic derivatives. */
int orc_grid_fold(orc_grid *G, int32_t K, const double *c, const double *w, const double *sigma, int nthreads)
{
    set_threads(nthreads);
    double h0 = (G->hi[0] - G->lo[0]) / (G->n[0] - 1), h1 = (G->hi[1] - G->lo[1]) / (G->n[1] - 1);
    double v0 = sigma[0] * sigma[0], v1 = sigma[1] * sigma[1];
#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < (int64_t)G->n[0] * G->n[1]; ++node) {
        int64_t a = node / G->n[1], b = node % G->n[1];
        double x = G->lo[0] + a * h0, y = G->lo[1] + b * h1;
        double *nd = G->data + node * 4;
        for (int32_t k = 0; k < K; ++k) {
            double dx = x - c[2 * k], dy = y - c[2 * k + 1];
            double g = w[k] * exp(-(dx * dx / (2.0 * v0) + dy * dy / (2.0 * v1)));
            nd[0] += g;
            nd[1] += g * (-dx / v0);
            nd[2] += g * (-dy / v1);
            nd[3] += g * (dx * dy / (v0 * v1));
        }
    }
    return 0;
}

/* -------------------------------------------------------------------- bias
 * V(s) = grid(s) + sum_k w_k exp(-sum_d (s_d - c_kd)^2 / (2 sigma_d^2))
 * dV/ds_d = grid' + sum_k w_k g_k (-(s_d - c_kd) / sigma_d^2)
 * (Eqs. 2-3 with a per-dimension sigma; hills in deposition order).
 * period (NULL, or double[ncv] with 0 for a non-periodic CV): a periodic CV
 * such as a torsion angle (Section "Alanine dipeptide torsion") sees the
 * difference s_d - c_kd wrapped into [-P/2, P/2], nearest image only
 * (reading: x - P * round-half-even(x / P)). */
static double hill_diff(double x, const double *period, int d)
{
    if (period && period[d] > 0.0) x -= period[d] * nearbyint(x / period[d]);
    return x;
}

int orc_bias(int32_t ncv, const double *s, int32_t K, const double *c, const double *w, const double *sigma,
             const double *period, const orc_grid *G, double *V, double *dV)
{
    double v = 0.0, g[ORC_MAXCV] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (G && G->data && ncv == 2) grid_eval(G, s, &v, g);
    for (int32_t k = 0; k < K; ++k) {
        double e = 0.0;
        for (int d = 0; d < ncv; ++d) {
            double x = hill_diff(s[d] - c[(int64_t)ncv * k + d], period, d);
            e += x * x / (2.0 * sigma[d] * sigma[d]);
        }
        double gk = w[k] * exp(-e);
        v += gk;
        for (int d = 0; d < ncv; ++d)
            g[d] += gk * (-hill_diff(s[d] - c[(int64_t)ncv * k + d], period, d) / (sigma[d] * sigma[d]));
    }
    *V = v;
    for (int d = 0; d < ncv; ++d) dV[d] = g[d];
    return 0;
}

/* Well-tempered heights, deposited in order (reading of the rule the paper
 * names but does not print):
 *   w_k = w0 exp(-V_{k-1}(c_k) / (kB * T * (gamma - 1)))
 * where V_{k-1} is the grid plus hills 0..k-1.  Hills 0..k_first-1 already
 * carry heights in w; hills k_first..K-1 get theirs here. */
int orc_deposit_sequence(int32_t ncv, int32_t K, int32_t k_first, const double *c, double *w,
                         const double *sigma, const double *period, double w0, double kbdt, const orc_grid *G)
{
    for (int32_t k = k_first; k < K; ++k) {
        double V, dV[ORC_MAXCV];
        orc_bias(ncv, c + (int64_t)ncv * k, k, c, w, sigma, period, G, &V, dV);
        w[k] = w0 * exp(-V / kbdt);
    }
    return 0;
}

/* ---------------------------------------------------------------- one step
 * Neighbours, CVs, bias, forces for one frame. */
int orc_step(int32_t n, const float *pos4, const orc_params *p, int32_t K, const double *c, const double *w,
             const double *sigma, const orc_grid *G, double *s, double *V, double *dV, double *F, int nthreads)
{
    cvstate S;
    if (cv_forward(n, pos4, p, &S, nthreads) != 0) { cv_free(&S); return -1; }
    s[0] = S.s[0];
    if (p->n_cv >= 2) s[1] = S.s[1];
    orc_bias(p->n_cv, S.s, K, c, w, sigma, NULL, G, V, dV);
    int rc = cv_reverse(pos4, p, &S, dV, F, NULL);
    cv_free(&S);
    return rc;
}

/* ------------------------------------------------------ lattice parameters
 * The GaN runs bias the coordination number together with the triaxial
 * lattice parameters under NPT (Section "B4-B1 phase transition in
 * Large-scale systems").  With lattice = 1 the CVs are
 *     s = (s1 [, s2], L_x, L_y, L_z)   (D = n_cv + 3 dimensions)
 * and hills are D-dimensional.  A barostat needs the derivative of the bias
 * with respect to each box length at fixed fractional coordinates (positions
 * scale with the box):
 *     dV/dL_a = dV/ds_{L_a} [lattice] + (1/L_a) sum_pairs (dV/dd_ij)_a (d_ij)_a
 * since every per-atom CV depends on the positions only through the pair
 * displacements d_ij, and d_ij,a = L_a (f_j - f_i - n_ij)_a under scaling.
 * The pair sum (the bias virial) is accumulated by the reverse pass.
 * box_grad receives dV/dL (the explicit term only with lattice = 1). */
int orc_step_box(int32_t n, const float *pos4, const orc_params *p, int32_t lattice, int32_t K, const double *c,
                 const double *w, const double *sigma, double *s, double *V, double *dV, double *F,
                 double *box_grad, int nthreads)
{
    cvstate S;
    if (cv_forward(n, pos4, p, &S, nthreads) != 0) { cv_free(&S); return -1; }
    const int D = p->n_cv + (lattice ? 3 : 0);
    double sv[ORC_MAXCV];
    for (int d = 0; d < p->n_cv; ++d) sv[d] = S.s[d];
    if (lattice)
        for (int a = 0; a < 3; ++a) sv[p->n_cv + a] = p->box[a];
    for (int d = 0; d < D; ++d) s[d] = sv[d];
    orc_bias(D, sv, K, c, w, sigma, NULL, NULL, V, dV);
    double vir[3];
    int rc = cv_reverse(pos4, p, &S, dV, F, vir);
    cv_free(&S);
    for (int a = 0; a < 3; ++a) box_grad[a] = (lattice ? dV[p->n_cv + a] : 0.0) + vir[a] / p->box[a];
    return rc;
}
