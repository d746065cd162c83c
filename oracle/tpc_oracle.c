/*
 * CPU oracle of the per-sector TPC tracker: Cellular-Automaton seeding and
 * simplified-Kalman-filter track following (Sec. 2, steps 1 and 2; Table 1
 * rows 1-2; Fig. 1 c,d).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no source with
 * the CUDA path.  It is plain, single-threaded per (event, sector) unit, and
 * brute force wherever the tracker uses a search structure: every neighbour
 * and every hit search scans the whole pad row.
 *
 * The same source is compiled twice:
 *   ORACLE_REAL=double  the accuracy reference (FP64);
 *   ORACLE_REAL=float   FP32_EXACT: the same expressions in binary32, in the
 *                       order written here, built with -ffp-contract=off so
 *                       no multiply-add is fused.
 *
 * The paper names the steps but fixes none of the constants, windows, the
 * link criterion, the filter equations or the selection rule; every such
 * choice below is a stated reading (the readings table of the design notes):
 *   N1-N5 neighbour finding, S1 start hits, T1-T8 tracklet construction,
 *   Sel1-Sel2 tracklet selection.
 *
 * Parity status per function (what pins it, in tests/test_oracle_*.py):
 *   propagate      closed-form helix of the generator (exact to 1e-10 cm)
 *   transport      finite differences of propagate (Bz = 0: exact derivative)
 *   update         Bayesian posterior in information form (numpy.linalg)
 *   fit (P2 pass)  noise-free helices: fixed point = truth within 1e-9;
 *                  Bz = 0: z-block equals weighted least squares, the
 *                  y-block's fixed point is the least-squares line;
 *                  chi2/ndf ~ 1
 *   neighbours     hand-built cases (collinear triple, exact tie, cuts) and
 *                  links == generator truth on isolated tracks
 *   cleaner        symmetry invariant + a hand-built asymmetric case
 *   start hits     one start per chain, chains disjoint, length >= 3
 *   selection      hand-built overlap cases, single-ownership invariant
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

#define RC(c) ((real)(c))
#define ORC_IS_FLOAT (sizeof(real) == sizeof(float))

static inline real r_sqrt(real v) { return ORC_IS_FLOAT ? (real)sqrtf((float)v) : (real)sqrt((double)v); }
static inline real r_fabs(real v) { return ORC_IS_FLOAT ? (real)fabsf((float)v) : (real)fabs((double)v); }
static inline real r_copysign(real v, real s)
{
    return ORC_IS_FLOAT ? (real)copysignf((float)v, (float)s) : (real)copysign((double)v, (double)s);
}

#define ORC_KAPPA 0.00299792458 /* curvature [1/cm] per (T * c/GeV) */

/* All tunable constants of the readings, in double; FP32_EXACT rounds each to
 * float once, where it is used. */
typedef struct {
    double k_win;      /* N2: window half-width per cm of row distance        */
    double d_max2;     /* N3: cut on the collinearity residual D (cm^2)       */
    double n_sigma;    /* T5: search window in units of sqrt(S)               */
    double w_min;      /* T5: window clamp (cm)                               */
    double w_max;
    double s_max;      /* propagation fails if |sin phi| exceeds this         */
    double y_margin;   /* T6: stop if |y| > X tan(half opening) + margin      */
    double sigma_y;    /* T1/T2: cluster errors (cm)                          */
    double sigma_z;
    double var_s;      /* T1: initial variances of sin phi, q/pT, tan lambda  */
    double var_q;
    double var_t;
    int g_max;         /* T6: stop after more than g_max consecutive misses   */
    int l_seed;        /* S1: minimum chain length                            */
    int n_min_tracklet;/* T8 */
    int n_min_track;   /* Sel2 */
    int own_num;       /* Sel2: owned * own_den >= own_num * nhits            */
    int own_den;
} orc_params;

typedef struct {
    int n_rows;
    int n_sectors;       /* per event; sector < n_sectors/2 is side A         */
    const float* row_x;  /* [n_rows] pad-row plane positions (cm)             */
    float tan_half_open; /* tan of the sector half-opening angle              */
    float z_max;         /* drift length (cm)                                 */
} orc_geom;

void orc_params_default(orc_params* p)
{
    p->k_win = 1.5;
    p->d_max2 = 0.25;
    p->n_sigma = 3.5;
    p->w_min = 0.3;
    p->w_max = 3.0;
    p->s_max = 0.95;
    p->y_margin = 2.0;
    p->sigma_y = 0.1;
    p->sigma_z = 0.1;
    p->var_s = 0.25;
    p->var_q = 100.0;
    p->var_t = 1.0;
    p->g_max = 8;
    p->l_seed = 3;
    p->n_min_tracklet = 10;
    p->n_min_track = 10;
    p->own_num = 7;
    p->own_den = 10;
}

int orc_real_size(void) { return (int)sizeof(real); }

/* ------------------------------------------------------------------------ */
/* Track state and the simplified Kalman filter (T2, T3)                    */
/* ------------------------------------------------------------------------ */

/* State at the plane x: y, z, s = sin(phi), t = tan(lambda), q = q/pT.
 * Two uncorrelated blocks (Sec. 2 step 2: uncorrelated coordinate errors):
 *   Y = (y, s, q) with covariance cy = {c00, c10, c11, c20, c21, c22}
 *   Z = (z, t)    with covariance cz = {c00, c10, c11}.                    */
typedef struct {
    real x, y, z, s, t, q;
    real cy[6];
    real cz[3];
} orc_state;

/* Exact helix step x -> x1 in constant Bz; kB = -kappa * Bz.
 *   s1 = s + k d, k = kB q, d = x1 - x
 *   dy = d (s + s1) / (c + c1), c = sqrt(1 - s^2)
 *   chord L = sign(d) sqrt(d^2 + dy^2), u = k L / 2   (signed: a step
 *   towards smaller x runs backwards along the track)
 *   arc = L (1 + u^2 / 6 + 3 u^4 / 40)   (2 asin(u) / k to order u^4)
 *   dz = t * arc
 * Covariance transport with the Jacobian (cross-block terms dropped):
 *   dy1/ds = d (1/c^3 + 1/c1^3) / 2, dy1/dq = kB d^2 / (2 c1^3),
 *   ds1/dq = kB d, dz1/dt = arc.
 * Returns 0 (state untouched) when |s| or |s1| exceeds s_max.              */
static int orc_prop(orc_state* st, real x1, real kB, real s_max)
{
    real d = x1 - st->x;
    real k = kB * st->q;
    real s0 = st->s;
    real s1 = s0 + k * d;
    if (r_fabs(s0) > s_max || r_fabs(s1) > s_max) return 0;
    real c0 = r_sqrt(RC(1) - s0 * s0);
    real c1 = r_sqrt(RC(1) - s1 * s1);
    real dy = d * (s0 + s1) / (c0 + c1);
    real L = r_copysign(r_sqrt(d * d + dy * dy), d);
    real u = k * L * RC(0.5);
    real u2 = u * u;
    real arc = L * (RC(1) + u2 * (RC(1.0 / 6.0) + u2 * RC(3.0 / 40.0)));
    real dz = st->t * arc;

    real ci3 = RC(1) / (c0 * c0 * c0);
    real c1i3 = RC(1) / (c1 * c1 * c1);
    real a = d * (ci3 + c1i3) * RC(0.5);
    real b = kB * d * d * RC(0.5) * c1i3;
    real e = kB * d;

    /* C' = F C F^T for F = [[1, a, b], [0, 1, e], [0, 0, 1]] */
    real c00 = st->cy[0], c10 = st->cy[1], c11 = st->cy[2];
    real c20 = st->cy[3], c21 = st->cy[4], c22 = st->cy[5];
    real r00 = c00 + a * c10 + b * c20;  /* (F C) row 0 */
    real r01 = c10 + a * c11 + b * c21;
    real r02 = c20 + a * c21 + b * c22;
    real r10 = c10 + e * c20;            /* (F C) row 1 */
    real r11 = c11 + e * c21;
    real r12 = c21 + e * c22;
    st->cy[0] = r00 + a * r01 + b * r02;
    st->cy[1] = r10 + a * r11 + b * r12;
    st->cy[2] = r11 + e * r12;
    st->cy[3] = c20 + a * c21 + b * c22;
    st->cy[4] = c21 + e * c22;
    st->cy[5] = c22;

    /* Z block: F = [[1, arc], [0, 1]] */
    real z00 = st->cz[0], z10 = st->cz[1], z11 = st->cz[2];
    real q00 = z00 + arc * z10;
    real q01 = z10 + arc * z11;
    st->cz[0] = q00 + arc * q01;
    st->cz[1] = q01;
    st->cz[2] = z11;

    st->x = x1;
    st->y = st->y + dy;
    st->z = st->z + dz;
    st->s = s1;
    return 1;
}

/* Measurement update with cluster (my, mz); H picks y (resp. z). */
static void orc_update(orc_state* st, real my, real mz, real sy2, real sz2, real* chi2)
{
    real S = sy2 + st->cy[0];
    real r = my - st->y;
    real K0 = st->cy[0] / S, K1 = st->cy[1] / S, K2 = st->cy[3] / S;
    real c00 = st->cy[0], c10 = st->cy[1], c11 = st->cy[2];
    real c20 = st->cy[3], c21 = st->cy[4], c22 = st->cy[5];
    st->y = st->y + K0 * r;
    st->s = st->s + K1 * r;
    st->q = st->q + K2 * r;
    st->cy[0] = c00 - K0 * c00;
    st->cy[1] = c10 - K1 * c00;
    st->cy[2] = c11 - K1 * c10;
    st->cy[3] = c20 - K2 * c00;
    st->cy[4] = c21 - K2 * c10;
    st->cy[5] = c22 - K2 * c20;
    real chi = r * r / S;

    real Sz = sz2 + st->cz[0];
    real rz = mz - st->z;
    real L0 = st->cz[0] / Sz, L1 = st->cz[1] / Sz;
    real z00 = st->cz[0], z10 = st->cz[1], z11 = st->cz[2];
    st->z = st->z + L0 * rz;
    st->t = st->t + L1 * rz;
    st->cz[0] = z00 - L0 * z00;
    st->cz[1] = z10 - L1 * z00;
    st->cz[2] = z11 - L1 * z10;
    *chi2 = *chi2 + chi + rz * rz / Sz;
}

static void orc_reset_cov(orc_state* st, real sy2, real sz2, real var_s, real var_q, real var_t)
{
    st->cy[0] = sy2; st->cy[1] = RC(0); st->cy[2] = var_s;
    st->cy[3] = RC(0); st->cy[4] = RC(0); st->cy[5] = var_q;
    st->cz[0] = sz2; st->cz[1] = RC(0); st->cz[2] = var_t;
}

/* ------------------------------------------------------------------------ */
/* Per-(event, sector) unit                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* constants in working precision */
    real k_win, d_max2, n_sigma, w_min, w_max, s_max, y_margin;
    real sy2, sz2, var_s, var_q, var_t, kB, tan_h, z_max;
    int g_max, l_seed, n_min_tracklet, n_min_track, own_num, own_den;
    int n_rows;
    const float* row_x;
} orc_ctx;

static void orc_ctx_init(orc_ctx* c, const orc_params* p, const orc_geom* g, double bz)
{
    c->k_win = RC(p->k_win);
    c->d_max2 = RC(p->d_max2);
    c->n_sigma = RC(p->n_sigma);
    c->w_min = RC(p->w_min);
    c->w_max = RC(p->w_max);
    c->s_max = RC(p->s_max);
    c->y_margin = RC(p->y_margin);
    real sy = RC(p->sigma_y), sz = RC(p->sigma_z);
    c->sy2 = sy * sy;
    c->sz2 = sz * sz;
    c->var_s = RC(p->var_s);
    c->var_q = RC(p->var_q);
    c->var_t = RC(p->var_t);
    c->kB = RC(-ORC_KAPPA * bz);
    c->tan_h = RC(g->tan_half_open);
    c->z_max = RC(g->z_max);
    c->g_max = p->g_max;
    c->l_seed = p->l_seed;
    c->n_min_tracklet = p->n_min_tracklet;
    c->n_min_track = p->n_min_track;
    c->own_num = p->own_num;
    c->own_den = p->own_den;
    c->n_rows = g->n_rows;
    c->row_x = g->row_x;
}

#define ORC_NTF 16 /* floats per tracklet record: x y z s t q cy[6] cz[3] chi2 */

typedef struct {
    /* inputs (unit-local views) */
    int n;                 /* clusters in the unit                              */
    int base;              /* global index of the unit's first cluster          */
    const int32_t* rcount; /* [n_rows]                                          */
    int* rstart;           /* [n_rows + 1] unit-local row offsets               */
    real* y;
    real* z;
    uint32_t* id;
    int* row;              /* row of each unit-local cluster                    */
    /* outputs */
    int n_start;
    int* start;            /* unit-local cluster index, canonical order         */
    double* tl_f;          /* [n_start][ORC_NTF]                                */
    int* tl_n;             /* P2 hit count                                      */
    int* tl_alive;
    int* tl_hits;          /* [n_start][n_rows], unit-local, rows ascending     */
    int n_tracks;
    int* trk_t;            /* unit-local tracklet index                         */
    int* trk_n;            /* owned hits                                        */
    int* trk_hits;         /* [n_tracks][n_rows] owned hits, rows ascending     */
} orc_unit;

typedef struct { uint32_t id; int idx; } orc_idpair;
static int orc_cmp_idpair(const void* a, const void* b)
{
    const orc_idpair* x = (const orc_idpair*)a;
    const orc_idpair* y = (const orc_idpair*)b;
    return (x->id > y->id) - (x->id < y->id);
}

/* N1-N3: for every hit on rows 1..n_rows-2 the best (up, down) pair.       */
static void orc_neighbours(const orc_ctx* c, const orc_unit* u, int* up, int* dn)
{
    for (int i = 0; i < u->n; i++) { up[i] = -1; dn[i] = -1; }
    int maxrow = 0;
    for (int r = 0; r < c->n_rows; r++) if (u->rcount[r] > maxrow) maxrow = u->rcount[r];
    int* cu = (int*)malloc(sizeof(int) * (size_t)(maxrow + 1));
    int* cd = (int*)malloc(sizeof(int) * (size_t)(maxrow + 1));
    for (int r = 1; r + 1 < c->n_rows; r++) {
        real Xr = RC(c->row_x[r]), Xu = RC(c->row_x[r + 1]), Xd = RC(c->row_x[r - 1]);
        real Ru = Xu / Xr, Rd = Xd / Xr;
        real Wu = c->k_win * r_fabs(Xu - Xr);
        real Wd = c->k_win * r_fabs(Xd - Xr);
        real tt = (Xr - Xd) / (Xu - Xd);
        for (int i = u->rstart[r]; i < u->rstart[r + 1]; i++) {
            real yi = u->y[i], zi = u->z[i];
            real ycu = yi * Ru, ycd = yi * Rd;
            int nu = 0, nd = 0;
            for (int j = u->rstart[r + 1]; j < u->rstart[r + 2]; j++)
                if (r_fabs(u->y[j] - ycu) <= Wu && r_fabs(u->z[j] - zi) <= Wu) cu[nu++] = j;
            for (int j = u->rstart[r - 1]; j < u->rstart[r]; j++)
                if (r_fabs(u->y[j] - ycd) <= Wd && r_fabs(u->z[j] - zi) <= Wd) cd[nd++] = j;
            int bu = -1, bd = -1;
            real bD = RC(0);
            for (int a = 0; a < nu; a++) {
                int ju = cu[a];
                for (int b = 0; b < nd; b++) {
                    int jd = cd[b];
                    real yp = u->y[jd] + (u->y[ju] - u->y[jd]) * tt;
                    real zp = u->z[jd] + (u->z[ju] - u->z[jd]) * tt;
                    real ey = yi - yp;
                    real ez = zi - zp;
                    real D = ey * ey + ez * ez;
                    if (!(D <= c->d_max2)) continue;
                    int better;
                    if (bu < 0) better = 1;
                    else if (D < bD) better = 1;
                    else if (D > bD) better = 0;
                    else if (u->id[ju] != u->id[bu]) better = u->id[ju] < u->id[bu];
                    else better = u->id[jd] < u->id[bd];
                    if (better) { bu = ju; bd = jd; bD = D; }
                }
            }
            up[i] = bu;
            dn[i] = bd;
        }
    }
    free(cu);
    free(cd);
}

/* N4: keep i -> j only if j links back to i, from the pre-clean snapshot.  */
static void orc_clean(const orc_unit* u, const int* up, const int* dn, int* up2, int* dn2)
{
    for (int i = 0; i < u->n; i++) {
        up2[i] = (up[i] >= 0 && dn[up[i]] == i) ? up[i] : -1;
        dn2[i] = (dn[i] >= 0 && up[dn[i]] == i) ? dn[i] : -1;
    }
}

/* S1: start hits in canonical order (row, then cluster id).                */
static void orc_start_hits(const orc_ctx* c, orc_unit* u, const int* up2, const int* dn2)
{
    u->start = (int*)malloc(sizeof(int) * (size_t)(u->n + 1));
    u->n_start = 0;
    orc_idpair* tmp = (orc_idpair*)malloc(sizeof(orc_idpair) * (size_t)(u->n + 1));
    for (int r = 0; r < c->n_rows; r++) {
        int m = 0;
        for (int i = u->rstart[r]; i < u->rstart[r + 1]; i++) {
            if (up2[i] < 0 || dn2[i] >= 0) continue;
            int len = 1, j = i;
            while (up2[j] >= 0) { j = up2[j]; len++; }
            if (len < c->l_seed) continue;
            tmp[m].id = u->id[i];
            tmp[m].idx = i;
            m++;
        }
        qsort(tmp, (size_t)m, sizeof(orc_idpair), orc_cmp_idpair);
        for (int k = 0; k < m; k++) u->start[u->n_start++] = tmp[k].idx;
    }
    free(tmp);
}

/* T5: closest cluster on row r to the predicted state, in the window.      */
static int orc_search(const orc_ctx* c, const orc_unit* u, const orc_state* st, int r)
{
    real Sy = c->sy2 + st->cy[0];
    real Sz = c->sz2 + st->cz[0];
    real wy = c->n_sigma * r_sqrt(Sy);
    real wz = c->n_sigma * r_sqrt(Sz);
    wy = wy < c->w_min ? c->w_min : (wy > c->w_max ? c->w_max : wy);
    wz = wz < c->w_min ? c->w_min : (wz > c->w_max ? c->w_max : wz);
    int best = -1;
    real bd2 = RC(0);
    for (int j = u->rstart[r]; j < u->rstart[r + 1]; j++) {
        real dy = u->y[j] - st->y;
        real dz = u->z[j] - st->z;
        if (!(r_fabs(dy) <= wy && r_fabs(dz) <= wz)) continue;
        real d2 = dy * dy / Sy + dz * dz / Sz;
        if (best < 0 || d2 < bd2 || (d2 == bd2 && u->id[j] < u->id[best])) { best = j; bd2 = d2; }
    }
    return best;
}

/* T6 stop rule on a predicted state at row r (besides propagation failure). */
static int orc_outside(const orc_ctx* c, const orc_state* st, int r)
{
    real X = RC(c->row_x[r]);
    return r_fabs(st->y) > X * c->tan_h + c->y_margin || r_fabs(st->z) > c->z_max;
}

static void orc_store(const orc_state* st, real chi2, double* f)
{
    f[0] = (double)st->x; f[1] = (double)st->y; f[2] = (double)st->z;
    f[3] = (double)st->s; f[4] = (double)st->t; f[5] = (double)st->q;
    for (int k = 0; k < 6; k++) f[6 + k] = (double)st->cy[k];
    for (int k = 0; k < 3; k++) f[12 + k] = (double)st->cz[k];
    f[15] = (double)chi2;
}

/* T1, T6, T7, T8: one tracklet from start hit h0.                          */
static void orc_tracklet(const orc_ctx* c, const orc_unit* u, const int* up2, int h0,
                         double* f, int* n_out, int* alive, int* hits)
{
    int hL = h0;
    while (up2[hL] >= 0) hL = up2[hL];
    real X0 = RC(c->row_x[u->row[h0]]);
    real XL = RC(c->row_x[u->row[hL]]);
    orc_state st;
    st.x = X0;
    st.y = u->y[h0];
    st.z = u->z[h0];
    real dx = XL - X0, dy = u->y[hL] - u->y[h0], dz = u->z[hL] - u->z[h0];
    real l = r_sqrt(dx * dx + dy * dy);
    st.s = dy / l;
    st.t = dz / l;
    st.q = RC(0);
    orc_reset_cov(&st, c->sy2, c->sz2, c->var_s, c->var_q, c->var_t);
    real chi2 = RC(0);

    /* Phase 1: the chain, then outward row by row.  Every row step predicts
     * on a copy of the state (T5); the state itself moves only when a cluster
     * is filtered, so after a miss the next prediction starts again from the
     * last filtered cluster. */
    int have = 0, stopped = 0, r_out = -1;
    orc_state pr;
    for (int h = h0; h >= 0; h = up2[h]) {
        int r = u->row[h];
        pr = st;
        if (!orc_prop(&pr, RC(c->row_x[r]), c->kB, c->s_max) || orc_outside(c, &pr, r)) {
            stopped = 1;
            break;
        }
        orc_update(&pr, u->y[h], u->z[h], c->sy2, c->sz2, &chi2);
        st = pr;
        r_out = r;
        have = 1;
    }
    if (!stopped) {
        int miss = 0;
        for (int r = u->row[hL] + 1; r < c->n_rows; r++) {
            pr = st;
            if (!orc_prop(&pr, RC(c->row_x[r]), c->kB, c->s_max) || orc_outside(c, &pr, r)) break;
            int j = orc_search(c, u, &pr, r);
            if (j >= 0) {
                orc_update(&pr, u->y[j], u->z[j], c->sy2, c->sz2, &chi2);
                st = pr;
                r_out = r;
                miss = 0;
            } else if (++miss > c->g_max) {
                break;
            }
        }
    }
    *n_out = 0;
    *alive = 0;
    for (int k = 0; k < ORC_NTF; k++) f[k] = 0.0;
    if (!have) return;

    /* Phase 2: fresh covariance, inward from P1's outermost cluster (where
     * the state now is) to row 0. */
    orc_reset_cov(&st, c->sy2, c->sz2, c->var_s, c->var_q, c->var_t);
    chi2 = RC(0);
    int n = 0, miss = 0;
    for (int r = r_out; r >= 0; r--) {
        pr = st;
        if (!orc_prop(&pr, RC(c->row_x[r]), c->kB, c->s_max) || orc_outside(c, &pr, r)) break;
        int j = orc_search(c, u, &pr, r);
        if (j >= 0) {
            orc_update(&pr, u->y[j], u->z[j], c->sy2, c->sz2, &chi2);
            st = pr;
            hits[n++] = j; /* rows descending for now */
            miss = 0;
        } else if (++miss > c->g_max) {
            break;
        }
    }
    *n_out = n;
    for (int a = 0, b = n - 1; a < b; a++, b--) { int x = hits[a]; hits[a] = hits[b]; hits[b] = x; }
    if (n > 0) orc_store(&st, chi2, f); /* the state at the innermost cluster */
    *alive = n >= c->n_min_tracklet;
}

/* Sel1, Sel2: best instance per hit, then acceptance.                      */
static void orc_select(const orc_ctx* c, orc_unit* u)
{
    uint64_t* owner = (uint64_t*)calloc((size_t)u->n + 1, sizeof(uint64_t));
    for (int t = 0; t < u->n_start; t++) {
        if (!u->tl_alive[t]) continue;
        uint64_t key = ((uint64_t)(uint32_t)u->tl_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
        for (int k = 0; k < u->tl_n[t]; k++) {
            int h = u->tl_hits[(size_t)t * (size_t)c->n_rows + (size_t)k];
            if (key > owner[h]) owner[h] = key;
        }
    }
    u->trk_t = (int*)malloc(sizeof(int) * (size_t)(u->n_start + 1));
    u->trk_n = (int*)malloc(sizeof(int) * (size_t)(u->n_start + 1));
    u->trk_hits = (int*)malloc(sizeof(int) * ((size_t)u->n_start * (size_t)c->n_rows + 1));
    u->n_tracks = 0;
    for (int t = 0; t < u->n_start; t++) {
        if (!u->tl_alive[t]) continue;
        uint64_t key = ((uint64_t)(uint32_t)u->tl_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
        int m = 0;
        int* dst = u->trk_hits + (size_t)u->n_tracks * (size_t)c->n_rows;
        for (int k = 0; k < u->tl_n[t]; k++) {
            int h = u->tl_hits[(size_t)t * (size_t)c->n_rows + (size_t)k];
            if (owner[h] == key) dst[m++] = h;
        }
        if (m >= c->n_min_track && (int64_t)m * c->own_den >= (int64_t)c->own_num * u->tl_n[t]) {
            u->trk_t[u->n_tracks] = t;
            u->trk_n[u->n_tracks] = m;
            u->n_tracks++;
        }
    }
    free(owner);
}

/* ------------------------------------------------------------------------ */
/* Batch driver: (event, sector) units are independent (Sec. 3.1)           */
/* ------------------------------------------------------------------------ */

typedef struct orc_result {
    int n_units, n_rows;
    int64_t n_clusters;
    int32_t *up_raw, *dn_raw, *up, *dn; /* global cluster indices, [N]       */
    orc_unit* units;
    int64_t* unit_base;                  /* [n_units]                         */
    int64_t* unit_t0;                    /* first global tracklet id          */
    int64_t* unit_m0;                    /* first global track index          */
    int64_t n_tracklets, n_tracklet_hits, n_tracks, n_track_hits;
    double seconds;
} orc_result;

static double orc_now(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return 0.0;
#endif
}

orc_result* orc_run(const orc_params* p, const orc_geom* g, double bz, int n_events,
                    const float* clusters, const int32_t* row_counts, int n_threads)
{
    orc_ctx c;
    orc_ctx_init(&c, p, g, bz);
    orc_result* res = (orc_result*)calloc(1, sizeof(orc_result));
    int n_units = n_events * g->n_sectors;
    res->n_units = n_units;
    res->n_rows = g->n_rows;
    res->units = (orc_unit*)calloc((size_t)n_units + 1, sizeof(orc_unit));
    res->unit_base = (int64_t*)calloc((size_t)n_units + 1, sizeof(int64_t));
    res->unit_t0 = (int64_t*)calloc((size_t)n_units + 1, sizeof(int64_t));
    res->unit_m0 = (int64_t*)calloc((size_t)n_units + 1, sizeof(int64_t));
    int64_t N = 0;
    for (int un = 0; un < n_units; un++) {
        res->unit_base[un] = N;
        for (int r = 0; r < g->n_rows; r++) N += row_counts[(size_t)un * g->n_rows + r];
    }
    res->unit_base[n_units] = N;
    res->n_clusters = N;
    size_t nn = (size_t)N + 1;
    res->up_raw = (int32_t*)malloc(sizeof(int32_t) * nn);
    res->dn_raw = (int32_t*)malloc(sizeof(int32_t) * nn);
    res->up = (int32_t*)malloc(sizeof(int32_t) * nn);
    res->dn = (int32_t*)malloc(sizeof(int32_t) * nn);

    double t0 = orc_now();
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int un = 0; un < n_units; un++) {
        orc_unit* u = &res->units[un];
        int64_t base = res->unit_base[un];
        int n = (int)(res->unit_base[un + 1] - base);
        u->n = n;
        u->base = (int)base;
        u->rcount = row_counts + (size_t)un * g->n_rows;
        u->rstart = (int*)malloc(sizeof(int) * (size_t)(g->n_rows + 2));
        u->rstart[0] = 0;
        for (int r = 0; r < g->n_rows; r++) u->rstart[r + 1] = u->rstart[r] + u->rcount[r];
        u->rstart[g->n_rows + 1] = u->rstart[g->n_rows];
        u->y = (real*)malloc(sizeof(real) * (size_t)(n + 1));
        u->z = (real*)malloc(sizeof(real) * (size_t)(n + 1));
        u->id = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
        u->row = (int*)malloc(sizeof(int) * (size_t)(n + 1));
        for (int r = 0; r < g->n_rows; r++)
            for (int i = u->rstart[r]; i < u->rstart[r + 1]; i++) u->row[i] = r;
        for (int i = 0; i < n; i++) {
            const float* cl = clusters + (size_t)(base + i) * 4;
            u->y[i] = RC(cl[1]);
            u->z[i] = RC(cl[2]);
            memcpy(&u->id[i], &cl[3], 4);
        }
        int* up = (int*)malloc(sizeof(int) * (size_t)(n + 1));
        int* dn = (int*)malloc(sizeof(int) * (size_t)(n + 1));
        int* up2 = (int*)malloc(sizeof(int) * (size_t)(n + 1));
        int* dn2 = (int*)malloc(sizeof(int) * (size_t)(n + 1));
        orc_neighbours(&c, u, up, dn);
        orc_clean(u, up, dn, up2, dn2);
        for (int i = 0; i < n; i++) {
            res->up_raw[base + i] = up[i] >= 0 ? (int32_t)(base + up[i]) : -1;
            res->dn_raw[base + i] = dn[i] >= 0 ? (int32_t)(base + dn[i]) : -1;
            res->up[base + i] = up2[i] >= 0 ? (int32_t)(base + up2[i]) : -1;
            res->dn[base + i] = dn2[i] >= 0 ? (int32_t)(base + dn2[i]) : -1;
        }
        orc_start_hits(&c, u, up2, dn2);
        int T = u->n_start;
        u->tl_f = (double*)calloc((size_t)T * ORC_NTF + 1, sizeof(double));
        u->tl_n = (int*)calloc((size_t)T + 1, sizeof(int));
        u->tl_alive = (int*)calloc((size_t)T + 1, sizeof(int));
        u->tl_hits = (int*)malloc(sizeof(int) * ((size_t)T * (size_t)g->n_rows + 1));
        for (int t = 0; t < T; t++)
            orc_tracklet(&c, u, up2, u->start[t], u->tl_f + (size_t)t * ORC_NTF, &u->tl_n[t],
                         &u->tl_alive[t], u->tl_hits + (size_t)t * (size_t)g->n_rows);
        orc_select(&c, u);
        free(up); free(dn); free(up2); free(dn2);
    }
    res->seconds = orc_now() - t0;

    int64_t T = 0, TH = 0, M = 0, MH = 0;
    for (int un = 0; un < n_units; un++) {
        orc_unit* u = &res->units[un];
        res->unit_t0[un] = T;
        res->unit_m0[un] = M;
        T += u->n_start;
        for (int t = 0; t < u->n_start; t++) TH += u->tl_n[t];
        M += u->n_tracks;
        for (int k = 0; k < u->n_tracks; k++) MH += u->trk_n[k];
    }
    res->unit_t0[n_units] = T;
    res->unit_m0[n_units] = M;
    res->n_tracklets = T;
    res->n_tracklet_hits = TH;
    res->n_tracks = M;
    res->n_track_hits = MH;
    return res;
}

/* sizes[0..5] = clusters, tracklets, tracklet hits, tracks, track hits; seconds */
void orc_sizes(const orc_result* r, int64_t* sizes, double* seconds)
{
    sizes[0] = r->n_clusters;
    sizes[1] = r->n_tracklets;
    sizes[2] = r->n_tracklet_hits;
    sizes[3] = r->n_tracks;
    sizes[4] = r->n_track_hits;
    if (seconds) *seconds = r->seconds;
}

void orc_copy_links(const orc_result* r, int32_t* up_raw, int32_t* dn_raw, int32_t* up, int32_t* dn)
{
    size_t n = (size_t)r->n_clusters;
    if (up_raw) memcpy(up_raw, r->up_raw, n * 4);
    if (dn_raw) memcpy(dn_raw, r->dn_raw, n * 4);
    if (up) memcpy(up, r->up, n * 4);
    if (dn) memcpy(dn, r->dn, n * 4);
}

/* Tracklets in canonical order t: start (global cluster index), unit,
 * f[ORC_NTF], nhits, alive, hit_off[T + 1], hits (global, rows ascending).  */
void orc_copy_tracklets(const orc_result* r, int32_t* start, int32_t* unit, double* f,
                        int32_t* nhits, int32_t* alive, int64_t* hit_off, int32_t* hits)
{
    int64_t t = 0, h = 0;
    for (int un = 0; un < r->n_units; un++) {
        const orc_unit* u = &r->units[un];
        for (int k = 0; k < u->n_start; k++, t++) {
            start[t] = u->base + u->start[k];
            unit[t] = un;
            memcpy(f + (size_t)t * ORC_NTF, u->tl_f + (size_t)k * ORC_NTF, sizeof(double) * ORC_NTF);
            nhits[t] = u->tl_n[k];
            alive[t] = u->tl_alive[k];
            hit_off[t] = h;
            for (int j = 0; j < u->tl_n[k]; j++)
                hits[h++] = u->base + u->tl_hits[(size_t)k * (size_t)r->n_rows + (size_t)j];
        }
    }
    hit_off[t] = h;
}

/* Tracks in canonical order: tracklet id, owned hit count, hit_off[M + 1],
 * owned hits (global, rows ascending).                                      */
void orc_copy_tracks(const orc_result* r, int32_t* trk_t, int32_t* nhits, int64_t* hit_off,
                     int32_t* hits)
{
    int64_t m = 0, h = 0;
    for (int un = 0; un < r->n_units; un++) {
        const orc_unit* u = &r->units[un];
        for (int k = 0; k < u->n_tracks; k++, m++) {
            trk_t[m] = (int32_t)(r->unit_t0[un] + u->trk_t[k]);
            nhits[m] = u->trk_n[k];
            hit_off[m] = h;
            for (int j = 0; j < u->trk_n[k]; j++)
                hits[h++] = u->base + u->trk_hits[(size_t)k * (size_t)r->n_rows + (size_t)j];
        }
    }
    hit_off[m] = h;
}

void orc_free(orc_result* r)
{
    if (!r) return;
    for (int un = 0; un < r->n_units; un++) {
        orc_unit* u = &r->units[un];
        free(u->rstart); free(u->y); free(u->z); free(u->id); free(u->row);
        free(u->start); free(u->tl_f); free(u->tl_n); free(u->tl_alive); free(u->tl_hits);
        free(u->trk_t); free(u->trk_n); free(u->trk_hits);
    }
    free(r->units); free(r->unit_base); free(r->unit_t0); free(r->unit_m0);
    free(r->up_raw); free(r->dn_raw); free(r->up); free(r->dn);
    free(r);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Single-function entry points for the pin tests.                          */
/* A state vector is 15 doubles: x y z s t q cy[6] cz[3].                    */
/* ------------------------------------------------------------------------ */

static void orc_unpack(const double* v, orc_state* st)
{
    st->x = RC(v[0]); st->y = RC(v[1]); st->z = RC(v[2]);
    st->s = RC(v[3]); st->t = RC(v[4]); st->q = RC(v[5]);
    for (int k = 0; k < 6; k++) st->cy[k] = RC(v[6 + k]);
    for (int k = 0; k < 3; k++) st->cz[k] = RC(v[12 + k]);
}

static void orc_pack(const orc_state* st, double* v)
{
    v[0] = (double)st->x; v[1] = (double)st->y; v[2] = (double)st->z;
    v[3] = (double)st->s; v[4] = (double)st->t; v[5] = (double)st->q;
    for (int k = 0; k < 6; k++) v[6 + k] = (double)st->cy[k];
    for (int k = 0; k < 3; k++) v[12 + k] = (double)st->cz[k];
}

int orc_propagate(const orc_params* p, double bz, double* v, double x1)
{
    orc_state st;
    orc_unpack(v, &st);
    int ok = orc_prop(&st, RC(x1), RC(-ORC_KAPPA * bz), RC(p->s_max));
    orc_pack(&st, v);
    return ok;
}

void orc_update_state(const orc_params* p, double* v, double my, double mz, double* chi2)
{
    orc_state st;
    orc_unpack(v, &st);
    real sy = RC(p->sigma_y), sz = RC(p->sigma_z);
    real c2 = RC(*chi2);
    orc_update(&st, RC(my), RC(mz), sy * sy, sz * sz, &c2);
    orc_pack(&st, v);
    *chi2 = (double)c2;
}

/* The Phase-2 fit on a given hit list: start from state v (its covariance is
 * reset to the T1 diagonal), propagate to x[k] and update with (y[k], z[k])
 * for k = 0..n-1 in the given order.  Returns the number of hits filtered
 * before a propagation failure; v receives the final state; chi2 the sum.    */
int orc_fit_hits(const orc_params* p, double bz, double* v, int n, const double* x,
                 const double* y, const double* z, double* chi2)
{
    orc_state st;
    orc_unpack(v, &st);
    real sy = RC(p->sigma_y), sz = RC(p->sigma_z);
    orc_reset_cov(&st, sy * sy, sz * sz, RC(p->var_s), RC(p->var_q), RC(p->var_t));
    real c2 = RC(0);
    real kB = RC(-ORC_KAPPA * bz);
    int k;
    for (k = 0; k < n; k++) {
        if (!orc_prop(&st, RC(x[k]), kB, RC(p->s_max))) break;
        orc_update(&st, RC(y[k]), RC(z[k]), sy * sy, sz * sz, &c2);
    }
    orc_pack(&st, v);
    *chi2 = (double)c2;
    return k;
}
