/*
 * CPU oracle of the final track fit: the full Kalman filter refit of each
 * selected track (Sec. 2, "Track fit"; Table 1 row 4), with the magnetic
 * field given as a polynomial instead of a field map (Sec. 2: the polynomial
 * approximation avoids slow field-map reads).
 *
 * TEST INFRASTRUCTURE ONLY, like tpc_oracle.c (built into the same library):
 * loaded by the tests, the package smoke check and the benchmark's
 * CPU-baseline leg, never by the CUDA path; it shares no source with it.
 *
 * The paper names the step but gives no equations; the readings (F1-F6 in
 * the design notes) are:
 *   F1 state p = (y, z, s = sin phi, t = tan lambda, q = q/pT) at the plane
 *      x, with a full symmetric 5x5 covariance C, carried as a square-root
 *      factor S (C = S S^T, S a full 5x5 matrix); the output is C (15 packed
 *      lower entries, C[i][j] at i (i + 1) / 2 + j for i >= j);
 *   F2 propagation is the exact helix step of the tracklet filter (signed
 *      chord, arc series to u^4); the covariance is transported with the full
 *      analytic Jacobian J of that step (all cross terms kept), S <- J S,
 *      no process noise;
 *   F3 the field is Bz(rho, z) = bz + z (b1 + z b2) + rho^2 (b3 + z (b4 + z b5)),
 *      rho^2 = x^2 + y^2 (frame independent), evaluated once per step at the
 *      straight-line midpoint and held constant over the step; the Jacobian
 *      ignores the field's derivatives;
 *   F4 update with the 2-D measurement (y, z) of variance diag(sy^2, sz^2),
 *      in the square-root form of J. E. Potter (1963; R. H. Battin,
 *      Astronautical Guidance, 1964): V is diagonal, so the update is the
 *      scalar update of y followed by that of z (the same posterior and chi2
 *      as the joint 2-D update); for measured component a with residual
 *      r = m_a - p_a:  phi = S^T e_a (row a of S), alpha = 1 / (phi.phi + V_a),
 *      gamma = alpha / (1 + sqrt(alpha V_a)), p += alpha r S phi,
 *      S -= gamma (S phi) phi^T, chi2 += alpha r^2.  (In binary32 the
 *      conventional C -= K H C lost up to 9 % of the q/pT variance against
 *      FP64 on steep low-momentum tracks, where the wide prior in sin phi is
 *      multiplied by 1 / cos^3 phi; the square-root form stays within ~1e-5.);
 *   F5 two passes over the track's clusters, each cluster on its own x:
 *      outward (rows ascending) from the tracklet state, then inward from the
 *      outermost cluster; each pass starts at its first cluster with y, z set
 *      to that measurement, S = diag(sqrt(sy^2), sqrt(sz^2), sqrt(var_s),
 *      sqrt(var_t), sqrt(var_q)) and chi2 = 0 (an infinite prior on y and z),
 *      then filters the rest.  The
 *      output is the inward pass's state at the innermost cluster,
 *      chi2, ndf = 2 n - 5;
 *   F6 a step with |sin phi| above s_max before or after it fails the fit:
 *      status 1, the output holds the state reached, ndf counts the clusters
 *      filtered in the failing pass.
 *
 * Parity status (tests/test_oracle_refit.py):
 *   propagate   closed-form helix (textbook arcsine form, not the series)
 *   Jacobian    every column against central finite differences of propagate
 *   update      Bayesian posterior in information form (numpy.linalg),
 *               for a 2-D measurement of (y, z)
 *   refit       small-noise limit equals one Gauss-Newton step of least
 *               squares on the closed-form helix, estimate and covariance;
 *               noise-free tracks: fixed point = truth; pulls and chi2/ndf on
 *               smeared tracks; non-uniform field: truth recovered on tracks
 *               integrated numerically through the same polynomial field
 *
 * Written with plain 5x5 matrices and loops; every product runs its sum in
 * increasing index order.
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
typedef ORACLE_REAL rreal;

#define RF(c) ((rreal)(c))
#define RF_IS_FLOAT (sizeof(rreal) == sizeof(float))
#define RF_KAPPA 0.00299792458 /* curvature [1/cm] per (T * c/GeV) */
#define RF_NOUT 24             /* x p[5] cov[15] chi2 ndf status */

static inline rreal f_sqrt(rreal v) { return RF_IS_FLOAT ? (rreal)sqrtf((float)v) : (rreal)sqrt((double)v); }
static inline rreal f_fabs(rreal v) { return RF_IS_FLOAT ? (rreal)fabsf((float)v) : (rreal)fabs((double)v); }
static inline rreal f_copysign(rreal v, rreal s)
{
    return RF_IS_FLOAT ? (rreal)copysignf((float)v, (float)s) : (rreal)copysign((double)v, (double)s);
}

/* Constants of the fit in working precision. */
typedef struct {
    double sigma_y, sigma_z, var_s, var_t, var_q, s_max;
    double bz;       /* constant term of the field (T)                          */
    double b[5];     /* field polynomial: z, z^2, rho^2, rho^2 z, rho^2 z^2       */
} orc_fit_params;

typedef struct {
    rreal sy2, sz2, var_s, var_t, var_q, s_max;
    rreal kB0;       /* -kappa * bz, rounded once from double                   */
    rreal kP;        /* -kappa                                                  */
    rreal b[5];
} rf_ctx;

static void rf_ctx_init(rf_ctx* c, const orc_fit_params* p)
{
    rreal sy = RF(p->sigma_y), sz = RF(p->sigma_z);
    c->sy2 = sy * sy;
    c->sz2 = sz * sz;
    c->var_s = RF(p->var_s);
    c->var_t = RF(p->var_t);
    c->var_q = RF(p->var_q);
    c->s_max = RF(p->s_max);
    c->kB0 = RF(-RF_KAPPA * p->bz);
    c->kP = RF(-RF_KAPPA);
    for (int j = 0; j < 5; j++) c->b[j] = RF(p->b[j]);
}

typedef struct {
    rreal x;
    rreal p[5];      /* y z s t q */
    rreal S[5][5];   /* covariance factor: C = S S^T */
} rf_state;

/* F2, F3: one step of the state (x, p) to the plane x1 and its Jacobian J.
 * Returns 1 on success, 0 when |sin phi| exceeds s_max before or after the
 * step (x, p untouched). */
static int rf_step(const rf_ctx* c, rreal* x, rreal* p, rreal J[5][5], rreal x1)
{
    memset(J, 0, sizeof(rreal) * 25);
    for (int i = 0; i < 5; i++) J[i][i] = RF(1);
    rreal d = x1 - *x;
    if (d == RF(0)) return 1;
    rreal y = p[0], z = p[1], s0 = p[2], t = p[3], q = p[4];
    if (f_fabs(s0) > c->s_max) return 0;
    rreal c0 = f_sqrt(RF(1) - s0 * s0);

    /* field at the straight-line midpoint of the step */
    rreal h = d * RF(0.5);
    rreal xm = *x + h;
    rreal ym = y + h * (s0 / c0);
    rreal zm = z + h * (t / c0);
    rreal r2 = xm * xm + ym * ym;
    rreal poly = zm * (c->b[0] + zm * c->b[1]) + r2 * (c->b[2] + zm * (c->b[3] + zm * c->b[4]));
    rreal kB = c->kB0 + c->kP * poly;

    rreal k = kB * q;
    rreal s1 = s0 + k * d;
    if (f_fabs(s1) > c->s_max) return 0;
    rreal c1 = f_sqrt(RF(1) - s1 * s1);
    rreal A = s0 + s1;
    rreal B = c0 + c1;
    rreal dy = d * A / B;
    rreal L = f_copysign(f_sqrt(d * d + dy * dy), d);
    rreal u = k * L * RF(0.5);
    rreal u2 = u * u;
    rreal arc = L * (RF(1) + u2 * (RF(1.0 / 6.0) + u2 * RF(3.0 / 40.0)));
    rreal dz = t * arc;

    /* Jacobian of (y1, z1, s1, t1, q1) by (y, z, s, t, q):
     *   dy1/ds = d (2 B + A (s0/c0 + s1/c1)) / B^2
     *   dy1/dq = d (kB d) (B + A s1/c1) / B^2
     *   ds1/dq = kB d
     *   arc(L, k): d arc/dL = 1 + u^2/2 + 3 u^4/8, d arc/dk = L^2/2 (u/3 + 3 u^3/10)
     *   dL/d(dy) = dy / L
     *   dz1/ds = t (d arc/dL) (dy/L) dy1/ds
     *   dz1/dq = t ((d arc/dL) (dy/L) dy1/dq + (d arc/dk) kB)
     *   dz1/dt = arc                                                        */
    rreal iB2 = RF(1) / (B * B);
    rreal hq = kB * d;
    rreal ja_in = RF(2) * B + A * (s0 / c0 + s1 / c1);
    rreal ja = d * ja_in * iB2;
    rreal jb_in = B + A * (s1 / c1);
    rreal jb = d * hq * jb_in * iB2;
    rreal g = RF(1) + u2 * (RF(0.5) + u2 * RF(0.375));
    rreal w = dy / L;
    rreal jcs = t * g * w * ja;
    rreal fp = u * (RF(1.0 / 3.0) + u2 * RF(0.3));
    rreal jcq = t * (g * w * jb + L * L * RF(0.5) * fp * kB);

    J[0][2] = ja;  J[0][4] = jb;
    J[1][2] = jcs; J[1][3] = arc; J[1][4] = jcq;
    J[2][4] = hq;

    *x = x1;
    p[0] = y + dy;
    p[1] = z + dz;
    p[2] = s1;
    return 1;
}

static int rf_prop(const rf_ctx* c, rf_state* st, rreal x1)
{
    if (x1 - st->x == RF(0)) return 1;
    rreal J[5][5];
    rreal x = st->x, p[5];
    for (int i = 0; i < 5; i++) p[i] = st->p[i];
    if (!rf_step(c, &x, p, J, x1)) return 0;
    /* S1 = J S */
    rreal S1[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            rreal acc = J[i][0] * st->S[0][j];
            for (int m = 1; m < 5; m++) acc = acc + J[i][m] * st->S[m][j];
            S1[i][j] = acc;
        }
    memcpy(st->S, S1, sizeof S1);
    st->x = x;
    for (int i = 0; i < 5; i++) st->p[i] = p[i];
    return 1;
}

/* F4: measurement update with (my, mz): scalar square-root updates of y,
 * then of z. */
static void rf_update_1(rf_state* st, int a, rreal m, rreal V, rreal* chi2)
{
    rreal r = m - st->p[a];
    rreal phi[5], Sphi[5];
    for (int j = 0; j < 5; j++) phi[j] = st->S[a][j];
    rreal pp = phi[0] * phi[0];
    for (int j = 1; j < 5; j++) pp = pp + phi[j] * phi[j];
    rreal alpha = RF(1) / (pp + V);
    rreal gamma = alpha / (RF(1) + f_sqrt(alpha * V));
    for (int i = 0; i < 5; i++) {
        rreal acc = st->S[i][0] * phi[0];
        for (int j = 1; j < 5; j++) acc = acc + st->S[i][j] * phi[j];
        Sphi[i] = acc;
    }
    rreal ar = alpha * r;
    for (int i = 0; i < 5; i++) st->p[i] = st->p[i] + ar * Sphi[i];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) st->S[i][j] = st->S[i][j] - gamma * Sphi[i] * phi[j];
    *chi2 = *chi2 + ar * r;
}

static void rf_update(const rf_ctx* c, rf_state* st, rreal my, rreal mz, rreal* chi2)
{
    rf_update_1(st, 0, my, c->sy2, chi2);
    rf_update_1(st, 1, mz, c->sz2, chi2);
}

/* F5: start of a pass at a cluster */
static void rf_init_pass(const rf_ctx* c, rf_state* st, rreal my, rreal mz, rreal* chi2)
{
    st->p[0] = my;
    st->p[1] = mz;
    memset(st->S, 0, sizeof st->S);
    st->S[0][0] = f_sqrt(c->sy2);
    st->S[1][1] = f_sqrt(c->sz2);
    st->S[2][2] = f_sqrt(c->var_s);
    st->S[3][3] = f_sqrt(c->var_t);
    st->S[4][4] = f_sqrt(c->var_q);
    *chi2 = RF(0);
}

/* C = S S^T, lower triangle */
static rreal rf_cov(const rf_state* st, int i, int j)
{
    rreal acc = st->S[i][0] * st->S[j][0];
    for (int m = 1; m < 5; m++) acc = acc + st->S[i][m] * st->S[j][m];
    return acc;
}

static void rf_store(const rf_state* st, rreal chi2, int ndf, int status, double* out)
{
    out[0] = (double)st->x;
    for (int i = 0; i < 5; i++) out[1 + i] = (double)st->p[i];
    for (int i = 0, k = 0; i < 5; i++)
        for (int j = 0; j <= i; j++, k++) out[6 + k] = (double)rf_cov(st, i, j);
    out[21] = (double)chi2;
    out[22] = (double)ndf;
    out[23] = (double)status;
}

/* One track: start state st6 = (x, y, z, s, t, q); n clusters (x, y, z, id)
 * in row-ascending order.  out[RF_NOUT]. */
static void rf_refit(const rf_ctx* c, const double* st6, int n, const float* const* cl, double* out)
{
    rf_state st;
    memset(&st, 0, sizeof st);
    st.x = RF(st6[0]);
    for (int i = 0; i < 5; i++) st.p[i] = RF(st6[1 + i]);
    rreal chi2 = RF(0);
    if (n <= 0) { rf_store(&st, chi2, -5, 1, out); return; }
    /* outward pass */
    for (int k = 0; k < n; k++) {
        if (!rf_prop(c, &st, RF(cl[k][0]))) { rf_store(&st, chi2, 2 * k - 5, 1, out); return; }
        if (k == 0) rf_init_pass(c, &st, RF(cl[k][1]), RF(cl[k][2]), &chi2);
        else rf_update(c, &st, RF(cl[k][1]), RF(cl[k][2]), &chi2);
    }
    /* inward pass, from the outermost cluster */
    for (int j = 0; j < n; j++) {
        int k = n - 1 - j;
        if (!rf_prop(c, &st, RF(cl[k][0]))) { rf_store(&st, chi2, 2 * j - 5, 1, out); return; }
        if (j == 0) rf_init_pass(c, &st, RF(cl[k][1]), RF(cl[k][2]), &chi2);
        else rf_update(c, &st, RF(cl[k][1]), RF(cl[k][2]), &chi2);
    }
    rf_store(&st, chi2, 2 * n - 5, 0, out);
}

/* ------------------------------------------------------------------------ */
/* Entry points                                                              */
/* ------------------------------------------------------------------------ */

/* Refit M tracks.  st6[M][6] start states; hit_off[M + 1] into hits; hits are
 * positions in clusters[.][4] (x, y, z, id bits); out[M][RF_NOUT]. */
void orc_refit_tracks(const orc_fit_params* p, int M, const double* st6, const int64_t* hit_off,
                      const int32_t* hits, const float* clusters, double* out, int n_threads)
{
    rf_ctx c;
    rf_ctx_init(&c, p);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int m = 0; m < M; m++) {
        int n = (int)(hit_off[m + 1] - hit_off[m]);
        const float* cl[512];
        if (n > 512) n = 512;
        for (int k = 0; k < n; k++) cl[k] = clusters + (size_t)hits[hit_off[m] + k] * 4;
        rf_refit(&c, st6 + (size_t)m * 6, n, cl, out + (size_t)m * RF_NOUT);
    }
    (void)n_threads;
}

/* A fit vector for the single-step entry points: x, p[5], S[5][5] row-major
 * (31 doubles). */
static void rf_unpack(const double* v, rf_state* st)
{
    st->x = RF(v[0]);
    for (int i = 0; i < 5; i++) st->p[i] = RF(v[1 + i]);
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) st->S[i][j] = RF(v[6 + 5 * i + j]);
}

static void rf_pack(const rf_state* st, double* v)
{
    v[0] = (double)st->x;
    for (int i = 0; i < 5; i++) v[1 + i] = (double)st->p[i];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) v[6 + 5 * i + j] = (double)st->S[i][j];
}

int orc_refit_propagate(const orc_fit_params* p, double* v, double x1)
{
    rf_ctx c;
    rf_ctx_init(&c, p);
    rf_state st;
    rf_unpack(v, &st);
    int ok = rf_prop(&c, &st, RF(x1));
    rf_pack(&st, v);
    return ok;
}

void orc_refit_update(const orc_fit_params* p, double* v, double my, double mz, double* chi2)
{
    rf_ctx c;
    rf_ctx_init(&c, p);
    rf_state st;
    rf_unpack(v, &st);
    rreal c2 = RF(*chi2);
    rf_update(&c, &st, RF(my), RF(mz), &c2);
    rf_pack(&st, v);
    *chi2 = (double)c2;
}

/* ------------------------------------------------------------------------ */
/* Phase II track merging (Sec. 2 step 3; Table 1 row 3: "matching           */
/* covariance").  Readings M1-M6 of the design notes:                        */
/*   M1 candidates: two refitted tracks (status 0) of one event, A inner, B  */
/*      outer: in one sector with x_last(A) < x_first(B) <= x_last(A) + gap  */
/*      (a gap the track following did not cover), or in adjacent sectors of */
/*      one side with x_last(A) - overlap <= x_first(B) <= x_last(A) + gap   */
/*      (the sector border);                                                 */
/*   M2 A's refit state (at its innermost cluster) is propagated with its    */
/*      covariance (C <- J C J^T) to x_first(B); across a border it is first */
/*      propagated to x_last(A), rotated into B's frame (M3), then to        */
/*      x_first(B);                                                          */
/*   M3 rotation by theta = alpha_B - alpha_A (+-20 deg): the point and the  */
/*      direction rotate (x' = x cos + y sin, y' = y cos - x sin,            */
/*      phi' = phi - theta), the state is referred to the plane through the  */
/*      rotated point; Jacobian dy'/dy = cos phi / cos phi',                  */
/*      dz'/dy = -t sin(theta) / cos phi', ds'/dy = -k sin(theta) (k of the  */
/*      uniform field), ds'/ds = cos phi' / cos phi; fails unless cos phi' > 0*/
/*      and |sin phi'| <= s_max;                                             */
/*   M4 compatibility chi2 = d^T (C_A + C_B)^-1 d, d = p_A - p_B, by a       */
/*      Cholesky factorisation and a forward solve; compatible iff every     */
/*      step succeeds, |d_y| <= window and |d_z| <= window (cm), the sum is  */
/*      positive definite and chi2 <= chi2_max;                              */
/*   M5 A and B are merged iff B is A's best outer candidate and A is B's    */
/*      best inner candidate (smallest chi2, ties by the smaller track       */
/*      index): each track has at most one outer and one inner partner, the  */
/*      links form chains ordered by x_first;                                */
/*   M6 output per track: the index of its outer partner (-1: none) and the */
/*      link's chi2.                                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    double chi2_max;
    double gap;        /* cm */
    double overlap;    /* cm */
    double window;     /* cm */
    double cos_t;      /* cos and sin of the angle between adjacent sectors */
    double sin_t;
} orc_merge_params;

typedef struct {
    rreal x;
    rreal p[5];
    rreal C[5][5];
} mg_state;

/* C <- J C J^T, sums in index order */
static void mg_transport(rreal C[5][5], rreal J[5][5])
{
    rreal F[5][5], C1[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            rreal acc = J[i][0] * C[0][j];
            for (int m = 1; m < 5; m++) acc = acc + J[i][m] * C[m][j];
            F[i][j] = acc;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            rreal acc = F[i][0] * J[j][0];
            for (int m = 1; m < 5; m++) acc = acc + F[i][m] * J[j][m];
            C1[i][j] = acc;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) { C[i][j] = C1[i][j]; C[j][i] = C1[i][j]; }
}

static int mg_prop(const rf_ctx* c, mg_state* st, rreal x1)
{
    if (x1 - st->x == RF(0)) return 1;
    rreal J[5][5];
    if (!rf_step(c, &st->x, st->p, J, x1)) return 0;
    mg_transport(st->C, J);
    return 1;
}

/* M3: rotate the state into the frame turned by theta (cos ct, sin st_). */
static int mg_rotate(const rf_ctx* c, mg_state* st, rreal ct, rreal stt)
{
    rreal x = st->x, y = st->p[0], s = st->p[2], t = st->p[3], q = st->p[4];
    if (f_fabs(s) > c->s_max) return 0;
    rreal cs = f_sqrt(RF(1) - s * s);
    rreal xb = x * ct + y * stt;
    rreal yb = y * ct - x * stt;
    rreal sb = s * ct - cs * stt;
    rreal cb = cs * ct + s * stt;
    if (!(cb > RF(0)) || f_fabs(sb) > c->s_max) return 0;
    rreal J[5][5];
    memset(J, 0, sizeof J);
    for (int i = 0; i < 5; i++) J[i][i] = RF(1);
    J[0][0] = cs / cb;
    J[1][0] = -(t * stt) / cb;
    J[2][0] = -(c->kB0 * q * stt);
    J[2][2] = cb / cs;
    mg_transport(st->C, J);
    st->x = xb;
    st->p[0] = yb;
    st->p[2] = sb;
    return 1;
}

/* M4: chi2 of d = pa - pb with covariance Ca + Cb; 0 when not positive
 * definite. */
static int mg_chi2(const mg_state* a, const mg_state* b, rreal* chi2)
{
    rreal C[5][5], L[5][5], d[5], w[5];
    memset(L, 0, sizeof L);
    for (int i = 0; i < 5; i++) {
        d[i] = a->p[i] - b->p[i];
        for (int j = 0; j < 5; j++) C[i][j] = a->C[i][j] + b->C[i][j];
    }
    for (int j = 0; j < 5; j++) {
        rreal acc = C[j][j];
        for (int m = 0; m < j; m++) acc = acc - L[j][m] * L[j][m];
        if (!(acc > RF(0))) return 0;
        L[j][j] = f_sqrt(acc);
        for (int i = j + 1; i < 5; i++) {
            rreal v = C[i][j];
            for (int m = 0; m < j; m++) v = v - L[i][m] * L[j][m];
            L[i][j] = v / L[j][j];
        }
    }
    rreal sum = RF(0);
    for (int i = 0; i < 5; i++) {
        rreal v = d[i];
        for (int m = 0; m < i; m++) v = v - L[i][m] * w[m];
        w[i] = v / L[i][i];
        sum = sum + w[i] * w[i];
    }
    *chi2 = sum;
    return 1;
}

static void mg_from_fit(const double* f, mg_state* st)
{
    st->x = RF(f[0]);
    for (int i = 0; i < 5; i++) st->p[i] = RF(f[1 + i]);
    for (int i = 0, k = 0; i < 5; i++)
        for (int j = 0; j <= i; j++, k++) { st->C[i][j] = RF(f[6 + k]); st->C[j][i] = RF(f[6 + k]); }
}

/* M1-M4 for one candidate pair; rot = 0 (same sector), +1 (B is the next
 * sector, theta = +20 deg), -1 (previous sector).  Returns 1 if compatible. */
static int mg_pair(const rf_ctx* c, const orc_merge_params* mp, const double* fa, double xa_last,
                   const double* fb, int rot, rreal* chi2)
{
    mg_state a, b;
    mg_from_fit(fa, &a);
    mg_from_fit(fb, &b);
    if (rot != 0) {
        if (!mg_prop(c, &a, RF(xa_last))) return 0;
        rreal ct = RF(mp->cos_t), stt = rot > 0 ? RF(mp->sin_t) : -RF(mp->sin_t);
        if (!mg_rotate(c, &a, ct, stt)) return 0;
    }
    if (!mg_prop(c, &a, b.x)) return 0;
    rreal w = RF(mp->window);
    if (!(f_fabs(a.p[0] - b.p[0]) <= w) || !(f_fabs(a.p[1] - b.p[1]) <= w)) return 0;
    if (!mg_chi2(&a, &b, chi2)) return 0;
    return *chi2 <= RF(mp->chi2_max);
}

/* M1: is B a candidate outer partner of A?  Returns rot + 2 (1..3) or 0. */
static int mg_candidate(const orc_merge_params* mp, int n_sectors, int ua, int ub, const double* fa,
                        double xa_last, const double* fb)
{
    if (fa[23] != 0.0 || fb[23] != 0.0) return 0;
    int half = n_sectors / 2;
    int ea = ua / n_sectors, eb = ub / n_sectors;
    if (ea != eb) return 0;
    int sa = ua % n_sectors, sb = ub % n_sectors;
    if (sa / half != sb / half) return 0;  /* same side */
    rreal xl = RF(xa_last), xf = RF(fb[0]);
    rreal gap = RF(mp->gap), ov = RF(mp->overlap);
    if (sa == sb) return (xl < xf && xf <= xl + gap) ? 2 : 0;
    int la = sa % half, lb = sb % half;
    int rot = 0;
    if (lb == (la + 1) % half) rot = 1;
    else if (lb == (la + half - 1) % half) rot = -1;
    else return 0;
    return (xl - ov <= xf && xf <= xl + gap) ? rot + 2 : 0;
}

/* Merge links of M refitted tracks (canonical order: grouped by unit).
 * unit[M] = event * n_sectors + sector; fits[M][RF_NOUT]; x_last[M] = x of
 * each track's outermost cluster.  next[M]: outer partner or -1; chi2[M]. */
void orc_merge_tracks(const orc_fit_params* p, const orc_merge_params* mp, int M, int n_sectors,
                      const int32_t* unit, const double* fits, const double* x_last, int32_t* next,
                      double* chi2, int n_threads)
{
    rf_ctx c;
    rf_ctx_init(&c, p);
    int n_units = M ? unit[M - 1] + 1 : 0;
    int* first = (int*)calloc((size_t)n_units + 2, sizeof(int));
    for (int u = 0, m = 0; u <= n_units; u++) {
        while (m < M && unit[m] < u) m++;
        first[u] = m;
    }
    double* bo = (double*)malloc(sizeof(double) * ((size_t)M + 1));
    double* bi = (double*)malloc(sizeof(double) * ((size_t)M + 1));
    int* io = (int*)malloc(sizeof(int) * ((size_t)M + 1));
    int* ii = (int*)malloc(sizeof(int) * ((size_t)M + 1));
    for (int m = 0; m < M; m++) { io[m] = -1; ii[m] = -1; }
    int half = n_sectors / 2;
    (void)n_threads;
    /* candidate units of A's outer partners: its own and the two neighbours */
    for (int a = 0; a < M; a++) {
        int ua = unit[a], e = ua / n_sectors, sa = ua % n_sectors;
        int base = (sa / half) * half, la = sa % half;
        int us[3] = {ua, e * n_sectors + base + (la + 1) % half, e * n_sectors + base + (la + half - 1) % half};
        for (int k = 0; k < 3; k++) {
            int ub = us[k];
            if (k > 0 && (ub >= n_units || us[2] == us[1] && k == 2)) continue;
            for (int b = first[ub]; b < first[ub + 1]; b++) {
                if (b == a) continue;
                int cnd = mg_candidate(mp, n_sectors, ua, ub, fits + (size_t)a * RF_NOUT, x_last[a],
                                       fits + (size_t)b * RF_NOUT);
                if (!cnd) continue;
                rreal x2;
                if (!mg_pair(&c, mp, fits + (size_t)a * RF_NOUT, x_last[a], fits + (size_t)b * RF_NOUT,
                             cnd - 2, &x2))
                    continue;
                double v = (double)x2;
                if (io[a] < 0 || v < bo[a] || (v == bo[a] && b < io[a])) { bo[a] = v; io[a] = b; }
                if (ii[b] < 0 || v < bi[b] || (v == bi[b] && a < ii[b])) { bi[b] = v; ii[b] = a; }
            }
        }
    }
    for (int a = 0; a < M; a++) {
        int b = io[a];
        if (b >= 0 && ii[b] == a) { next[a] = b; chi2[a] = bo[a]; }
        else { next[a] = -1; chi2[a] = 0.0; }
    }
    free(first); free(bo); free(bi); free(io); free(ii);
}

/* Single-step entries for the pins: a merge vector is x, p[5], C[5][5]
 * row-major (31 doubles). */
static void mg_unpack(const double* v, mg_state* st)
{
    st->x = RF(v[0]);
    for (int i = 0; i < 5; i++) st->p[i] = RF(v[1 + i]);
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) st->C[i][j] = RF(v[6 + 5 * i + j]);
}

static void mg_pack(const mg_state* st, double* v)
{
    v[0] = (double)st->x;
    for (int i = 0; i < 5; i++) v[1 + i] = (double)st->p[i];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) v[6 + 5 * i + j] = (double)st->C[i][j];
}

int orc_merge_rotate(const orc_fit_params* p, double* v, double cos_t, double sin_t)
{
    rf_ctx c;
    rf_ctx_init(&c, p);
    mg_state st;
    mg_unpack(v, &st);
    int ok = mg_rotate(&c, &st, RF(cos_t), RF(sin_t));
    mg_pack(&st, v);
    return ok;
}

int orc_merge_propagate(const orc_fit_params* p, double* v, double x1)
{
    rf_ctx c;
    rf_ctx_init(&c, p);
    mg_state st;
    mg_unpack(v, &st);
    int ok = mg_prop(&c, &st, RF(x1));
    mg_pack(&st, v);
    return ok;
}

int orc_merge_chi2(const double* va, const double* vb, double* chi2)
{
    mg_state a, b;
    mg_unpack(va, &a);
    mg_unpack(vb, &b);
    rreal x2 = RF(0);
    int ok = mg_chi2(&a, &b, &x2);
    *chi2 = (double)x2;
    return ok;
}

/* ------------------------------------------------------------------------ */
/* Continuous readout (Sec. 3.3, Run 3 conditions): the drift coordinate z'  */
/* of a cluster is its spatial z only once the collision time is known, so   */
/* transformation and tracking are coupled.  Readings T01-T05:               */
/*   T01 the tracker runs on z' (a collision's unknown time shifts all its   */
/*       clusters by sign(side) dz, which the track model absorbs);          */
/*   T02 each refitted track (status 0) is stepped to the beam line x = 0 of */
/*       its sector frame in 16 equal steps (targets x0 - i (x0 / 16), the   */
/*       last exactly 0: short enough for the arc series); it is a primary   */
/*       candidate if every step succeeds and |y(0)| <= y_cut; its offset   */
/*       estimate is u = sign(side) z'(0), sign = +1 on side A (sectors <    */
/*       n_sectors / 2), -1 on side C;                                       */
/*   T03 per time frame (one event of the batch) the candidates' u in        */
/*       [-z_max, z_max) are binned, h[b] with b = floor((u + z_max) / w);  */
/*       n[b] = sum of h over b-2..b+2, s[b] the same with weights 1 2 3 2 1;*/
/*       bin b is a collision peak if n[b] >= n_min, s[b] > s[b'] for b' in  */
/*       [b - W, b) and s[b] >= s[b'] for b' in (b, b + W] (the lowest of    */
/*       equal maxima); collisions are numbered by increasing peak bin;      */
/*       centre c = -z_max + (b + 1/2) w;                                    */
/*   T04 a candidate belongs to the collision whose centre is nearest, if    */
/*       |u - c| <= r (ties: the lower one); the collision's offset D is the */
/*       mean u of its tracks, summed as integers (u in units of 1e-4 cm,    */
/*       rounded to nearest) so the sum does not depend on order:            */
/*       D = (sum / n) 1e-4;                                                 */
/*   T05 per track: its collision (-1: none), u, and D (0 without one); the  */
/*       track's spatial z is z' - sign(side) D.                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    double y_cut;      /* cm */
    double bin;        /* cm */
    double z_max;      /* cm */
    double radius;     /* r, cm */
    int window;        /* W, bins */
    int n_min;
} orc_t0_params;

/* out[M][3]: collision, u, D (collision -1: none) */
void orc_t0_tracks(const orc_fit_params* p, const orc_t0_params* tp, int M, int n_sectors,
                   const int32_t* unit, const double* fits, double* out)
{
    rf_ctx c;
    rf_ctx_init(&c, p);
    rreal zmax = RF(tp->z_max), w = RF(tp->bin), ycut = RF(tp->y_cut);
    int nb = (int)ceil(2.0 * tp->z_max / tp->bin);
    int n_events = M ? unit[M - 1] / n_sectors + 1 : 0;
    int* bin = (int*)malloc(sizeof(int) * ((size_t)M + 1));
    rreal* u = (rreal*)malloc(sizeof(rreal) * ((size_t)M + 1));
    int* hist = (int*)calloc((size_t)nb, sizeof(int));
    int* grp = (int*)malloc(sizeof(int) * (size_t)nb);
    int64_t* gsum = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    int* gcnt = (int*)malloc(sizeof(int) * (size_t)nb);
    /* T02 */
    for (int m = 0; m < M; m++) {
        const double* f = fits + (size_t)m * RF_NOUT;
        bin[m] = -1;
        out[(size_t)m * 3 + 0] = -1.0;
        out[(size_t)m * 3 + 1] = 0.0;
        out[(size_t)m * 3 + 2] = 0.0;
        if (f[23] != 0.0) continue;
        rreal x = RF(f[0]), pp[5], J[5][5];
        for (int i = 0; i < 5; i++) pp[i] = RF(f[1 + i]);
        rreal h = x * RF(0.0625);
        rreal x0 = x;
        int ok = 1;
        for (int i = 1; i <= 16 && ok; i++) {
            rreal xt = i == 16 ? RF(0) : x0 - (rreal)i * h;
            if (xt - x != RF(0)) ok = rf_step(&c, &x, pp, J, xt);
        }
        if (!ok) continue;
        if (!(f_fabs(pp[0]) <= ycut)) continue;
        int side_a = (unit[m] % n_sectors) < n_sectors / 2;
        rreal um = side_a ? pp[1] : -pp[1];
        u[m] = um;
        out[(size_t)m * 3 + 1] = (double)um;
        if (!(um >= -zmax && um < zmax)) continue;
        int b = (int)floor((double)((um + zmax) / w));
        if (b < 0) b = 0;
        if (b >= nb) b = nb - 1;
        bin[m] = b;
    }
    /* T03, T04 per event */
    int* sm = (int*)malloc(sizeof(int) * (size_t)nb);
    int* peak = (int*)malloc(sizeof(int) * (size_t)nb);
    for (int e = 0, m0 = 0; e < n_events; e++) {
        int m1 = m0;
        while (m1 < M && unit[m1] / n_sectors == e) m1++;
        memset(hist, 0, sizeof(int) * (size_t)nb);
        for (int m = m0; m < m1; m++)
            if (bin[m] >= 0) hist[bin[m]]++;
        for (int b = 0; b < nb; b++) {
            int acc = 0, cnt = 0;
            for (int j = b - 2; j <= b + 2; j++)
                if (j >= 0 && j < nb) {
                    acc += (3 - abs(j - b)) * hist[j];
                    cnt += hist[j];
                }
            sm[b] = acc;
            grp[b] = cnt;  /* n[b] */
        }
        int np_ = 0;
        for (int b = 0; b < nb; b++) {
            if (grp[b] < tp->n_min) continue;
            int is_peak = 1;
            for (int j = b - tp->window; j < b && is_peak; j++)
                if (j >= 0 && !(sm[b] > sm[j])) is_peak = 0;
            for (int j = b + 1; j <= b + tp->window && is_peak; j++)
                if (j < nb && !(sm[b] >= sm[j])) is_peak = 0;
            if (is_peak) peak[np_++] = b;
        }
        for (int k = 0; k < np_; k++) { gsum[k] = 0; gcnt[k] = 0; }
        for (int m = m0; m < m1; m++) {
            if (bin[m] < 0) continue;
            int best = -1;
            rreal bd = RF(0);
            for (int k = 0; k < np_; k++) {
                rreal cen = -zmax + ((rreal)peak[k] + RF(0.5)) * w;
                rreal dd = f_fabs(u[m] - cen);
                if (dd <= RF(tp->radius) && (best < 0 || dd < bd)) { best = k; bd = dd; }
            }
            bin[m] = best < 0 ? -1 : nb + best;  /* reuse: nb + collision */
            if (best < 0) continue;
            gsum[best] += (int64_t)llrint((double)u[m] * 1e4);
            gcnt[best]++;
        }
        for (int m = m0; m < m1; m++) {
            if (bin[m] < nb) continue;
            int k = bin[m] - nb;
            out[(size_t)m * 3 + 0] = (double)k;
            out[(size_t)m * 3 + 2] = (double)(float)((double)gsum[k] / (double)gcnt[k] * 1e-4);
        }
        m0 = m1;
    }
    free(sm); free(peak);
    free(bin); free(u); free(hist); free(grp); free(gsum); free(gcnt);
}
