/*
 * FP64 CPU oracle of the batched alternating-minimization (AM) loop of
 * "GPU Accelerated Batch Multi-Convex Trajectory Optimization for a
 * Rectangular Holonomic Mobile Robot" (arXiv 2109.13030).
 *
 * TEST INFRASTRUCTURE ONLY: it is the plain, slow, checkable statement of
 * what the CUDA path must compute.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * Every matrix is built dense from its definition in the paper and every QP
 * is solved by an LU factorisation of its own KKT matrix (Eq. over_2), never
 * through a stored inverse.  The angles use atan2/cos/sin exactly as written
 * in Eq. zeta_2 - alpha_a.  Per trajectory the iteration runs the steps in
 * the order of Sec. III-D: xi1, xi2, xi3, xi4, then the multipliers.
 *
 * Readings of points the paper leaves open (each is a flag or a stated
 * choice, matched by the CUDA path):
 *  - alpha for an ellipse: default atan2(a*yt, b*xt), the exact joint (alpha,
 *    d) minimiser outside the ellipse; alpha_mode=1 gives the printed
 *    atan2(yt, xt).  Both agree for circles.
 *  - d_ij is clipped to d >= 1; d_v, d_a to [0, 1] (a speed bound).
 *  - each obstacle's semi-axes are inflated by the robot circle radius.
 *  - g uses v_max d_v cos(alpha_v) and a_max d_a cos(alpha_a) (Eq. fv, fa).
 *  - KKT right-hand side is [-qbar; b] (stationarity of Eq. over_1).
 *  - obstacle rows: m*n*q per side, circle-major, then obstacle, then step.
 *  - Q stacks Pdd^T Pdd on all four blocks of xi1; the slack blocks carry
 *    boundary rows from the chain rule on psi's boundary values.
 *  - psi_t = psi + wrap(atan2(s, c) - psi) with psi the previous P xi2.
 *  - lam_psi -= rho_psi P^T (P xi2 - psi_t)  (method-of-multipliers sign).
 *  - the xi3/xi4 step uses cos/sin of P xi2 (Eq. compute_zeta_33); the
 *    residual uses the slack rows of F (Eq. coll_con).
 *
 * Every function here is pinned by a CPU test against something other than
 * itself (exact values, scipy, brute force, closed forms, a numpy KKT solve).
 * Parity unpinned: the per-trajectory monotonicity of the residual and the
 * absolute values of the final cost, which the paper prints for no instance.
 */
#include "am_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- basis */

static double choose(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
    return c;
}

/* B_{i,N}(tau) = C(N,i) tau^i (1-tau)^(N-i); zero outside 0 <= i <= N. */
static double bern(int N, int i, double tau)
{
    if (N < 0 || i < 0 || i > N) return 0.0;
    return choose(N, i) * pow(tau, i) * pow(1.0 - tau, N - i);
}

/* Eq. param: x = P c_x with P[k][i] = B_{i,N}(t_k / T).  Derivatives use the
 * degree-lowering identities dB_{i,N}/dtau = N (B_{i-1,N-1} - B_{i,N-1}) and
 * the chain rule d/dt = (1/T) d/dtau. */
void or_bernstein(int degree, int q, double T, double *P, double *Pd, double *Pdd)
{
    const int N = degree, nv = degree + 1;
    for (int k = 0; k < q; ++k) {
        double tau = (q > 1) ? (double)k / (double)(q - 1) : 0.0;
        for (int i = 0; i < nv; ++i) {
            P[k * nv + i] = bern(N, i, tau);
            Pd[k * nv + i] = N * (bern(N - 1, i - 1, tau) - bern(N - 1, i, tau)) / T;
            Pdd[k * nv + i] = N * (N - 1) *
                              (bern(N - 2, i - 2, tau) - 2.0 * bern(N - 2, i - 1, tau) +
                               bern(N - 2, i, tau)) / (T * T);
        }
    }
}

/* ---------------------------------------------------------------- LU */

static int lu_factor(int n, double *A, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
        if (best == 0.0) return -1;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
        for (int i = k + 1; i < n; ++i) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

static void lu_solve(int n, const double *LU, const int *piv, double *x)
{
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) x[i] -= LU[i * n + j] * x[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) x[i] -= LU[i * n + j] * x[j];
        x[i] /= LU[i * n + i];
    }
}

int or_dense_solve(int n, const double *A, const double *b, double *x)
{
    double *LU = malloc(sizeof(double) * n * n);
    int *piv = malloc(sizeof(int) * n);
    memcpy(LU, A, sizeof(double) * n * n);
    memcpy(x, b, sizeof(double) * n);
    int rc = lu_factor(n, LU, piv);
    if (rc == 0) lu_solve(n, LU, piv, x);
    free(LU);
    free(piv);
    return rc;
}

/* ------------------------------------------------- closed-form xi3, xi4 */

/* Eq. zeta_2 (alpha) then Eq. compute_zeta_3 (d): the 1-D least squares of
 * (xt - a d cos alpha)^2 + (yt - b d sin alpha)^2 over d, clipped to d >= 1. */
void or_project_obstacle(double xt, double yt, double a, double b, int alpha_mode,
                         double *alpha, double *d)
{
    double al = (alpha_mode == 0) ? atan2(a * yt, b * xt) : atan2(yt, xt);
    double ca = cos(al), sa = sin(al);
    double dd = (a * xt * ca + b * yt * sa) / (a * a * ca * ca + b * b * sa * sa);
    *alpha = al;
    *d = (dd < 1.0) ? 1.0 : dd;
}

/* Eq. alpha_v and Eq. compute_dv: projection of (ux, uy) onto the circle of
 * radius d umax; d is the 1-D least squares clipped to [0, 1]. */
void or_project_bound(double ux, double uy, double umax, double *alpha, double *d)
{
    double al = atan2(uy, ux);
    double dd = (ux * cos(al) + uy * sin(al)) / umax;
    *alpha = al;
    *d = (dd < 0.0) ? 0.0 : (dd > 1.0 ? 1.0 : dd);
}

/* ---------------------------------------------------------------- setup */

typedef struct {
    int q, nv, m, n, R1, R, nx, neq, nk1, nkp;
    double *P, *Pd, *Pdd, *H, *F;
    double *K1, *Kp;       /* LU factors of the two KKT matrices */
    int *piv1, *pivp;
    double b1[24], bpsi[6];
    double *ai, *bi;       /* inflated semi-axes */
} setup_t;

int or_rows_per_side(const or_problem *pb) { return (3 + pb->m * pb->n) * pb->q; }

/* F of the display after Eq. ine_1: per side [A_v 0; A_a 0; A_ob; 0 P] acting
 * on (c_pos, c_slack); the y side repeats the x side on (c_y, c_s). */
int or_build_F(const or_problem *pb, double *F)
{
    const int q = pb->q, nv = pb->degree + 1, nx = 4 * nv;
    const int R1 = or_rows_per_side(pb);
    double *P = malloc(sizeof(double) * q * nv), *Pd = malloc(sizeof(double) * q * nv),
           *Pdd = malloc(sizeof(double) * q * nv);
    or_bernstein(pb->degree, q, pb->T, P, Pd, Pdd);
    memset(F, 0, sizeof(double) * 2 * R1 * nx);
    for (int side = 0; side < 2; ++side) {
        const int r0 = side * R1, cpos = side * 2 * nv, csl = cpos + nv;
        for (int t = 0; t < q; ++t)
            for (int k = 0; k < nv; ++k) {
                F[(r0 + t) * nx + cpos + k] = Pd[t * nv + k];          /* A_v */
                F[(r0 + q + t) * nx + cpos + k] = Pdd[t * nv + k];     /* A_a */
                for (int i = 0; i < pb->m; ++i)
                    for (int j = 0; j < pb->n; ++j) {               /* A_ob */
                        int row = r0 + 2 * q + (i * pb->n + j) * q + t;
                        F[row * nx + cpos + k] = P[t * nv + k];
                        F[row * nx + csl + k] = pb->r[i] * P[t * nv + k];
                    }
                F[(r0 + (2 + pb->m * pb->n) * q + t) * nx + csl + k] = P[t * nv + k]; /* [0 P] */
            }
    }
    free(P); free(Pd); free(Pdd);
    return 0;
}

static void free_setup(setup_t *S)
{
    free(S->P); free(S->Pd); free(S->Pdd); free(S->H); free(S->F);
    free(S->K1); free(S->Kp); free(S->piv1); free(S->pivp); free(S->ai); free(S->bi);
}

/* Boundary values of cos(psi) and sin(psi) and their first two derivatives,
 * by the chain rule, from (psi, psi', psi''). */
static void slack_boundary(const double *pbc, double *cbc, double *sbc)
{
    for (int e = 0; e < 2; ++e) {
        double p = pbc[3 * e], pd = pbc[3 * e + 1], pdd = pbc[3 * e + 2];
        double c = cos(p), s = sin(p);
        cbc[3 * e] = c;
        cbc[3 * e + 1] = -s * pd;
        cbc[3 * e + 2] = -c * pd * pd - s * pdd;
        sbc[3 * e] = s;
        sbc[3 * e + 1] = c * pd;
        sbc[3 * e + 2] = -s * pd * pd + c * pdd;
    }
}

static int make_setup(const or_problem *pb, setup_t *S)
{
    memset(S, 0, sizeof(*S));
    const int q = pb->q, nv = pb->degree + 1, nx = 4 * nv;
    S->q = q; S->nv = nv; S->m = pb->m; S->n = pb->n; S->nx = nx;
    S->R1 = or_rows_per_side(pb);
    S->R = 2 * S->R1;
    S->P = malloc(sizeof(double) * q * nv);
    S->Pd = malloc(sizeof(double) * q * nv);
    S->Pdd = malloc(sizeof(double) * q * nv);
    or_bernstein(pb->degree, q, pb->T, S->P, S->Pd, S->Pdd);

    /* H = Pdd^T Pdd: the smoothness cost of one polynomial (Eq. reform_cost). */
    S->H = calloc(nv * nv, sizeof(double));
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b)
            for (int t = 0; t < q; ++t) S->H[a * nv + b] += S->Pdd[t * nv + a] * S->Pdd[t * nv + b];

    S->F = malloc(sizeof(double) * S->R * nx);
    or_build_F(pb, S->F);

    /* A: first and last rows of P, Pd, Pdd (Eq. reform_eq). */
    double A[6 * 16];
    const int ends[2] = {0, q - 1};
    for (int e = 0; e < 2; ++e)
        for (int k = 0; k < nv; ++k) {
            A[(3 * e + 0) * nv + k] = S->P[ends[e] * nv + k];
            A[(3 * e + 1) * nv + k] = S->Pd[ends[e] * nv + k];
            A[(3 * e + 2) * nv + k] = S->Pdd[ends[e] * nv + k];
        }
    double cbc[6], sbc[6];
    slack_boundary(pb->psi_bc, cbc, sbc);

    /* xi1 KKT (Eq. over_2 with Qbar = Q + rho F^T F, Eq. zeta_1_sepration_3). */
    const int nblk = pb->cs_boundary ? 4 : 2;
    S->neq = 6 * nblk;
    const int n1 = nx + S->neq;
    S->nk1 = n1;
    S->K1 = calloc(n1 * n1, sizeof(double));
    for (int blk = 0; blk < 4; ++blk)
        for (int a = 0; a < nv; ++a)
            for (int b = 0; b < nv; ++b)
                S->K1[(blk * nv + a) * n1 + blk * nv + b] = S->H[a * nv + b];
    for (int a = 0; a < nx; ++a)
        for (int b = 0; b < nx; ++b) {
            double s = 0.0;
            for (int r = 0; r < S->R; ++r) s += S->F[r * nx + a] * S->F[r * nx + b];
            S->K1[a * n1 + b] += pb->rho * s;
        }
    /* equality rows: blocks (c_x, c_c, c_y, c_s), or (c_x, c_y) without slack rows */
    const int blocks4[4] = {0, 1, 2, 3}, blocks2[2] = {0, 2};
    const int *blocks = pb->cs_boundary ? blocks4 : blocks2;
    for (int e = 0; e < nblk; ++e) {
        int blk = blocks[e];
        const double *bv = (blk == 0) ? pb->x_bc : (blk == 1) ? cbc : (blk == 2) ? pb->y_bc : sbc;
        for (int row = 0; row < 6; ++row) {
            int rr = nx + 6 * e + row;
            for (int k = 0; k < nv; ++k) {
                S->K1[rr * n1 + blk * nv + k] = A[row * nv + k];
                S->K1[(blk * nv + k) * n1 + rr] = A[row * nv + k];
            }
            S->b1[6 * e + row] = bv[row];
        }
    }
    S->piv1 = malloc(sizeof(int) * n1);
    if (lu_factor(n1, S->K1, S->piv1) != 0) return -2;

    /* xi2 KKT (Eq. compute_convex_surrogate): [H + rho P^T P, A^T; A, 0]. */
    const int np = nv + 6;
    S->nkp = np;
    S->Kp = calloc(np * np, sizeof(double));
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
            double s = 0.0;
            for (int t = 0; t < q; ++t) s += S->P[t * nv + a] * S->P[t * nv + b];
            S->Kp[a * np + b] = S->H[a * nv + b] + pb->rho * s;
        }
    for (int row = 0; row < 6; ++row)
        for (int k = 0; k < nv; ++k) {
            S->Kp[(nv + row) * np + k] = A[row * nv + k];
            S->Kp[k * np + nv + row] = A[row * nv + k];
        }
    for (int row = 0; row < 6; ++row) S->bpsi[row] = pb->psi_bc[row];
    S->pivp = malloc(sizeof(int) * np);
    if (lu_factor(np, S->Kp, S->pivp) != 0) return -2;

    S->ai = malloc(sizeof(double) * (pb->n + 1));
    S->bi = malloc(sizeof(double) * (pb->n + 1));
    for (int j = 0; j < pb->n; ++j) {
        S->ai[j] = pb->ao[j] + pb->r_c;
        S->bi[j] = pb->bo[j] + pb->r_c;
    }
    return 0;
}

/* ------------------------------------------------------------ iteration */

typedef struct {
    double *x, *xd, *xdd, *y, *yd, *ydd, *c, *s, *psi, *psidd, *psit, *psiprev;
    double *g, *Fx, *Ftv, *rhs1, *rhsp;
} work_t;

static void matvec(const double *M, int rows, int cols, const double *v, double *out)
{
    for (int i = 0; i < rows; ++i) {
        double s = 0.0;
        for (int k = 0; k < cols; ++k) s += M[i * cols + k] * v[k];
        out[i] = s;
    }
}

static void matTvec(const double *M, int rows, int cols, const double *v, double *out)
{
    for (int k = 0; k < cols; ++k) out[k] = 0.0;
    for (int i = 0; i < rows; ++i)
        for (int k = 0; k < cols; ++k) out[k] += M[i * cols + k] * v[i];
}

/* x, y and derivatives from xi1, c and s slacks, psi and psi'' from xi2
 * (Eq. param). */
static void evaluate(const setup_t *S, const double *xi1, const double *xi2, work_t *w)
{
    const int q = S->q, nv = S->nv;
    matvec(S->P, q, nv, xi1, w->x);
    matvec(S->Pd, q, nv, xi1, w->xd);
    matvec(S->Pdd, q, nv, xi1, w->xdd);
    matvec(S->P, q, nv, xi1 + nv, w->c);
    matvec(S->P, q, nv, xi1 + 2 * nv, w->y);
    matvec(S->Pd, q, nv, xi1 + 2 * nv, w->yd);
    matvec(S->Pdd, q, nv, xi1 + 2 * nv, w->ydd);
    matvec(S->P, q, nv, xi1 + 3 * nv, w->s);
    matvec(S->P, q, nv, xi2, w->psi);
    matvec(S->Pdd, q, nv, xi2, w->psidd);
}

/* Steps xi3 and xi4 (Eq. zeta_2 - alpha_a, Eq. compute_zeta_3 - compute_da)
 * and the vector g of the display after Eq. ine_1 built from them. */
static void build_g(const or_problem *pb, const setup_t *S, work_t *w)
{
    const int q = S->q, m = S->m, n = S->n, R1 = S->R1;
    double *gx = w->g, *gy = w->g + R1;
    for (int t = 0; t < q; ++t) {
        double al, d;
        or_project_bound(w->xd[t], w->yd[t], pb->v_max, &al, &d);
        gx[t] = pb->v_max * d * cos(al);
        gy[t] = pb->v_max * d * sin(al);
        or_project_bound(w->xdd[t], w->ydd[t], pb->a_max, &al, &d);
        gx[q + t] = pb->a_max * d * cos(al);
        gy[q + t] = pb->a_max * d * sin(al);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double xt = w->x[t] + pb->r[i] * cos(w->psi[t]) - pb->xo[j * q + t];
                double yt = w->y[t] + pb->r[i] * sin(w->psi[t]) - pb->yo[j * q + t];
                or_project_obstacle(xt, yt, S->ai[j], S->bi[j], pb->alpha_mode, &al, &d);
                int row = 2 * q + (i * n + j) * q + t;
                gx[row] = pb->xo[j * q + t] + S->ai[j] * d * cos(al);
                gy[row] = pb->yo[j * q + t] + S->bi[j] * d * sin(al);
            }
        gx[(2 + m * n) * q + t] = cos(w->psi[t]);
        gy[(2 + m * n) * q + t] = sin(w->psi[t]);
    }
}

static double wrap_pi(double a)
{
    /* into (-pi, pi] */
    const double twopi = 2.0 * M_PI;
    return a - twopi * ceil((a - M_PI) / twopi);
}

static int solve_one(const or_problem *pb, const setup_t *S, int iters, double *xi1,
                     double *xi2, double *lam, double *lampsi, double *res_o,
                     double *respsi_o, double *cost_o, double *mind_o, double *hist, work_t *w)
{
    const int q = S->q, nv = S->nv, nx = S->nx, R = S->R;
    double res = 0.0, respsi = 0.0, cost = 0.0;

    /* Step 1 of Sec. III-D: xi2, xi3, xi4 initialised from the initial samples. */
    evaluate(S, xi1, xi2, w);
    build_g(pb, S, w);

    for (int k = 0; k < iters; ++k) {
        /* xi1: Eq. zeta_1_sepration_1 as Eq. over_2 with -qbar = lam + rho F^T g. */
        matTvec(S->F, R, nx, w->g, w->Ftv);
        for (int a = 0; a < nx; ++a) w->rhs1[a] = lam[a] + pb->rho * w->Ftv[a];
        for (int e = 0; e < S->neq; ++e) w->rhs1[nx + e] = S->b1[e];
        lu_solve(S->nk1, S->K1, S->piv1, w->rhs1);
        memcpy(xi1, w->rhs1, sizeof(double) * nx);

        /* xi2: Eq. compute_convex_surrogate, fitting P xi2 to atan2(s, c). */
        matvec(S->P, q, nv, xi2, w->psiprev);
        matvec(S->P, q, nv, xi1 + nv, w->c);
        matvec(S->P, q, nv, xi1 + 3 * nv, w->s);
        for (int t = 0; t < q; ++t)
            w->psit[t] = w->psiprev[t] + wrap_pi(atan2(w->s[t], w->c[t]) - w->psiprev[t]);
        matTvec(S->P, q, nv, w->psit, w->rhsp);
        for (int a = 0; a < nv; ++a) w->rhsp[a] = lampsi[a] + pb->rho * w->rhsp[a];
        for (int e = 0; e < 6; ++e) w->rhsp[nv + e] = S->bpsi[e];
        lu_solve(S->nkp, S->Kp, S->pivp, w->rhsp);
        memcpy(xi2, w->rhsp, sizeof(double) * nv);

        /* xi3 and xi4 from the new trajectory and heading. */
        evaluate(S, xi1, xi2, w);
        build_g(pb, S, w);

        /* Multipliers: Eq. update_lambda_1 and Eq. update_lambda_psi. */
        matvec(S->F, R, nx, xi1, w->Fx);
        res = 0.0;
        for (int r = 0; r < R; ++r) {
            w->Fx[r] -= w->g[r];
            res += w->Fx[r] * w->Fx[r];
        }
        res = sqrt(res);
        matTvec(S->F, R, nx, w->Fx, w->Ftv);
        for (int a = 0; a < nx; ++a) lam[a] -= pb->rho * w->Ftv[a];

        respsi = 0.0;
        for (int t = 0; t < q; ++t) {
            w->psit[t] = w->psi[t] - w->psit[t];  /* P xi2 - psi_t */
            respsi += w->psit[t] * w->psit[t];
        }
        respsi = sqrt(respsi);
        matTvec(S->P, q, nv, w->psit, w->rhsp);
        const double sgn = pb->psi_dual_sign ? -1.0 : 1.0;
        for (int a = 0; a < nv; ++a) lampsi[a] -= sgn * pb->rho_psi * w->rhsp[a];

        /* Cost of Eq. acc_cost on the grid. */
        cost = 0.0;
        for (int t = 0; t < q; ++t)
            cost += w->xdd[t] * w->xdd[t] + w->ydd[t] * w->ydd[t] + w->psidd[t] * w->psidd[t];

        if (hist) {
            hist[3 * k] = res;
            hist[3 * k + 1] = respsi;
            hist[3 * k + 2] = cost;
        }
    }

    /* Smallest ellipse distance of any circle to any obstacle (Eq. coll_multiagent
     * reads it as >= 1) on the final trajectory and heading. */
    double mind = INFINITY;
    for (int t = 0; t < q; ++t)
        for (int i = 0; i < S->m; ++i)
            for (int j = 0; j < S->n; ++j) {
                double xt = w->x[t] + pb->r[i] * cos(w->psi[t]) - pb->xo[j * q + t];
                double yt = w->y[t] + pb->r[i] * sin(w->psi[t]) - pb->yo[j * q + t];
                double dd = sqrt(xt * xt / (S->ai[j] * S->ai[j]) + yt * yt / (S->bi[j] * S->bi[j]));
                if (dd < mind) mind = dd;
            }
    if (res_o) *res_o = res;
    if (respsi_o) *respsi_o = respsi;
    if (cost_o) *cost_o = cost;
    if (mind_o) *mind_o = mind;
    return 0;
}

static double *alloc0(size_t n) { return calloc(n ? n : 1, sizeof(double)); }

int or_solve(const or_problem *pb, int B, int iters, double *xi1_io, double *xi2_io,
             double *lam_io, double *lampsi_io, double *res, double *res_psi,
             double *cost, double *mind, double *hist, int nthreads)
{
    if (!pb || B < 0 || iters < 1 || pb->q < 2 || pb->degree < 2 || pb->degree > 15 ||
        pb->m < 1 || pb->n < 0 || pb->T <= 0.0)
        return -1;
    setup_t S;
    int rc = make_setup(pb, &S);
    if (rc != 0) { free_setup(&S); return rc; }
    const int nv = S.nv, nx = S.nx, q = S.q;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        work_t w;
        w.x = alloc0(q); w.xd = alloc0(q); w.xdd = alloc0(q);
        w.y = alloc0(q); w.yd = alloc0(q); w.ydd = alloc0(q);
        w.c = alloc0(q); w.s = alloc0(q); w.psi = alloc0(q); w.psidd = alloc0(q);
        w.psit = alloc0(q); w.psiprev = alloc0(q);
        w.g = alloc0(S.R); w.Fx = alloc0(S.R); w.Ftv = alloc0(nx);
        w.rhs1 = alloc0(S.nk1); w.rhsp = alloc0(S.nkp);
#pragma omp for schedule(dynamic, 1)
        for (int l = 0; l < B; ++l) {
            solve_one(pb, &S, iters, xi1_io + (size_t)l * nx, xi2_io + (size_t)l * nv,
                      lam_io + (size_t)l * nx, lampsi_io + (size_t)l * nv,
                      res ? res + l : NULL, res_psi ? res_psi + l : NULL,
                      cost ? cost + l : NULL, mind ? mind + l : NULL,
                      hist ? hist + (size_t)l * iters * 3 : NULL, &w);
        }
        free(w.x); free(w.xd); free(w.xdd); free(w.y); free(w.yd); free(w.ydd);
        free(w.c); free(w.s); free(w.psi); free(w.psidd); free(w.psit); free(w.psiprev);
        free(w.g); free(w.Fx); free(w.Ftv); free(w.rhs1); free(w.rhsp);
    }
    free_setup(&S);
    return 0;
}
