/*
 * FP64 CPU oracle of the batched alternating-minimization (AM) loop of
 * "GPU Accelerated Batch Multi-Convex Trajectory Optimization for a
 * Rectangular Holonomic Mobile Robot" (arXiv 2109.13030).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Layout conventions (all row-major, double precision):
 *   basis matrices P, Pd, Pdd        q x nv     (nv = degree + 1)
 *   xi1 per trajectory               [c_x, c_c, c_y, c_s]   4*nv
 *   xi2 per trajectory               c_psi                  nv
 *   lambda per trajectory            4*nv
 *   lambda_psi per trajectory        nv
 *   obstacle tracks xo, yo           n x q
 */
#ifndef AM_ORACLE_H
#define AM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int q;              /* planning steps                                  */
    double T;           /* horizon in seconds; t_k = k T / (q - 1)         */
    int degree;         /* Bernstein degree; nv = degree + 1               */
    int m;              /* robot circles                                   */
    const double *r;    /* m body-frame offsets r_i along the heading      */
    double r_c;         /* circle radius, added to each obstacle semi-axis */
    int n;              /* obstacles                                       */
    const double *xo, *yo;  /* n x q obstacle centre tracks                */
    const double *ao, *bo;  /* n obstacle semi-axes (before inflation)     */
    double v_max, a_max, rho, rho_psi;
    double x_bc[6], y_bc[6], psi_bc[6];  /* value, 1st, 2nd derivative at t=0, then at t=T */
    int alpha_mode;     /* 0: alpha = atan2(a*yt, b*xt); 1: atan2(yt, xt)  */
    int psi_dual_sign;  /* 0: lam_psi -= rho_psi P^T (P xi2 - psi_t); 1: opposite sign */
    int cs_boundary;    /* 1: slack blocks c, s carry boundary rows; 0: they do not */
} or_problem;

/* Bernstein basis of the given degree and its first and second time
 * derivatives on t_k = k T / (q - 1).  Each output is q x (degree + 1). */
void or_bernstein(int degree, int q, double T, double *P, double *Pd, double *Pdd);

/* Dense solve of A x = b (n x n, row-major) by LU with partial pivoting.
 * Returns 0 on success, -1 on a zero pivot.  A and b are not modified. */
int or_dense_solve(int n, const double *A, const double *b, double *x);

/* Closed-form alpha and d of one collision pair (Eq. zeta_2 and Eq.
 * compute_zeta_3): (xt, yt) is the offset of a robot circle from the obstacle
 * centre, (a, b) the inflated semi-axes. d is clipped to d >= 1. */
void or_project_obstacle(double xt, double yt, double a, double b, int alpha_mode,
                         double *alpha, double *d);

/* Closed-form alpha and d of the velocity or acceleration bound (Eq. alpha_v,
 * Eq. compute_dv): (ux, uy) is the velocity (or acceleration), umax its
 * bound. d is clipped to [0, 1]. */
void or_project_bound(double ux, double uy, double umax, double *alpha, double *d);

/* Rows of F per side, (3 + m n) q, and the dense F (2 rows-per-side x 4 nv). */
int or_rows_per_side(const or_problem *pb);
int or_build_F(const or_problem *pb, double *F);

/* The AM loop for B trajectories.
 *  xi1_io   B x 4nv   in: initial coefficients (the c, s blocks are unused),
 *                     out: final xi1
 *  xi2_io   B x nv    in: initial c_psi, out: final
 *  lam_io   B x 4nv   in/out (in: zeros for a cold start)
 *  lampsi_io B x nv   in/out
 *  res, res_psi, cost, mind   B each (may be NULL): last iteration's
 *                     ||F xi1 - g||, ||P xi2 - psi_t||, sum_t xdd^2+ydd^2+psidd^2,
 *                     min over circles/obstacles/steps of the ellipse distance
 *  hist     B x iters x 3 (may be NULL): res, res_psi, cost per iteration
 *  nthreads OpenMP threads (0: runtime default)
 * Returns 0, or -1 on bad arguments, -2 on a singular KKT matrix. */
int or_solve(const or_problem *pb, int B, int iters, double *xi1_io, double *xi2_io,
             double *lam_io, double *lampsi_io, double *res, double *res_psi,
             double *cost, double *mind, double *hist, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
