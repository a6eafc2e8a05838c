/*
 * A plain-C client of libtrajam: one solve through the C ABI alone, with no
 * Python and no torch in the process.  Used by tests/test_c_client.py.
 *
 * usage: am_client IN OUT
 *
 * IN (little-endian): int32 q, m, n, B, iters, kernel; float64 T, r_c, v_max,
 * a_max, rho, rho_psi, x_bc[6], y_bc[6], psi_bc[6], r[m]; float32 xo[n q],
 * yo[n q], a[n], b[n], init[B 33].
 * OUT: float32 state[B AM_STATE_FLOATS], res[B], res_psi[B], cost[B],
 * mind[B], then index (as a float), cost, residual and the 33 coefficients
 * of the best trajectory.
 *
 * Exit status: 0 on success, 1 on a usage or file error, 2 on a library
 * error (its message on stderr).
 */
#include <stdio.h>
#include <stdlib.h>

#include "trajam.h"

static int read_all(FILE *f, void *p, size_t size, size_t count)
{
    return fread(p, size, count, f) == count;
}

static int check(int rc, const char *what)
{
    if (rc != AM_OK) fprintf(stderr, "%s failed (%d): %s\n", what, rc, am_last_error());
    return rc == AM_OK;
}

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s IN OUT\n", argv[0]);
        return 1;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 1;
    int hdr[6];
    double sc[6], bc[18];
    if (!read_all(in, hdr, sizeof(int), 6) || !read_all(in, sc, sizeof(double), 6) ||
        !read_all(in, bc, sizeof(double), 18)) {
        fclose(in);
        return 1;
    }
    const int q = hdr[0], m = hdr[1], n = hdr[2], B = hdr[3], iters = hdr[4], kernel = hdr[5];
    if (q < 2 || m < 1 || n < 0 || B < 1 || iters < 1) {
        fclose(in);
        return 1;
    }
    double *r = malloc(sizeof(double) * (size_t)m);
    float *xo = malloc(sizeof(float) * ((size_t)n * q + 1)), *yo = malloc(sizeof(float) * ((size_t)n * q + 1));
    float *a = malloc(sizeof(float) * ((size_t)n + 1)), *b = malloc(sizeof(float) * ((size_t)n + 1));
    float *init = malloc(sizeof(float) * (size_t)B * 33);
    const size_t out_floats = (size_t)B * AM_STATE_FLOATS + 4 * (size_t)B + 36;
    float *out = malloc(sizeof(float) * out_floats);
    int ok = r && xo && yo && a && b && init && out && read_all(in, r, sizeof(double), (size_t)m) &&
             read_all(in, xo, sizeof(float), (size_t)n * q) && read_all(in, yo, sizeof(float), (size_t)n * q) &&
             read_all(in, a, sizeof(float), (size_t)n) && read_all(in, b, sizeof(float), (size_t)n) &&
             read_all(in, init, sizeof(float), (size_t)B * 33);
    fclose(in);
    int status = ok ? 0 : 1;
    am_problem *h = NULL;
    if (ok) {
        am_problem_desc d;
        d.q = q;
        d.T = sc[0];
        d.degree = 10;
        d.m = m;
        d.r = r;
        d.r_c = sc[1];
        d.v_max = sc[2];
        d.a_max = sc[3];
        d.rho = sc[4];
        d.rho_psi = sc[5];
        for (int i = 0; i < 6; ++i) {
            d.x_bc[i] = bc[i];
            d.y_bc[i] = bc[6 + i];
            d.psi_bc[i] = bc[12 + i];
        }
        d.precision = AM_FP32;
        d.alpha_mode = 0;
        d.psi_dual_sign = 0;
        d.cs_boundary = 1;
        float *state = out, *res = out + (size_t)B * AM_STATE_FLOATS;
        float *best = res + 4 * (size_t)B;
        float best_cost = 0.f, best_res = 0.f;
        int best_idx = -1;
        ok = check(am_init_problem(&d, &h), "am_init_problem") &&
             check(am_set_option(h, AM_OPT_KERNEL, kernel), "am_set_option") &&
             (n == 0 || check(am_set_obstacles(h, n, xo, yo, a, b, AM_HOST), "am_set_obstacles")) &&
             check(am_solve_batch(h, B, init, NULL, iters, NULL, AM_HOST), "am_solve_batch") &&
             check(am_get_results(h, res, res + B, res + 2 * (size_t)B, res + 3 * (size_t)B, AM_HOST),
                   "am_get_results") &&
             check(am_get_best(h, best + 3, &best_cost, &best_res, &best_idx), "am_get_best") &&
             check(am_get_state(h, state, AM_HOST), "am_get_state");
        if (ok) {
            best[0] = (float)best_idx;
            best[1] = best_cost;
            best[2] = best_res;
            FILE *o = fopen(argv[2], "wb");
            ok = o && fwrite(out, sizeof(float), out_floats, o) == out_floats;
            if (o) fclose(o);
            status = ok ? 0 : 1;
        } else {
            status = 2;
        }
        if (h) am_destroy(h);
    }
    free(r);
    free(xo);
    free(yo);
    free(a);
    free(b);
    free(init);
    free(out);
    return status;
}
