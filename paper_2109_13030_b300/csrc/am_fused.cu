// Fused persistent kernel of the batched alternating-minimization loop
// (Sec. III-D, steps 1-5, and the batch solution of Sec. III-E).
//
// One CTA stays resident on each SM and works through tiles of T trajectories.
// It stages the constant block into shared memory once (bulk async copy,
// completion on an mbarrier), keeps xi1, xi2, lambda, lambda_psi and the
// residual contraction R = F^T (g - F xi1) of every trajectory of the tile in
// shared memory for all iterations, and writes the state back only after the
// last one.  Nothing per element (alpha, d, g) is ever stored.
//
// The position step of Eq. over_3, xi1' = Minv (lam + rho F^T g) + kb, is
// evaluated in the algebraically equal increment form
//     xi1' = xi1 + Minv (lam - Q xi1 + rho F^T (g - F xi1))
// (from Minv Qbar + N A = I, kb = N b and A xi1 = b), so FP32 works on the
// small constraint residual instead of on |F^T g| ~ 1e3, which the explicit
// inverse would amplify by its conditioning.  The multiplier update of
// Eq. update_lambda_1 is lam' = lam + rho R with the same R.  A solve starts
// from a reference xi1 whose boundary control points are set from the
// boundary conditions, so A xi1 = b holds from the first step on.
//
// Thread roles inside a tile (all threads run every phase; idle ones skip):
//   per-step phases   thread <-> (trajectory tt, step t), tt*q + t < T*q
//   dot phases        thread <-> (trajectory, output, part) tasks
// Phases of one iteration, separated by __syncthreads():
//   XI1   lam += rho R; xi1 += Minv (lam - Q xi1 + rho R); lambda_psi update
//         (Eq. update_lambda_psi); per-trajectory sums of the last sweep
//   EVAL  x, xdot, xddot, y, ..., c, s at step t (Eq. param); psi_t target
//   PSI   xi2 = Mpsi lam_psi + kbpsi + rho W^T psi_t (Eq. compute_convex_surrogate)
//   SWEEP psi = P xi2; the closed-form alpha/d steps for every circle and
//         obstacle (Eq. zeta_2 - compute_da) in the trig-free form
//         (xt, yt) * max(1, 1/sqrt(xt^2/a^2 + yt^2/b^2)), the velocity and
//         acceleration projections, and the per-step residual vectors of R
//   DOT   R per side: Pd^T rv + Pdd^T ra + P^T r0 and P^T r1
#include <cuda_runtime.h>

#include <cstdint>

#include "am_internal.h"

namespace trajam {
namespace {

constexpr int kMaxThreads = 768;
constexpr int kVecs = 12;       // per-step vectors in G
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kPi = 3.14159265358979323846f;

struct Smem {
    int cst, xi1, lam, rb, xi2, dx2, lps, ptp, G, psit, bar, total;  // float offsets
};

__host__ __device__ inline Smem smem_layout(const ConstLayout &L, int T)
{
    Smem s;
    int o = 0;
    s.cst = o; o += L.total;
    s.xi1 = o; o += 2 * T * 48;
    s.lam = o; o += 2 * T * 48;
    s.rb = o; o += T * 48;
    s.xi2 = o; o += 2 * T * 12;   // double-buffered c_psi
    s.dx2 = o; o += T * 12;       // last heading increment
    s.lps = o; o += T * 12;
    s.ptp = o; o += T * 12;
    s.G = o; o += T * kVecs * L.qs;
    s.psit = o; o += T * L.qs;
    o = (o + 3) & ~3;
    s.bar = o; o += 4;  // one 8-byte mbarrier, kept 16-byte aligned
    s.total = o;
    return s;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bulk async copy global -> shared, completion counted on an mbarrier.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Side-row r (0..21) of (c_pos, c_slack) -> padded index within a 24-float side block.
__device__ __forceinline__ int rowpad(int r) { return r < NV ? r : r + 1; }

__device__ __forceinline__ float dot11(const float *a, const float *b)
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NV; ++k) s = fmaf(a[k], b[k], s);
    return s;
}

__device__ __forceinline__ void load12(float (&r)[12], const float *p)
{
    const float4 *v = reinterpret_cast<const float4 *>(p);
    float4 a = v[0], b = v[1], c = v[2];
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
}

// Wrap into (-pi, pi].
__device__ __forceinline__ float wrap_pi(float a)
{
    return a - kTwoPi * ceilf((a - kPi) * (1.0f / kTwoPi));
}

struct Tile {
    int first, count;  // trajectories [first, first + count)
};

struct KParams {
    const float *cblob;
    ConstLayout L;
    int B, iters, T, ntiles;
    float *state, *res, *res_psi, *cost, *mind, *hist;
    int *err;
};

__device__ __forceinline__ Tile tile_of(int i, int B, int ntiles)
{
    const long long lo = (long long)i * B / ntiles, hi = (long long)(i + 1) * B / ntiles;
    return {int(lo), int(hi - lo)};
}

// ----------------------------------------------------------------- phases

// XI1 phase: the multiplier update of the finished iteration, the next xi1 in
// increment form, the lambda_psi update and the per-trajectory sums.
//   first: lam' = lam,          xi1' = xi1 + Minv (lam + rho R) - MQ xi1
//   later: lam' = lam + rho R,  xi1' = xi1 + Minv (lam + 2 rho R) - MQ xi1
//   post (no solve): lam' = lam + rho R, xi1' = xi1
__device__ void phase_xi1(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur,
                          bool first, bool solve, bool sums, bool final_out, int kprev)
{
    const ConstLayout &L = p.L;
    const float *cst = sm + S.cst;
    const float rho = L.rho;
    const int Tn = tl.count;
    const int n_xi = Tn * 44, n_lp = Tn * NV, n_sc = sums ? Tn * 4 : 0;
    const int ntask = n_xi + n_lp + n_sc;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        if (task < n_xi) {
            const int tt = task / 44, rem = task - 44 * tt, side = rem / NS, row = rem - NS * side;
            const float *lam = sm + S.lam + (cur * p.T + tt) * 48 + 24 * side;
            const float *xi = sm + S.xi1 + (cur * p.T + tt) * 48 + 24 * side;
            const float *R = sm + S.rb + tt * 48 + 24 * side;
            float *lam_n = sm + S.lam + ((cur ^ 1) * p.T + tt) * 48 + 24 * side;
            float *xi_n = sm + S.xi1 + ((cur ^ 1) * p.T + tt) * 48 + 24 * side;
            const int rp = rowpad(row);
            float xn = xi[rp];
            if (solve) {
                const float coef = first ? rho : 2.f * rho;
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int c = 0; c < NS; ++c) {
                    const int cp = rowpad(c);
                    a0 = fmaf(cst[L.off_mt + c * 24 + row], fmaf(coef, R[cp], lam[cp]), a0);
                    a1 = fmaf(cst[L.off_mq + c * 24 + row], xi[cp], a1);
                }
                xn += a0 - a1;
            }
            xi_n[rp] = xn;
            lam_n[rp] = first ? lam[rp] : fmaf(rho, R[rp], lam[rp]);
        } else if (task < n_xi + n_lp) {
            if (first) continue;
            // P^T (P xi2' - psi_t) = P^T P dxi2 - P^T delta, delta = psi_t - P xi2
            const int s = task - n_xi, tt = s / NV, k = s - NV * tt;
            const float *dx2 = sm + S.dx2 + tt * 12;
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < NV; ++c) a = fmaf(cst[L.off_ptp + c * 12 + k], dx2[c], a);
            float *lp = sm + S.lps + tt * 12;
            lp[k] -= L.psi_sign * L.rho_psi * (a - sm[S.ptp + tt * 12 + k]);
        } else {
            const int s = task - n_xi - n_lp, tt = s >> 2, w = s & 3;
            const float *gv = sm + S.G + (tt * kVecs + 8 + w) * L.qs;
            float v;
            if (w < 3) {
                const float4 *g = reinterpret_cast<const float4 *>(gv);
                float a0 = 0.f, a1 = 0.f;
                for (int i = 0; i < L.qs / 4; ++i) {  // padding past q is zero
                    const float4 x = g[i];
                    a0 += x.x + x.y;
                    a1 += x.z + x.w;
                }
                v = a0 + a1;
                if (w < 2) v = sqrtf(v);
            } else {
                if (!final_out) continue;
                float mn = 3.0e38f;
                for (int t = 0; t < L.q; ++t) mn = fminf(mn, gv[t]);
                v = sqrtf(mn);
            }
            const int traj = tl.first + tt;
            if (p.hist && w < 3) p.hist[((size_t)traj * p.iters + kprev) * 3 + w] = v;
            if (final_out) {
                float *dst = w == 0 ? p.res : w == 1 ? p.res_psi : w == 2 ? p.cost : p.mind;
                dst[traj] = v;
            }
        }
    }
}

// DOT phase: R = F^T (g - F xi1) per trajectory and side from the per-step
// residual vectors.  Task = (trajectory, side, k, part); parts 0..2 contract
// rv, ra, r0 with Pd, Pdd, P and are summed into the c_pos row k; part 3
// contracts r1 with P into the c_slack row k.
__device__ void phase_dot(const KParams &p, float *sm, const Smem &S, const Tile &tl)
{
    const ConstLayout &L = p.L;
    const int ntask = tl.count * 88;
    const int q4 = L.qs / 4;
    for (int base = 0; base < ntask; base += blockDim.x) {
        const int task = base + threadIdx.x;
        float tot = 0.f;
        int tt = 0, side = 0, k = 0, part = 0;
        if (task < ntask) {
            part = task & 3;
            const int g = task >> 2;
            tt = g / NS;
            const int rem = g - NS * tt;
            side = rem / NV;
            k = rem - NV * side;
            const int bsel = part == 0 ? 1 : part == 1 ? 2 : 0;
            const float4 *col = reinterpret_cast<const float4 *>(sm + S.cst + L.off_pcol + (bsel * NV + k) * L.qs);
            const float4 *vec = reinterpret_cast<const float4 *>(sm + S.G + (tt * kVecs + 4 * side + part) * L.qs);
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 5
            for (int i = 0; i < q4; ++i) {
                const float4 a = vec[i], b = col[i];
                a0 = fmaf(a.x, b.x, a0);
                a1 = fmaf(a.y, b.y, a1);
                a2 = fmaf(a.z, b.z, a2);
                a3 = fmaf(a.w, b.w, a3);
            }
            tot = (a0 + a1) + (a2 + a3);
        }
        const float s1 = __shfl_down_sync(0xffffffffu, tot, 1);
        const float s2 = __shfl_down_sync(0xffffffffu, tot, 2);
        if (task < ntask) {
            float *R = sm + S.rb + tt * 48 + 24 * side;
            if (part == 0) R[k] = tot + s1 + s2;
            else if (part == 3) R[12 + k] = tot;
        }
    }
}

// PSI phase: the heading step of Eq. compute_convex_surrogate in increment form,
//   xi2' = xi2 + Mpsi (lam_psi - H xi2) + rho W^T delta,  W = P Mpsi^T,
// with delta = psi_t - P xi2 per step (equal to Mpsi (lam_psi + rho P^T psi_t)
// + kbpsi when A xi2 = b_psi), plus P^T delta for the multiplier update.
// Task = (trajectory, output kk in 0..21, chunk 0..3); the four chunks of one
// output sit in adjacent lanes and are summed with shuffles.
__device__ void phase_psi(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur2)
{
    const ConstLayout &L = p.L;
    const float *cst = sm + S.cst;
    const int ntask = tl.count * 88;
    const int q4 = L.qs / 4;
    for (int base = 0; base < ntask; base += blockDim.x) {
        const int task = base + threadIdx.x;
        float tot = 0.f;
        int tt = 0, kk = 0, chunk = 0;
        if (task < ntask) {
            chunk = task & 3;
            const int g = task >> 2;
            tt = g / NS;
            kk = g - NS * tt;
            const float4 *col = reinterpret_cast<const float4 *>(
                cst + (kk < NV ? L.off_wcol + kk * L.qs : L.off_pcol + (kk - NV) * L.qs));
            const float4 *ps = reinterpret_cast<const float4 *>(sm + S.psit + tt * L.qs);
            float a0 = 0.f, a1 = 0.f;
            for (int i = chunk; i < q4; i += 4) {
                const float4 a = ps[i], b = col[i];
                a0 = fmaf(a.x, b.x, a0);
                a1 = fmaf(a.y, b.y, a1);
                a0 = fmaf(a.z, b.z, a0);
                a1 = fmaf(a.w, b.w, a1);
            }
            tot = a0 + a1;
        }
        tot += __shfl_xor_sync(0xffffffffu, tot, 1);
        tot += __shfl_xor_sync(0xffffffffu, tot, 2);
        if (task < ntask && chunk == 0) {
            if (kk < NV) {
                const float *lp = sm + S.lps + tt * 12;
                const float *x2 = sm + S.xi2 + (cur2 * p.T + tt) * 12;
                float b0 = 0.f, b1 = 0.f;
#pragma unroll
                for (int c = 0; c < NV; ++c) {
                    b0 = fmaf(cst[L.off_mpsi + c * 12 + kk], lp[c], b0);
                    b1 = fmaf(cst[L.off_mpsih + c * 12 + kk], x2[c], b1);
                }
                const float d = fmaf(L.rho, tot, b0 - b1);
                sm[S.dx2 + tt * 12 + kk] = d;
                sm[S.xi2 + ((cur2 ^ 1) * p.T + tt) * 12 + kk] = x2[kk] + d;
            } else {
                sm[S.ptp + tt * 12 + (kk - NV)] = tot;
            }
        }
    }
}

struct StepRegs {
    float x, xd, xdd, y, yd, ydd, c, s;
    float psi_t;     // heading target atan2(s, c), unwrapped
    float psi_prev;  // heading the unwrap refers to (the previous P xi2)
    float psi_cur;   // P xi2 of the current coefficients
};

// EVAL: trajectory values at this thread's step from a padded xi1 block.
__device__ __forceinline__ void eval_xy(const float *sm, const Smem &S, const ConstLayout &L,
                                        const float *xi, int t, const float (&Prow)[12],
                                        StepRegs &r)
{
    float pd[12], pdd[12], cx[12], cc[12], cy[12], cs[12];
    load12(pd, sm + S.cst + L.off_prow + (1 * L.q + t) * 12);
    load12(pdd, sm + S.cst + L.off_prow + (2 * L.q + t) * 12);
    load12(cx, xi);
    load12(cc, xi + 12);
    load12(cy, xi + 24);
    load12(cs, xi + 36);
    r.x = dot11(Prow, cx);
    r.xd = dot11(pd, cx);
    r.xdd = dot11(pdd, cx);
    r.c = dot11(Prow, cc);
    r.y = dot11(Prow, cy);
    r.yd = dot11(pd, cy);
    r.ydd = dot11(pdd, cy);
    r.s = dot11(Prow, cs);
}

// SWEEP: heading at this step, the closed-form xi3/xi4 steps for every
// (circle, obstacle) pair and the bounds, and the per-step residual vectors
// (g - F xi1 summed per row block).  g is built from r; F xi1 from ref when
// PRO (first step of a solve: g from the initial samples, F xi1 from the
// boundary-consistent reference), else from r as well.
// RES also accumulates the step's squared residual and cost; FIN the smallest
// squared ellipse distance.
template <int M, bool LIT, bool RES, bool FIN, bool PRO>
__device__ __forceinline__ void sweep(float *sm, const Smem &S, const ConstLayout &L, const float *xi2,
                                      int t, int tt, const float (&Prow)[12], StepRegs &r,
                                      const StepRegs &ref)
{
    const float *cst = sm + S.cst;
    float x2[12];
    load12(x2, xi2);
    const float psi = dot11(Prow, x2);
    float psidd = 0.f;
    if (RES) {
        float pdd[12];
        load12(pdd, cst + L.off_prow + (2 * L.q + t) * 12);
        psidd = dot11(pdd, x2);
    }
    const float pr = psi - kTwoPi * rintf(psi * (1.0f / kTwoPi));
    const float cp = __cosf(pr), sp = __sinf(pr);
    const float cf = PRO ? ref.c : r.c, sf = PRO ? ref.s : r.s;   // slack values of F xi1

    // velocity and acceleration: project onto the disc of radius v_max / a_max
    const float v2 = fmaf(r.xd, r.xd, r.yd * r.yd);
    const float sv = fminf(1.f, L.v_max * rsqrtf(v2));
    const float a2 = fmaf(r.xdd, r.xdd, r.ydd * r.ydd);
    const float sa = fminf(1.f, L.a_max * rsqrtf(a2));

    float X[M], Y[M], ax[M], ay[M], ee[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        X[i] = fmaf(L.r[i], cp, r.x);
        Y[i] = fmaf(L.r[i], sp, r.y);
        ax[i] = 0.f;
        ay[i] = 0.f;
        ee[i] = 0.f;
    }
    float dmin = 3.0e38f;
    const float2 *obs = reinterpret_cast<const float2 *>(cst + L.off_obs);
    const float4 *obc = reinterpret_cast<const float4 *>(cst + L.off_obc);
    const int n = L.n;
    for (int j = 0; j < n; ++j) {
        const float2 o = obs[j * L.qs + t];   // (x_j(t)/a_j, y_j(t)/b_j)
        const float4 c = obc[j];              // (1/a_j, 1/b_j, a_j, b_j)
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float xh = fmaf(X[i], c.x, -o.x);   // (x + r_i cos psi - x_j) / a_j
            const float yh = fmaf(Y[i], c.y, -o.y);
            const float D = fmaf(xh, xh, fmaf(yh, yh, 1e-30f));
            float tx, ty;
            if (!LIT) {
                const float h = fmaxf(rsqrtf(D), 1.f) - 1.f;  // max(1, 1/d) - 1
                tx = xh * h;
                ty = yh * h;
            } else {
                // printed alpha = atan2(yt, xt): the point (a d cos, b d sin) with
                // d = max(1, rho (a xt^2 + b yt^2) / (a^2 xt^2 + b^2 yt^2)), rho = |(xt, yt)|
                const float xt = c.z * xh, yt = c.w * yh;
                const float r2 = fmaf(xt, xt, yt * yt);
                const float u = c.z * xt, v = c.w * yt;
                const float den = fmaf(u, u, v * v);
                if (r2 > 0.f) {
                    const float ir = rsqrtf(r2);
                    const float d = fmaxf(1.f, r2 * ir * fmaf(c.z, xt * xt, c.w * yt * yt) / den);
                    tx = (d * ir * u - xt) * c.x;  // offset, scaled back by 1/a (e = a tx)
                    ty = (d * ir * v - yt) * c.y;
                } else {
                    tx = 1.f;  // alpha = atan2(0, 0) = 0, d = 1: point (a, 0)
                    ty = 0.f;
                }
            }
            if (RES) {
                const float ex = c.z * tx, ey = c.w * ty;
                ax[i] += ex;
                ay[i] += ey;
                ee[i] = fmaf(ex, ex, fmaf(ey, ey, ee[i]));
            } else {
                ax[i] = fmaf(c.z, tx, ax[i]);  // e_ij = projected point - (xt, yt)
                ay[i] = fmaf(c.w, ty, ay[i]);
            }
            if (FIN) dmin = fminf(dmin, D);
        }
    }
    // Obstacle rows: g_ij - (x + r_i c) = r_i (cos psi - c) + e_ij (+ x - x_ref in PRO)
    const float fn = float(n);
    const float dxp = PRO ? r.x - ref.x : 0.f, dyp = PRO ? r.y - ref.y : 0.f;
    const float dcx = cp - cf, dsy = sp - sf;
    float r0x = 0.f, r1x = 0.f, r0y = 0.f, r1y = 0.f, rob = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const float bx = fn * fmaf(L.r[i], dcx, dxp) + ax[i];
        const float by = fn * fmaf(L.r[i], dsy, dyp) + ay[i];
        r0x += bx;
        r0y += by;
        r1x = fmaf(L.r[i], bx, r1x);
        r1y = fmaf(L.r[i], by, r1y);
        if (RES) {
            // sum_j (r_i (c - cos psi) - e_ij)^2, expanded
            const float dx = L.r[i] * dcx, dy = L.r[i] * dsy;
            rob += fn * fmaf(dx, dx, dy * dy) + 2.f * fmaf(dx, ax[i], dy * ay[i]) + ee[i];
        }
    }
    float *G = sm + S.G + tt * kVecs * L.qs + t;
    const int qs = L.qs;
    const float svm = sv - 1.f, sam = sa - 1.f;
    // v and a rows: projected value - F xi1 value
    G[0 * qs] = PRO ? fmaf(r.xd, svm, r.xd - ref.xd) : r.xd * svm;
    G[1 * qs] = PRO ? fmaf(r.xdd, sam, r.xdd - ref.xdd) : r.xdd * sam;
    G[2 * qs] = r0x;
    G[3 * qs] = r1x + dcx;
    G[4 * qs] = PRO ? fmaf(r.yd, svm, r.yd - ref.yd) : r.yd * svm;
    G[5 * qs] = PRO ? fmaf(r.ydd, sam, r.ydd - ref.ydd) : r.ydd * sam;
    G[6 * qs] = r0y;
    G[7 * qs] = r1y + dsy;
    if (RES) {
        G[8 * qs] = v2 * svm * svm + a2 * sam * sam + rob + dcx * dcx + dsy * dsy;
        const float dp = psi - r.psi_t;
        G[9 * qs] = dp * dp;
        G[10 * qs] = fmaf(r.xdd, r.xdd, fmaf(r.ydd, r.ydd, psidd * psidd));
    }
    if (FIN) G[11 * qs] = dmin;
    r.psi_prev = psi;
    r.psi_cur = psi;
}

template <int M, bool LIT>
__device__ void sweep_dispatch(float *sm, const Smem &S, const ConstLayout &L, const float *xi2,
                               int tt, int t, const float (&Prow)[12], StepRegs &r, bool res,
                               bool fin)
{
    if (fin) sweep<M, LIT, true, true, false>(sm, S, L, xi2, t, tt, Prow, r, r);
    else if (res) sweep<M, LIT, true, false, false>(sm, S, L, xi2, t, tt, Prow, r, r);
    else sweep<M, LIT, false, false, false>(sm, S, L, xi2, t, tt, Prow, r, r);
}

template <int M, bool LIT>
__global__ void __launch_bounds__(kMaxThreads, 1) am_fused_kernel(KParams p)
{
    extern __shared__ __align__(128) float sm[];
    const ConstLayout &L = p.L;
    const Smem S = smem_layout(L, p.T);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S.bar);

    // Stage the constant block once per CTA.
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = uint32_t(L.total) * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
        bulk_load(sm + S.cst, p.cblob, bytes, bar);
    }
    // zero the per-step buffers (their padding past q must read as zero)
    for (int i = threadIdx.x; i < p.T * (kVecs + 1) * L.qs; i += blockDim.x) sm[S.G + i] = 0.f;
    for (int i = threadIdx.x; i < 2 * p.T * 48; i += blockDim.x) {
        sm[S.xi1 + i] = 0.f;
        sm[S.lam + i] = 0.f;
    }
    for (int i = threadIdx.x; i < p.T * 48; i += blockDim.x) sm[S.rb + i] = 0.f;
    for (int i = threadIdx.x; i < p.T * 12; i += blockDim.x) {
        sm[S.xi2 + i] = 0.f;
        sm[S.xi2 + p.T * 12 + i] = 0.f;
        sm[S.dx2 + i] = 0.f;
        sm[S.lps + i] = 0.f;
    }
    // Bounded wait for the staged constants; the block agrees on the outcome
    // before anyone leaves, so no thread is left waiting at a barrier.
    int ok = 0;
    for (int spin = 0; spin < (1 << 24) && !ok; ++spin) ok = mbar_try_wait(bar, 0) ? 1 : 0;
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicExch(p.err, 1);
        return;
    }

    for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
        const Tile tl = tile_of(tile, p.B, p.ntiles);
        const int Tn = tl.count;
        // The tile's state: xi1 as given into buffer 1, multipliers into buffer 0.
        for (int i = threadIdx.x; i < Tn * STATE; i += blockDim.x) {
            const int tt = i / STATE, e = i - STATE * tt;
            const float v = p.state[(size_t)tl.first * STATE + i];
            if (e < 44) sm[S.xi1 + (p.T + tt) * 48 + (e / NV) * 12 + e % NV] = v;
            else if (e < 55) sm[S.xi2 + (p.T + tt) * 12 + (e - 44)] = v;
            else if (e < 99) sm[S.lam + tt * 48 + ((e - 55) / NV) * 12 + (e - 55) % NV] = v;
            else sm[S.lps + tt * 12 + (e - 99)] = v;
        }
        __syncthreads();
        // Reference xi1, xi2 into buffer 0: boundary control points from the
        // boundary conditions on every block that has boundary rows, the rest as given.
        for (int i = threadIdx.x; i < Tn * 55; i += blockDim.x) {
            const int tt = i / 55, e = i - 55 * tt, blk = e / NV, k = e - NV * blk;
            const bool has_bc = (blk == 0 || blk == 2 || blk == 4 || L.cs_boundary);
            float *src = blk < 4 ? sm + S.xi1 + (p.T + tt) * 48 + blk * 12 : sm + S.xi2 + (p.T + tt) * 12;
            float *dst = blk < 4 ? sm + S.xi1 + tt * 48 + blk * 12 : sm + S.xi2 + tt * 12;
            float v = src[k];
            if (has_bc && k <= 2) v = sm[S.cst + L.off_ends + blk * 8 + k];
            if (has_bc && k >= 8) v = sm[S.cst + L.off_ends + blk * 8 + (k - 5)];
            dst[k] = v;
        }
        __syncthreads();

        const int tid = threadIdx.x;
        const bool stepper = tid < Tn * L.q;
        const int tt = stepper ? tid / L.q : 0;
        const int t = stepper ? tid - tt * L.q : 0;
        float Prow[12];
        load12(Prow, sm + S.cst + L.off_prow + t * 12);
        StepRegs r;
        r.psi_t = 0.f;
        int cur = 0, cur2 = 0;

        // Step 1 of Sec. III-D: xi3, xi4 and g from the initial samples, the
        // residual against the reference.
        if (stepper) {
            StepRegs ref;
            eval_xy(sm, S, L, sm + S.xi1 + (p.T + tt) * 48, t, Prow, r);
            eval_xy(sm, S, L, sm + S.xi1 + tt * 48, t, Prow, ref);
            sweep<M, LIT, false, false, true>(sm, S, L, sm + S.xi2 + (p.T + tt) * 12, t, tt, Prow, r, ref);
            float x2[12];
            load12(x2, sm + S.xi2 + tt * 12);
            r.psi_cur = dot11(Prow, x2);  // heading of the reference c_psi
        }
        __syncthreads();
        phase_dot(p, sm, S, tl);
        __syncthreads();

        for (int k = 0; k < p.iters; ++k) {
            const bool res = (p.hist != nullptr) || (k == p.iters - 1);
            const bool prev_res = (p.hist != nullptr) && k > 0;
            phase_xi1(p, sm, S, tl, cur, k == 0, true, prev_res, false, k - 1);
            cur ^= 1;
            __syncthreads();
            if (stepper) {
                eval_xy(sm, S, L, sm + S.xi1 + (cur * p.T + tt) * 48, t, Prow, r);
                // psi_t = psi + wrap(atan2(s, c) - psi), psi the previous heading;
                // the heading step works on delta = psi_t - P xi2
                r.psi_t = r.psi_prev + wrap_pi(atan2f(r.s, r.c) - r.psi_prev);
                sm[S.psit + tt * L.qs + t] = r.psi_t - r.psi_cur;
            }
            __syncthreads();
            phase_psi(p, sm, S, tl, cur2);
            cur2 ^= 1;
            __syncthreads();
            if (stepper)
                sweep_dispatch<M, LIT>(sm, S, L, sm + S.xi2 + (cur2 * p.T + tt) * 12, tt, t, Prow, r,
                                       res, k == p.iters - 1);
            __syncthreads();
            phase_dot(p, sm, S, tl);
            __syncthreads();
        }
        // Multipliers of the last iteration and the final per-trajectory results.
        phase_xi1(p, sm, S, tl, cur, false, false, true, true, p.iters - 1);
        cur ^= 1;
        __syncthreads();
        for (int i = threadIdx.x; i < Tn * STATE; i += blockDim.x) {
            const int tq = i / STATE, e = i - STATE * tq;
            float v;
            if (e < 44) v = sm[S.xi1 + (cur * p.T + tq) * 48 + (e / NV) * 12 + e % NV];
            else if (e < 55) v = sm[S.xi2 + (cur2 * p.T + tq) * 12 + (e - 44)];
            else if (e < 99) v = sm[S.lam + (cur * p.T + tq) * 48 + ((e - 55) / NV) * 12 + (e - 55) % NV];
            else v = sm[S.lps + tq * 12 + (e - 99)];
            p.state[(size_t)tl.first * STATE + i] = v;
        }
        __syncthreads();
    }
}

}  // namespace

size_t fused_smem_bytes(const ConstLayout &L, int tile)
{
    return size_t(smem_layout(L, tile).total) * sizeof(float);
}

int fused_auto_tile(const ConstLayout &L, int B, int num_sms)
{
    // Largest tile that fits one CTA per SM, then shrink so every SM gets work.
    int tmax = kMaxThreads / (L.q > 88 ? L.q : 88);
    if (tmax < 1) tmax = 1;
    while (tmax > 1 && fused_smem_bytes(L, tmax) > 227 * 1024) --tmax;
    int want = (B + num_sms - 1) / num_sms;
    if (want < 1) want = 1;
    return want < tmax ? want : tmax;
}

int launch_fused(const SolveArgs &a, void *stream, int *launches)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const ConstLayout &L = a.L;
    int T = a.tile > 0 ? a.tile : fused_auto_tile(L, a.B, sms);
    const int tq = T * (L.q > 88 ? L.q : 88);
    if (tq > kMaxThreads || T < 1) return -1;
    const size_t smem = fused_smem_bytes(L, T);
    if (smem > 227 * 1024) return -1;
    const int threads = (tq + 31) & ~31;
    const int ntiles = (a.B + T - 1) / T;
    const int grid = ntiles < sms ? ntiles : sms;

    KParams p;
    p.cblob = a.cblob;
    p.L = L;
    p.B = a.B;
    p.iters = a.iters;
    p.T = T;
    p.ntiles = ntiles;
    p.state = a.state;
    p.res = a.res;
    p.res_psi = a.res_psi;
    p.cost = a.cost;
    p.mind = a.mind;
    p.hist = a.hist;
    p.err = a.err;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const int sel = L.m * 2 + (L.alpha_mode ? 1 : 0);
    switch (sel) {
#define AM_CASE(MM, LL)                                                                       \
    case MM * 2 + LL:                                                                         \
        e = cudaFuncSetAttribute(am_fused_kernel<MM, LL>,                                     \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));     \
        if (e != cudaSuccess) return -2;                                                      \
        am_fused_kernel<MM, LL><<<grid, threads, smem, st>>>(p);                              \
        break;
        AM_CASE(1, 0)
        AM_CASE(2, 0)
        AM_CASE(3, 0)
        AM_CASE(4, 0)
        AM_CASE(1, 1)
        AM_CASE(2, 1)
        AM_CASE(3, 1)
        AM_CASE(4, 1)
#undef AM_CASE
    default:
        return -1;
    }
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam
