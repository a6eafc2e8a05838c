// Plain FP32 GPU loop: the same AM iteration as the fused kernel (same
// formulation, same precision), written the straightforward way -- one launch
// per step, every intermediate (trajectory values, the projected obstacle
// points of Eq. compute_zeta_3, the per-step residual vectors) stored in
// global memory between launches.  It is the comparator the fused, persistent
// kernel is measured against.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "am_internal.h"
#include "../../include/trajam.h"

namespace trajam {
namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kPi = 3.14159265358979323846f;

struct PlainBufs {
    float *xi1[2]; // [B][44]  current / next
    float *xi0;    // [B][44]  xi1 as given (first step only)
    float *lam;    // [B][44]
    float *xi2[2]; // [B][11]  current / next c_psi
    float *xi20;   // [B][11]  c_psi as given (first step only)
    float *dx2;    // [B][11]  last heading increment
    float *lps;    // [B][11]
    float *rr;     // [B][44]  R = F^T (g - F xi1)
    float *ptp;    // [B][11]  P^T delta, delta = psi_t - P xi2
    float *ev;     // [B][8][q]   x, xd, xdd, c, y, yd, ydd, s of the current xi1
    float *ev0;    // [B][8][q]   the same for xi1 as given
    float *psit;   // [B][q]      psi_t
    float *dps;    // [B][q]      delta = psi_t - P xi2
    float *psicur; // [B][q]      P xi2 of the current coefficients
    float *psi;    // [B][4][q]   psi, cos, sin, psidd of the heading g is built from
    float *gob;    // [B][m][n][q][2]  projected obstacle points minus (xt, yt)
    float *dob;    // [B][m][n][q]     squared ellipse distance
    float *gv;     // [B][12][q]  rv_x ra_x r0_x r1_x rv_y ra_y r0_y r1_y res2 respsi2 cost dmin
};

size_t plain_layout(const ConstLayout &L, int B, PlainBufs *b, float *base)
{
    const size_t q = L.q, mn = size_t(L.m) * L.n;
    size_t o = 0;
    auto take = [&](float *&p, size_t n) {
        if (b) p = base + o;
        o += (n + 63) & ~size_t(63);
    };
    PlainBufs d;
    PlainBufs *t = b ? b : &d;
    take(t->xi1[0], size_t(B) * 44);
    take(t->xi1[1], size_t(B) * 44);
    take(t->xi0, size_t(B) * 44);
    take(t->lam, size_t(B) * 44);
    take(t->xi2[0], size_t(B) * 11);
    take(t->xi2[1], size_t(B) * 11);
    take(t->xi20, size_t(B) * 11);
    take(t->dx2, size_t(B) * 11);
    take(t->lps, size_t(B) * 11);
    take(t->rr, size_t(B) * 44);
    take(t->ptp, size_t(B) * 11);
    take(t->ev, size_t(B) * 8 * q);
    take(t->ev0, size_t(B) * 8 * q);
    take(t->psit, size_t(B) * q);
    take(t->dps, size_t(B) * q);
    take(t->psicur, size_t(B) * q);
    take(t->psi, size_t(B) * 4 * q);
    take(t->gob, size_t(B) * mn * q * 2);
    take(t->dob, size_t(B) * mn * q);
    take(t->gv, size_t(B) * 12 * q);
    return o;
}

__device__ __forceinline__ float wrap_pi(float a)
{
    return a - kTwoPi * ceilf((a - kPi) * (1.0f / kTwoPi));
}

__global__ void k_unpack(const float *state, PlainBufs b, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * STATE) return;
    const int l = i / STATE, e = i - STATE * l;
    const float v = state[i];
    if (e < 44) b.xi0[l * 44 + e] = v;
    else if (e < 55) b.xi20[l * 11 + e - 44] = v;
    else if (e < 99) b.lam[l * 44 + e - 55] = v;
    else b.lps[l * 11 + e - 99] = v;
}

__global__ void k_pack(float *state, PlainBufs b, const float *xi1, const float *xi2, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * STATE) return;
    const int l = i / STATE, e = i - STATE * l;
    float v;
    if (e < 44) v = xi1[l * 44 + e];
    else if (e < 55) v = xi2[l * 11 + e - 44];
    else if (e < 99) v = b.lam[l * 44 + e - 55];
    else v = b.lps[l * 11 + e - 99];
    state[i] = v;
}

// Reference xi1, xi2: boundary control points from the boundary conditions.
__global__ void k_reference(const float *cst, ConstLayout L, const float *xi0, float *xi1,
                            const float *x20, float *x2, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 55) return;
    const int l = i / 55, e = i - 55 * l, blk = e / NV, k = e - NV * blk;
    const bool has_bc = (blk == 0 || blk == 2 || blk == 4 || L.cs_boundary);
    float v = blk < 4 ? xi0[l * 44 + e] : x20[l * 11 + k];
    if (has_bc && k <= 2) v = cst[L.off_ends + blk * 8 + k];
    if (has_bc && k >= 8) v = cst[L.off_ends + blk * 8 + (k - 5)];
    if (blk < 4) xi1[l * 44 + e] = v;
    else x2[l * 11 + k] = v;
}

// lam += rho R (Eq. update_lambda_1 with R = F^T (g - F xi1)).
__global__ void k_lambda(ConstLayout L, PlainBufs b, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 44) return;
    b.lam[i] += L.rho * b.rr[i];
}

// xi1' = xi1 + Minv (lam - Q xi1 + rho R)  (Eq. over_3 in increment form).
__global__ void k_xi1(const float *cst, ConstLayout L, PlainBufs b, const float *xi1, float *xo, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 44) return;
    const int l = i / 44, u = i - 44 * l, side = u / NS, row = u - NS * side;
    const float *lam = b.lam + l * 44 + NS * side, *rr = b.rr + l * 44 + NS * side;
    const float *xi = xi1 + l * 44 + NS * side;
    float a0 = 0.f, a1 = 0.f;
    for (int c = 0; c < NS; ++c) {
        a0 = fmaf(cst[L.off_mt + c * 24 + row], lam[c] + L.rho * rr[c], a0);
        a1 = fmaf(cst[L.off_mq + c * 24 + row], xi[c], a1);
    }
    xo[i] = xi[row] + (a0 - a1);
}

// Trajectory values at every step (Eq. param).
__global__ void k_eval(const float *cst, ConstLayout L, const float *xi1, float *ev, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * L.q) return;
    const int l = i / L.q, t = i - L.q * l, q = L.q;
    const float *P = cst + L.off_prow + t * 12, *Pd = P + q * 12, *Pdd = P + 2 * q * 12;
    const float *xi = xi1 + l * 44;
    float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < NV; ++k) {
        v[0] = fmaf(P[k], xi[k], v[0]);
        v[1] = fmaf(Pd[k], xi[k], v[1]);
        v[2] = fmaf(Pdd[k], xi[k], v[2]);
        v[3] = fmaf(P[k], xi[11 + k], v[3]);
        v[4] = fmaf(P[k], xi[22 + k], v[4]);
        v[5] = fmaf(Pd[k], xi[22 + k], v[5]);
        v[6] = fmaf(Pdd[k], xi[22 + k], v[6]);
        v[7] = fmaf(P[k], xi[33 + k], v[7]);
    }
    for (int c = 0; c < 8; ++c) ev[(size_t(l) * 8 + c) * q + t] = v[c];
}

// psi_t = psi + wrap(atan2(s, c) - psi) against the previous heading, and
// delta = psi_t - P xi2 for the incremental heading step.
__global__ void k_psit(ConstLayout L, PlainBufs b, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * L.q) return;
    const int l = i / L.q, t = i - L.q * l, q = L.q;
    const float c = b.ev[(size_t(l) * 8 + 3) * q + t], s = b.ev[(size_t(l) * 8 + 7) * q + t];
    const float prev = b.psi[size_t(l) * 4 * q + t];
    const float pt = prev + wrap_pi(atan2f(s, c) - prev);
    b.psit[i] = pt;
    b.dps[i] = pt - b.psicur[i];
}

// xi2' = xi2 + Mpsi (lam_psi - H xi2) + rho W^T delta and P^T delta
// (Eq. compute_convex_surrogate in increment form).
__global__ void k_xi2(const float *cst, ConstLayout L, PlainBufs b, const float *x2, float *x2n, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 22) return;
    const int l = i / 22, kk = i - 22 * l;
    const float *col = cst + (kk < NV ? L.off_wcol + kk * L.qs : L.off_pcol + (kk - NV) * L.qs);
    const float *ps = b.dps + size_t(l) * L.q;
    float d = 0.f;
    for (int t = 0; t < L.q; ++t) d = fmaf(col[t], ps[t], d);
    if (kk < NV) {
        float a0 = 0.f, a1 = 0.f;
        for (int c = 0; c < NV; ++c) {
            a0 = fmaf(cst[L.off_mpsi + c * 12 + kk], b.lps[l * 11 + c], a0);
            a1 = fmaf(cst[L.off_mpsih + c * 12 + kk], x2[l * 11 + c], a1);
        }
        const float dx = L.rho * d + (a0 - a1);
        b.dx2[l * 11 + kk] = dx;
        x2n[l * 11 + kk] = x2[l * 11 + kk] + dx;
    } else {
        b.ptp[l * 11 + kk - NV] = d;
    }
}

// psi = P xi2 into psicur; with trig, also its cosine, sine and second
// derivative for the steps that build g from it.
__global__ void k_psi(const float *cst, ConstLayout L, PlainBufs b, const float *x2, int B, int trig)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * L.q) return;
    const int l = i / L.q, t = i - L.q * l, q = L.q;
    const float *P = cst + L.off_prow + t * 12, *Pdd = P + 2 * q * 12;
    float p = 0.f, pdd = 0.f;
    for (int k = 0; k < NV; ++k) {
        p = fmaf(P[k], x2[l * 11 + k], p);
        pdd = fmaf(Pdd[k], x2[l * 11 + k], pdd);
    }
    b.psicur[i] = p;
    if (!trig) return;
    float *o = b.psi + size_t(l) * 4 * q;
    o[t] = p;
    o[q + t] = cosf(p);
    o[2 * q + t] = sinf(p);
    o[3 * q + t] = pdd;
}

// The alpha/d steps per (trajectory, circle, obstacle, step), stored as the
// offset e = projected point - (xt, yt), with the projected point
// (a d cos alpha, b d sin alpha) = (xt, yt) max(1, 1/d_raw).
__global__ void k_obstacles(const float *cst, ConstLayout L, PlainBufs b, const float *ev, int B)
{
    const int mn = L.m * L.n;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * mn * L.q) return;
    const int q = L.q;
    const int t = int(i % q);
    const long long r = i / q;
    const int ij = int(r % mn), l = int(r / mn), ci = ij / L.n, j = ij - L.n * ci;
    const float x = ev[(size_t(l) * 8 + 0) * q + t], y = ev[(size_t(l) * 8 + 4) * q + t];
    const float cp = b.psi[size_t(l) * 4 * q + q + t], sp = b.psi[size_t(l) * 4 * q + 2 * q + t];
    const float4 c = reinterpret_cast<const float4 *>(cst + L.off_obc)[j];
    const float2 o = reinterpret_cast<const float2 *>(cst + L.off_obs)[j * L.qs + t];
    const float xt = x + L.r[ci] * cp - o.x * c.z, yt = y + L.r[ci] * sp - o.y * c.w;
    const float D = xt * xt * c.x * c.x + yt * yt * c.y * c.y;
    float2 e;
    if (!L.alpha_mode) {
        const float f = D > 0.f ? fmaxf(1.f, rsqrtf(D)) : 1.f;
        e = make_float2(xt * (f - 1.f), yt * (f - 1.f));
    } else {
        // printed alpha = atan2(yt, xt); d = max(1, least squares along that ray)
        const float rr = sqrtf(xt * xt + yt * yt);
        const float ca = rr > 0.f ? xt / rr : 1.f, sa = rr > 0.f ? yt / rr : 0.f;
        const float d = fmaxf(1.f, (c.z * xt * ca + c.w * yt * sa) / (c.z * c.z * ca * ca + c.w * c.w * sa * sa));
        e = make_float2(c.z * d * ca - xt, c.w * d * sa - yt);
    }
    if (D == 0.f) e = make_float2(c.z, 0.f);  // alpha = atan2(0, 0) = 0, d = 1
    reinterpret_cast<float2 *>(b.gob)[i] = e;
    b.dob[i] = D;
}

// Per-step residual vectors g - F xi1 (g from ev_g, F xi1 from ev_f) and the
// step's squared residual and cost terms.
__global__ void k_gsum(const float *cst, ConstLayout L, PlainBufs b, const float *ev_g,
                       const float *ev_f, int B, int res)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * L.q) return;
    const int l = i / L.q, t = i - L.q * l, q = L.q, mn = L.m * L.n;
    const float *eg = ev_g + size_t(l) * 8 * q, *ef = ev_f + size_t(l) * 8 * q;
    const float x = eg[t], xd = eg[q + t], xdd = eg[2 * q + t];
    const float y = eg[4 * q + t], yd = eg[5 * q + t], ydd = eg[6 * q + t];
    const float xf = ef[t], xdf = ef[q + t], xddf = ef[2 * q + t], c = ef[3 * q + t];
    const float yf = ef[4 * q + t], ydf = ef[5 * q + t], yddf = ef[6 * q + t], s = ef[7 * q + t];
    const float *ps = b.psi + size_t(l) * 4 * q;
    const float psi = ps[t], cp = ps[q + t], sp = ps[2 * q + t], psidd = ps[3 * q + t];
    const float vn = sqrtf(xd * xd + yd * yd), an = sqrtf(xdd * xdd + ydd * ydd);
    const float sv = vn > L.v_max ? L.v_max / vn : 1.f, sa = an > L.a_max ? L.a_max / an : 1.f;
    float r0x = 0, r1x = 0, r0y = 0, r1y = 0, r2 = 0, dmin = 3.0e38f;
    const float2 *g = reinterpret_cast<const float2 *>(b.gob) + size_t(l) * mn * q;
    for (int ij = 0; ij < mn; ++ij) {
        const int ci = ij / L.n;
        const float2 e = g[ij * q + t];
        // g_ij - (x_f + r_i c): g_ij = x + r_i cos psi + e_ij
        const float ex = (x - xf) + L.r[ci] * (cp - c) + e.x;
        const float ey = (y - yf) + L.r[ci] * (sp - s) + e.y;
        r0x += ex;
        r0y += ey;
        r1x += L.r[ci] * ex;
        r1y += L.r[ci] * ey;
        if (res) {
            r2 += ex * ex + ey * ey;
            dmin = fminf(dmin, b.dob[(size_t(l) * mn + ij) * q + t]);
        }
    }
    float *G = b.gv + size_t(l) * 12 * q + t;
    G[0] = xd * sv - xdf;
    G[q] = xdd * sa - xddf;
    G[2 * q] = r0x;
    G[3 * q] = r1x + (cp - c);
    G[4 * q] = yd * sv - ydf;
    G[5 * q] = ydd * sa - yddf;
    G[6 * q] = r0y;
    G[7 * q] = r1y + (sp - s);
    if (res) {
        const float ov = xd - xd * sv, ow = yd - yd * sv, oa = xdd - xdd * sa, ob = ydd - ydd * sa;
        r2 += ov * ov + ow * ow + oa * oa + ob * ob + (c - cp) * (c - cp) + (s - sp) * (s - sp);
        G[8 * q] = r2;
        const float dp = psi - b.psit[size_t(l) * q + t];
        G[9 * q] = dp * dp;
        G[10 * q] = xdd * xdd + ydd * ydd + psidd * psidd;
        G[11 * q] = dmin;
    }
}

// R per (trajectory, unknown): Pd^T rv + Pdd^T ra + P^T r0, or P^T r1.
__global__ void k_rdot(const float *cst, ConstLayout L, PlainBufs b, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 44) return;
    const int l = i / 44, u = i - 44 * l, side = u / NS, row = u - NS * side, q = L.q;
    const float *G = b.gv + size_t(l) * 12 * q + 4 * side * q;
    const float *P = cst + L.off_pcol, *Pd = P + NV * L.qs, *Pdd = P + 2 * NV * L.qs;
    float acc = 0.f;
    if (row < NV) {
        for (int t = 0; t < q; ++t) {
            acc = fmaf(Pd[row * L.qs + t], G[t], acc);
            acc = fmaf(Pdd[row * L.qs + t], G[q + t], acc);
            acc = fmaf(P[row * L.qs + t], G[2 * q + t], acc);
        }
    } else {
        for (int t = 0; t < q; ++t) acc = fmaf(P[(row - NV) * L.qs + t], G[3 * q + t], acc);
    }
    b.rr[i] = acc;
}

// lam_psi -= sign rho_psi P^T (P xi2' - psi_t) = sign rho_psi (P^T P dxi2 - P^T delta)
// (Eq. update_lambda_psi).
__global__ void k_lampsi(const float *cst, ConstLayout L, PlainBufs b, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * NV) return;
    const int l = i / NV, k = i - NV * l;
    float a = 0.f;
    for (int c = 0; c < NV; ++c) a = fmaf(cst[L.off_ptp + c * 12 + k], b.dx2[l * 11 + c], a);
    b.lps[i] -= L.psi_sign * L.rho_psi * (a - b.ptp[i]);
}

// Per-trajectory residual, heading residual, cost and smallest distance.
__global__ void k_scalars(ConstLayout L, PlainBufs b, int B, float *res, float *res_psi,
                          float *cost, float *mind, float *hist, int iters, int k)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= B) return;
    const int q = L.q;
    const float *G = b.gv + size_t(l) * 12 * q;
    // reductions over the steps in FP64, as in the fused kernel
    double r2 = 0, rp2 = 0, c2 = 0;
    float dm = 3.0e38f;
    for (int t = 0; t < q; ++t) {
        r2 += G[8 * q + t];
        rp2 += G[9 * q + t];
        c2 += G[10 * q + t];
        dm = fminf(dm, G[11 * q + t]);
    }
    const float r = float(sqrt(r2)), rp = float(sqrt(rp2)), c = float(c2);
    if (hist) {
        hist[(size_t(l) * iters + k) * 3 + 0] = r;
        hist[(size_t(l) * iters + k) * 3 + 1] = rp;
        hist[(size_t(l) * iters + k) * 3 + 2] = c;
    }
    if (k == iters - 1) {
        res[l] = r;
        res_psi[l] = rp;
        cost[l] = c;
        mind[l] = sqrtf(dm);
    }
}

inline int blocks(long long n, int t) { return int((n + t - 1) / t); }

}  // namespace

size_t plain_scratch_floats(const ConstLayout &L, int B) { return plain_layout(L, B, nullptr, nullptr); }

int launch_plain(const SolveArgs &a, float *scratch, size_t scratch_floats, void *stream, int *launches)
{
    const ConstLayout &L = a.L;
    const int B = a.B;
    if (plain_scratch_floats(L, B) > scratch_floats) return -1;
    PlainBufs b;
    plain_layout(L, B, &b, scratch);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *cst = a.cblob;
    const int T = 256;
    int nl = 0;
    const long long nq = (long long)B * L.q, nobs = (long long)B * L.m * L.n * L.q;
    const long long nx = (long long)B * 44;
#define LAUNCH(kern, n, ...)                                      \
    do {                                                          \
        if ((n) > 0) {                                            \
            kern<<<blocks((n), T), T, 0, st>>>(__VA_ARGS__);      \
            ++nl;                                                 \
        }                                                         \
    } while (0)
    int cur = 0, c2 = 0;
    LAUNCH(k_unpack, (long long)B * STATE, a.state, b, B);
    LAUNCH(k_reference, (long long)B * 55, cst, L, b.xi0, b.xi1[cur], b.xi20, b.xi2[c2], B);
    // Step 1: g from the initial samples, the residual against the reference.
    LAUNCH(k_eval, nq, cst, L, b.xi0, b.ev0, B);
    LAUNCH(k_eval, nq, cst, L, b.xi1[cur], b.ev, B);
    LAUNCH(k_psi, nq, cst, L, b, b.xi20, B, 1);
    LAUNCH(k_psi, nq, cst, L, b, b.xi2[c2], B, 0);
    LAUNCH(k_obstacles, nobs, cst, L, b, b.ev0, B);
    LAUNCH(k_gsum, nq, cst, L, b, b.ev0, b.ev, B, 0);
    LAUNCH(k_rdot, nx, cst, L, b, B);
    for (int k = 0; k < a.iters; ++k) {
        const int res = (a.hist != nullptr) || (k == a.iters - 1);
        if (k > 0) LAUNCH(k_lambda, nx, L, b, B);
        LAUNCH(k_xi1, nx, cst, L, b, b.xi1[cur], b.xi1[cur ^ 1], B);
        cur ^= 1;
        LAUNCH(k_eval, nq, cst, L, b.xi1[cur], b.ev, B);
        LAUNCH(k_psit, nq, L, b, B);
        LAUNCH(k_xi2, (long long)B * 22, cst, L, b, b.xi2[c2], b.xi2[c2 ^ 1], B);
        c2 ^= 1;
        LAUNCH(k_psi, nq, cst, L, b, b.xi2[c2], B, 1);
        LAUNCH(k_obstacles, nobs, cst, L, b, b.ev, B);
        LAUNCH(k_gsum, nq, cst, L, b, b.ev, b.ev, B, res);
        LAUNCH(k_rdot, nx, cst, L, b, B);
        LAUNCH(k_lampsi, (long long)B * NV, cst, L, b, B);
        if (res) LAUNCH(k_scalars, B, L, b, B, a.res, a.res_psi, a.cost, a.mind, a.hist, a.iters, k);
    }
    LAUNCH(k_lambda, nx, L, b, B);
    LAUNCH(k_pack, (long long)B * STATE, a.state, b, b.xi1[cur], b.xi2[c2], B);
#undef LAUNCH
    if (launches) *launches += nl;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam

// ---------------------------------------------------------------------------
// Allocation-free variant of the plain loop.
//
// Some callers must not allocate device memory at solve time: a real-time
// re-planning step has a fixed time budget, and cudaMalloc/cudaFree can block
// for an unbounded time and synchronise the whole device; code running while a
// stream is being captured, or under an external memory manager that owns all
// device allocations, may not call them at all.  For them the plain loop can
// keep its intermediates in a fixed area that is part of this library's device
// image: every GPU that loads the library holds it until the process exits.
//
// kNoallocScratchFloats bounds the batch: the loop needs plain_scratch_floats()
// floats, about (17 + 3 m n) q + 300 per trajectory (12.8 k floats at q = 100,
// m = 3, n = 10, i.e. up to 650 trajectories in 32 MiB).
namespace {

constexpr size_t kNoallocScratchFloats = size_t(8) << 20;  // 32 MiB of FP32
static __device__ __align__(256) float g_noalloc_scratch[kNoallocScratchFloats];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
float *g_noalloc_addr[kMaxDevices] = {};

// Device address of the fixed area on the current device.  Host code cannot
// use the symbol itself (it names a host-side stand-in), so the address is
// looked up once per device, with that device current, and cached.  Every
// call checks that the cached address is still a device allocation of the
// current context (a cudaDeviceReset destroys the context and reloads the
// module, possibly elsewhere) and looks it up again when it is not; neither
// query allocates.
int noalloc_scratch(float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return trajam::report_error(AM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return trajam::report_error(AM_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev]) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, g_noalloc_addr[dev]) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != dev) {
            cudaGetLastError();  // a failed query leaves no error behind
            g_noalloc_addr[dev] = nullptr;
        }
    }
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return trajam::report_error(AM_ERR_CUDA, "cudaGetSymbolAddress of the fixed scratch area failed");
        g_noalloc_addr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_addr[dev];
    return AM_OK;
}

}  // namespace

extern "C" AM_API int am_solve_batch_noalloc(const am_problem *h, int B, float *state, float *res,
                                             float *res_psi, float *cost, float *mind, int iters,
                                             void *stream)
{
    using namespace trajam;
    const float *cblob = nullptr;
    ConstLayout L;
    int rc = handle_constants(h, &cblob, &L);
    if (rc) return rc;
    if (!state || !res || !res_psi || !cost || !mind) return report_error(AM_ERR_ARG, "null device buffer");
    if (L.precision != 0) return report_error(AM_ERR_ARG, "reduced precision runs on the fused kernel only");
    if (B < 1 || iters < 1 || iters > 100000) return report_error(AM_ERR_ARG, "B >= 1 and 1 <= iters <= 100000 required");
    const size_t need = plain_scratch_floats(L, B);
    if (need > kNoallocScratchFloats) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "batch of %d needs %zu floats of scratch; the fixed area holds %zu (32 MiB)", B, need,
                 kNoallocScratchFloats);
        return report_error(AM_ERR_BUDGET, msg);
    }
    float *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    // the handle's constants must live on the device whose area is used
    int dev = 0;
    cudaPointerAttributes at;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&at, cblob) != cudaSuccess ||
        at.type != cudaMemoryTypeDevice || at.device != dev) {
        cudaGetLastError();
        return report_error(AM_ERR_ARG, "the handle's constants are not on the current device");
    }
    rc = handle_order_before(h, stream);
    if (rc) return rc;
    SolveArgs a;
    a.cblob = cblob;
    a.L = L;
    a.B = B;
    a.iters = iters;
    a.state = state;
    a.res = res;
    a.res_psi = res_psi;
    a.cost = cost;
    a.mind = mind;
    a.hist = nullptr;
    a.tile = 0;
    a.err = nullptr;
    rc = launch_plain(a, scratch, kNoallocScratchFloats, stream, nullptr);
    if (rc) return report_error(AM_ERR_CUDA, "plain loop launch failed");
    return AM_OK;
}
