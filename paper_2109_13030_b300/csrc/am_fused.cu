// Fused persistent kernel of the batched alternating-minimization loop
// (Sec. III-D, steps 1-5, and the batch solution of Sec. III-E).
//
// One CTA stays resident on each SM and works through tiles of T <= 8
// trajectories.  It stages the constant block into shared memory once (bulk
// async copy, completion on an mbarrier), keeps xi1, xi2, lambda, lambda_psi
// and the residual contraction R = F^T (g - F xi1) of every trajectory of the
// tile in shared memory for all iterations, and writes the state back only
// after the last one.  Nothing per element (alpha, d, g) is ever stored.
//
// The position step of Eq. over_3, xi1' = Minv (lam + rho F^T g) + kb, is
// evaluated in the algebraically equal increment form
//     xi1' = xi1 + Minv (lam - Q xi1 + rho F^T (g - F xi1))
// (from Minv Qbar + N A = I, kb = N b and A xi1 = b), so FP32 works on the
// small constraint residual instead of on |F^T g| ~ 1e3, which the explicit
// inverse would amplify by its conditioning.  The multiplier update of
// Eq. update_lambda_1 is lam' = lam + rho R with the same R.  The heading
// step of Eq. compute_convex_surrogate is treated the same way.  A solve
// starts from a reference whose boundary control points are set from the
// boundary conditions, so A xi = b holds from the first step on.
//
// The two contractions over the time steps -- R (Pd^T rv + Pdd^T ra + P^T r0
// and P^T r1 per side) and the heading right-hand side (W^T delta, P^T delta)
// -- are dense products of a [rows x steps] operand written by the sweep with
// constant basis columns.  They run on the tensor cores as mma.sync
// m16n8k8 TF32 with each FP32 operand split into a TF32 high part and a TF32
// remainder (three products: hi*hi + hi*lo + lo*hi), which keeps FP32-level
// accuracy.
//
// Phases of one iteration, separated by __syncthreads():
//   XI1   lam += rho R; xi1 += Minv (lam - Q xi1 + rho R); lambda_psi update
//         (Eq. update_lambda_psi); per-trajectory sums of the last sweep
//   EVAL  x, xdot, xddot, y, ..., c, s at step t (Eq. param); heading target
//         psi_t and delta = psi_t - P xi2
//   PSI   W^T delta and P^T delta on the tensor cores; Mpsi lam_psi -
//         Mpsi H xi2 on warps without an MMA task (in EVAL on a small block)
//   SWEEP xi2 += Mpsi (lam_psi - H xi2) + rho W^T delta; psi = P xi2; the
//         closed-form alpha/d steps for every circle and obstacle (Eq. zeta_2 -
//         compute_da) in the trig-free form (xt, yt) max(1, 1/sqrt(xt^2/a^2 +
//         yt^2/b^2)), the velocity and acceleration projections, and the
//         per-step residual vectors of R
//   DOT   R on the tensor cores
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "am_internal.h"

namespace trajam {
namespace {

constexpr int kMaxThreads = 768;
constexpr int kMaxTile = 8;     // rows (side, trajectory) of one 16-row MMA tile
constexpr int kDotParts = 2;    // parts of the steps per segment of R in the DOT phase
constexpr int kRParts = 3 * kDotParts;  // partials of R: (rv | ra | r0 segment) x part of the steps
constexpr int kPsiParts = 4;    // partials of W^T delta, P^T delta: quarters of the steps

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kPi = 3.14159265358979323846f;

struct Smem {
    int cst, xi1, lam, rb, xi2, dx2, lps, ptp, psp, bas, G2, RS, GX, PS, XA, NR, NM, bar, total, T;
};

// Shared-memory layout (float offsets).
//   xi1, lam  [2][T][48]   double-buffered, padded blocks of 12 per polynomial
//   rb        [3D][T][48]  partials of R per side (c_pos rows 0..10, c_slack rows
//                          12..22), D = kDotParts: (rv, ra, r0 segment) x part of
//                          the steps; the c_slack rows in the first D (R is the sum of all)
//   xi2       [2][T][12]   double-buffered c_psi;  dx2 [T][12] last increment
//   lps       [T][12]      lambda_psi
//   ptp       [8][12]      P^T delta
//   psp       [4][8][24]   partials of W^T delta (0..10) and P^T delta (12..22) per quarter
//   bas       [8][12]      Mpsi lam_psi - Mpsi H xi2
//   G2        [2T][RS]     residual vectors, row = side*T + trajectory; segments
//                          rv | ra | r0 | r1 of qp steps
//   GX        [T][4][qs]   per-step squared residual, heading residual, cost, distance
//   PS        [T][qp]      delta = psi_t - P xi2 per trajectory
//   XA        [2T][56][2]  A operand of the position step as TF32 pairs, row =
//                          side*T + trajectory: lam + coef R (24) | xi1 (24)
//   NR        [T*q][2]     robot centre of each step when its warp's near list was formed
//   NM        [24][2]      near-obstacle bit lists per warp (obstacles 0..31, 32..63)
// The constant block is staged from its offset off_fused on; cst is shifted so
// that sm + cst + off_x addresses section x.
__host__ __device__ inline Smem smem_layout(const ConstLayout &L, int T)
{
    Smem s;
    int o = 0;
    s.T = T;
    s.bar = o; o += 4;  // one 8-byte mbarrier at a fixed offset, 16-byte aligned
    s.cst = o - L.off_fused; o += L.total - L.off_fused;
    s.xi1 = o; o += 2 * T * 48;
    s.lam = o; o += 2 * T * 48;
    s.rb = o; o += kRParts * T * 48;
    s.xi2 = o; o += 2 * T * 12;
    s.dx2 = o; o += T * 12;
    s.lps = o; o += T * 12;
    s.ptp = o; o += kMaxTile * 12;
    s.psp = o; o += kPsiParts * kMaxTile * 24;
    s.bas = o; o += kMaxTile * 12;
    // RS = 8 mod 32 and qp = 8 mod 16: the 64-bit fragment loads of four
    // neighbouring rows fall on distinct banks
    s.RS = 4 * L.qp + 8;
    s.G2 = o; o += 2 * T * s.RS;
    s.GX = o; o += T * 4 * L.qs;
    s.PS = o; o += T * L.qp;
    s.XA = o; o += 2 * T * 56 * 2;
    s.NR = o; o += 2 * T * L.q;
    s.NM = o; o += 24 * 2;
    o = (o + 3) & ~3;
    s.total = o;
    return s;
}

// R of the position step: the sum of the partials the DOT phase writes.
__device__ __forceinline__ float rsum(const float *sm, const Smem &S, int i)
{
    const int n = S.T * 48;
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < kRParts; ++k) r += sm[S.rb + k * n + i];
    return r;
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

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Limit of the device-side wait for the constant copy: about a second of
// the global timer (and an iteration cap behind it).
constexpr uint64_t kWaitLimitNs = 1000000000ull;

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

// ------------------------------------------------------------ tensor cores

// Round a finite FP32 value to the nearest TF32 (ties away from zero): add half
// a TF32 unit to the magnitude bits and clear the 13 low mantissa bits.  A carry
// into the exponent gives the correctly rounded next binade.
__device__ __forceinline__ uint32_t round_tf32(uint32_t bits)
{
    return (bits + 0x1000u) & 0xFFFFE000u;
}

// x = hi + lo with hi, lo both TF32: |x - hi| <= 2^-11 |x| and lo = round(x - hi),
// so hi + lo is within ~2^-22 |x| of x.  Full-rate integer and FP32 operations
// only (no conversion instruction).
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo)
{
    hi = round_tf32(__float_as_uint(x));
    lo = round_tf32(__float_as_uint(x - __uint_as_float(hi)));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Reduced-precision product (AM_BF16): one m16n8k8.bf16 product of the
// operands rounded to BF16.  The k index of the fragment is permuted
// (fragment k = 2t, 2t+1 <-> columns t, t+4 of the step), identically in A
// and B, so the same loads serve the TF32 and BF16 forms.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const float (&a)[4], float b0, float b1)
{
    const uint32_t a01 = pack_bf16(a[0], a[2]), a23 = pack_bf16(a[1], a[3]), b = pack_bf16(b0, b1);
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a01), "r"(a23), "r"(b));
}

// One 16x8x8 step of D += A B on operands split into TF32 (hi, lo) pairs
// (the constants on the host, the residual rows and heading increments by
// the phases that produce them, so the tensor-core phases only load).
// PR = 0 (FP32 form): three products lo*hi, hi*lo, hi*hi into d0, d1, d2,
// which the caller sums at the end (passing one array twice shares a chain);
// PR = 1 (AM_TF32): hi*hi only; PR = 2 (AM_BF16): the hi parts rounded to BF16.
// a: A[g][k], A[g+8][k], A[g][k+4], A[g+8][k+4]; b: B[k][n], B[k+4][n] with
// g = lane/4, k = lane%4 within the step, n = lane/4 (PTX m16n8k8 layouts).
template <int PR>
__device__ __forceinline__ void mma_pairs(float (&d0)[4], float (&d1)[4], float (&d2)[4],
                                          const uint2 (&a)[4], uint2 b0, uint2 b1)
{
    if constexpr (PR == 0) {
        mma_tf32(d0, a[0].y, a[1].y, a[2].y, a[3].y, b0.x, b1.x);
        mma_tf32(d1, a[0].x, a[1].x, a[2].x, a[3].x, b0.y, b1.y);
        mma_tf32(d2, a[0].x, a[1].x, a[2].x, a[3].x, b0.x, b1.x);
    } else if constexpr (PR == 1) {
        mma_tf32(d2, a[0].x, a[1].x, a[2].x, a[3].x, b0.x, b1.x);
    } else {
        const float f[4] = {__uint_as_float(a[0].x), __uint_as_float(a[1].x), __uint_as_float(a[2].x),
                            __uint_as_float(a[3].x)};
        mma_bf16(d2, f, __uint_as_float(b0.x), __uint_as_float(b1.x));
    }
}

__device__ __forceinline__ void st_split(uint2 *dst, float v)
{
    uint2 w;
    split_tf32(v, w.x, w.y);
    *dst = w;
}

// The columns of one k-step are permuted so that the two k elements a lane
// holds (fragment k = t and t + 4) are the adjacent columns 2t, 2t + 1: one
// 128-bit load brings both (hi, lo) pairs.  A and B use the same permutation,
// so the product is unchanged.
__device__ __forceinline__ void ld_pair2(const uint2 *p, uint2 &e0, uint2 &e1)
{
    const uint4 v = *reinterpret_cast<const uint4 *>(p);
    e0 = make_uint2(v.x, v.y);
    e1 = make_uint2(v.z, v.w);
}

// Row of a fragment lane: lanes past the tile read a row of the same parity
// (their results are discarded; MMA rows are independent), keeping the
// neighbouring-row bank pattern.
__device__ __forceinline__ int frag_row(int g, int count)
{
    return g < count ? g : (count > 1 ? (g & 1) : 0);
}

// The same for 64-bit loads, whose 16-lane wavefronts hold four rows: a row
// equal to the lane's modulo 4 where the tile has one.
__device__ __forceinline__ int frag_row4(int g, int count)
{
    return g < count ? g : (g & 3) < count ? (g & 3) : 0;
}

__device__ __forceinline__ void split4(const float (&a)[4], uint2 (&ap)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) split_tf32(a[i], ap[i].x, ap[i].y);
}

// ------------------------------------------------------------------ small

// atan2 for the heading target psi_t = atan2(s, c).  Octant reduction to
// a = min(|x|, |y|) / max(|x|, |y|) in [0, 1], atan(a) = a P(a^2) with P of
// degree 8 fitted for this kernel (iteratively reweighted least squares,
// Lawson's method, on [0, 1]: relative error 1.5e-8 in exact arithmetic,
// within 2 ulp when evaluated in FP32), then the octant is restored.
// atan2(0, 0) = 0, the reading the method takes.
__device__ __constant__ const float kAtanPoly[9] = {1.0f, -0.33333072f, 0.1999262f, -0.14203647f, 0.106409416f,
                                                    -0.07504311f, 0.042691723f, -0.016068758f, 0.002849923f};

__device__ __forceinline__ float atan2_heading(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    const float s = a * a;
    float p = kAtanPoly[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) p = fmaf(p, s, kAtanPoly[k]);
    float r = a * p;
    if (ay > ax) r = 1.57079637f - r;
    if (x < 0.f) r = 3.14159274f - r;
    return copysignf(r, y);  // the sign of y, -0 included (atan2(-0, -1) = -pi)
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

using KParams = FusedProblem;

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
// Position step on the tensor cores, one 16-row tile (row = side*8 + trajectory):
//   D[row][np] = sum_k A[row][k] Bt[np][k],  A = [lam + coef R | xi1],  Bt = [Minv | -Minv Q]
// on padded indices (k, np in 0..23 per side, 11 and 23 are zero pads), then
// xi1' = xi1 + D.  The whole block first forms A (split into TF32 pairs) and
// lam' once; three warp tasks, one per n-tile of 8 output columns, then run
// the products.
__device__ void xi1_operand(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur,
                            bool first)
{
    const float rho = p.L.rho, coef = first ? rho : 2.f * rho;
    uint2 *XA = reinterpret_cast<uint2 *>(sm + S.XA);
    // the tile's lam + coef R entries first, then its xi1 entries, so that
    // the threads summing the partials of R fill whole warps
    const int nr = tl.count * 48;
    for (int i = threadIdx.x; i < 2 * nr; i += blockDim.x) {
        const bool lam_part = i < nr;
        const int j = lam_part ? i : i - nr;
        const int tt = j / 48, o = j - 48 * tt, side = o / 24;
        const int k = lam_part ? o - 24 * side : o - 24 * side + 24;
        const int src = (cur * p.T + tt) * 48 + o;
        float v;
        if (lam_part) {
            const float lam = sm[S.lam + src], R = rsum(sm, S, tt * 48 + o);
            v = fmaf(coef, R, lam);
            sm[S.lam + ((cur ^ 1) * p.T + tt) * 48 + o] = first ? lam : fmaf(rho, R, lam);
        } else {
            v = sm[S.xi1 + src];
        }
        st_split(XA + (side * S.T + tt) * 56 + k, v);
    }
}

__device__ void xi1_mma(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur)
{
    const ConstLayout &L = p.L;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    const bool valid = g < tl.count;
    const int row = frag_row(g, tl.count);
    const uint2 *XA = reinterpret_cast<const uint2 *>(sm + S.XA);
    const uint2 *a_lo = XA + row * 56, *a_hi = XA + (S.T + row) * 56;
    for (int nt = warp; nt < 3; nt += blockDim.x >> 5) {
        const uint2 *brow = reinterpret_cast<const uint2 *>(sm + S.cst + L.off_xib2) + (nt * 8 + g) * 56;
        float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f}, d2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 6; ++ks) {
            const int c0 = ks * 8 + 2 * tq;  // permuted k-step columns
            uint2 a[4], b0, b1;
            ld_pair2(a_lo + c0, a[0], a[2]);
            ld_pair2(a_hi + c0, a[1], a[3]);
            ld_pair2(brow + c0, b0, b1);
            mma_pairs<0>(d0, d1, d2, a, b0, b1);
        }
        if (valid) {
            const float *xi = sm + S.xi1 + (cur * p.T + g) * 48;
            float *xi_n = sm + S.xi1 + ((cur ^ 1) * p.T + g) * 48;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = nt * 8 + 2 * tq + (e & 1);
                if (c == NV || c == 23) continue;  // pads stay zero
                const int o = (e >> 1) * 24 + c;
                xi_n[o] = xi[o] + (d0[e] + d1[e] + d2[e]);
            }
        }
    }
}

__device__ void phase_xi1(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur,
                          bool first, bool solve, bool sums, bool final_out, int kprev)
{
    const ConstLayout &L = p.L;
    const float *cst = sm + S.cst;
    const float rho = L.rho;
    const int Tn = tl.count;
    // With the position step on the tensor cores (warps 0..2), the remaining
    // tasks go to the threads after them when the block has enough.
    const int n_xi = solve ? 0 : Tn * 44, n_lp = Tn * NV, n_sc = sums ? Tn * 4 : 0;
    const int ntask = n_xi + n_lp + n_sc;
    int base = 0;
    if (solve) {
        xi1_operand(p, sm, S, tl, cur, first);
        __syncthreads();
        xi1_mma(p, sm, S, tl, cur);
        if (int(blockDim.x) >= 96 + ntask) base = 96;
    }
    const int stride = int(blockDim.x) - base;
    for (int task = int(threadIdx.x) - base; task >= 0 && task < ntask; task += stride) {
        if (task < n_xi) {
            const int tt = task / 44, rem = task - 44 * tt, side = rem / NS, row = rem - NS * side;
            const float *lam = sm + S.lam + (cur * p.T + tt) * 48 + 24 * side;
            const float *xi = sm + S.xi1 + (cur * p.T + tt) * 48 + 24 * side;
            const int rbase = tt * 48 + 24 * side;
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
                    a0 = fmaf(cst[L.off_mt + c * 24 + row], fmaf(coef, rsum(sm, S, rbase + cp), lam[cp]), a0);
                    a1 = fmaf(cst[L.off_mq + c * 24 + row], xi[cp], a1);
                }
                xn += a0 - a1;
            }
            xi_n[rp] = xn;
            lam_n[rp] = first ? lam[rp] : fmaf(rho, rsum(sm, S, rbase + rp), lam[rp]);
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
            const float *gv = sm + S.GX + (tt * 4 + w) * L.qs;
            float v;
            if (w < 3) {
                // the reductions over the steps of the residuals and the cost
                // accumulate in FP64 (q terms of similar size each)
                const float4 *g = reinterpret_cast<const float4 *>(gv);
                double acc = 0.0;
                for (int i = 0; i < L.qs / 4; ++i) {  // padding past q is zero
                    const float4 x = g[i];
                    acc += (double(x.x) + double(x.y)) + (double(x.z) + double(x.w));
                }
                v = float(w < 2 ? sqrt(acc) : acc);
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

// Mpsi lam_psi - Mpsi H xi2 for the heading step, row j of trajectory tt
// (i = tt * NV + j).  Formed after XI1 has updated lam_psi and before the
// PSI epilogue applies the step: in the PSI phase by warps that have no MMA
// task when the block has them, else by the whole block in the EVAL phase.
__device__ __forceinline__ void heading_base(const KParams &p, float *sm, const Smem &S, int i, int cur2)
{
    const ConstLayout &L = p.L;
    const float *cst = sm + S.cst;
    const int tt = i / NV, j = i - NV * tt;
    const float *lp = sm + S.lps + tt * 12;
    const float *x2 = sm + S.xi2 + (cur2 * p.T + tt) * 12;
    float b0 = 0.f, b1 = 0.f;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        b0 = fmaf(cst[L.off_mpsi + c * 12 + j], lp[c], b0);
        b1 = fmaf(cst[L.off_mpsih + c * 12 + j], x2[c], b1);
    }
    sm[S.bas + tt * 12 + j] = b0 - b1;
}

// Warps of the PSI phase: twelve (n-tile, quarter) MMA tasks when the block
// has twelve warps, and three more forming the heading base when it has
// fifteen (tile * NV <= 88 rows).
constexpr int kBaseWarps = 3;

__device__ __forceinline__ bool base_in_psi()
{
    return int(blockDim.x >> 5) >= 3 * kPsiParts + kBaseWarps;
}

// DOT phase on the tensor cores.  One 16-row tile: row = side*8 + trajectory.
// 4 kDotParts warp tasks: (segment rv | ra | r0 | r1, part of the steps),
// each for both n-tiles of 8 output columns, so a task loads its A fragment
// once (FP32, split here) for two products.  Each task writes its own partial
// of R (rv, ra, r0 -> c_pos rows of partial kDotParts seg + part; r1 -> c_slack
// rows of partial part), so no two tasks write one word.  A block with fewer
// warps runs the tasks in turn.  Few long tasks measured faster than many
// short ones: every partial costs shared-memory stores here and loads in XI1.
template <int PR>
__device__ void phase_dot(const KParams &p, float *sm, const Smem &S, const Tile &tl)
{
    const ConstLayout &L = p.L;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    const int nks = (L.q + 7) >> 3, per = (nks + kDotParts - 1) / kDotParts;
    const int row = frag_row4(g, tl.count);
    for (int task = warp; task < 4 * kDotParts; task += blockDim.x >> 5) {
        const int seg = task / kDotParts, part = task - kDotParts * seg;
        const int bsel = seg == 0 ? 1 : seg == 1 ? 2 : 0;  // Pd, Pdd, P, P
        const uint2 *B = reinterpret_cast<const uint2 *>(sm + S.cst + L.off_pcol2) + bsel * NV * L.qp;
        // n-tile 1 holds columns 8..10; its other lanes give discarded
        // outputs and read real columns of the same parity
        const uint2 *bc0 = B + g * L.qp, *bc1 = B + (g < 3 ? 8 + g : g) * L.qp;
        const float *a_lo = sm + S.G2 + row * S.RS + seg * L.qp;
        const float *a_hi = sm + S.G2 + (S.T + row) * S.RS + seg * L.qp;
        // the two cross products (lo*hi, hi*lo) share an accumulator: two
        // chains per n-tile (measured faster than three, fewer registers)
        float d0[4] = {0.f, 0.f, 0.f, 0.f}, d2[4] = {0.f, 0.f, 0.f, 0.f};
        float e0[4] = {0.f, 0.f, 0.f, 0.f}, e2[4] = {0.f, 0.f, 0.f, 0.f};
        const int k0 = part * per, k1 = min(nks, k0 + per);
#pragma unroll 1
        for (int ks = k0; ks < k1; ++ks) {
            const int c0 = ks * 8 + 2 * tq;
            const float2 lo = *reinterpret_cast<const float2 *>(a_lo + c0);
            const float2 hi = *reinterpret_cast<const float2 *>(a_hi + c0);
            const float a[4] = {lo.x, hi.x, lo.y, hi.y};
            uint2 ap[4], b0, b1, b2, b3;
            split4(a, ap);
            ld_pair2(bc0 + c0, b0, b1);
            ld_pair2(bc1 + c0, b2, b3);
            mma_pairs<PR>(d0, d0, d2, ap, b0, b1);
            mma_pairs<PR>(e0, e0, e2, ap, b2, b3);
        }
        if (g < tl.count) {
            float *R = sm + S.rb + (seg < 3 ? kDotParts * seg + part : part) * S.T * 48 + g * 48;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int side = e >> 1, c = 2 * tq + (e & 1);
                R[24 * side + (seg < 3 ? c : 12 + c)] = d0[e] + d2[e];
                if (c < 3) R[24 * side + (seg < 3 ? 8 + c : 20 + c)] = e0[e] + e2[e];
            }
        }
    }
}

// PSI phase on the tensor cores: W^T delta (cols 0..10) and P^T delta (cols
// 11..21) per trajectory; rows 0..7 = trajectories, rows 8..15 are zero.  The
// heading step is then applied once per coefficient:
//   xi2' = xi2 + (Mpsi lam_psi - Mpsi H xi2) + rho W^T delta
// (the first bracket formed by the base warps of this phase, or in the EVAL
// phase on a small block), writing xi2' and the increment.
// Partials over four quarters of the steps (three n-tiles each) are written,
// the task warps meet at a named barrier, and the first of them sum the
// partials and apply the step.
__device__ __forceinline__ void psi_apply(const KParams &p, float *sm, const Smem &S, int g, int c,
                                          float v, int cur2)
{
    if (c < NV) {
        const float d = fmaf(p.L.rho, v, sm[S.bas + g * 12 + c]);
        sm[S.xi2 + ((cur2 ^ 1) * p.T + g) * 12 + c] = sm[S.xi2 + (cur2 * p.T + g) * 12 + c] + d;
        sm[S.dx2 + g * 12 + c] = d;
    } else if (c < NS) {
        sm[S.ptp + g * 12 + (c - NV)] = v;
    }
}

template <int PR>
__device__ void phase_psi(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur2)
{
    const ConstLayout &L = p.L;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    const int nks = (L.q + 7) >> 3, per = (nks + kPsiParts - 1) / kPsiParts;
    // Twelve task warps take one (n-tile, quarter) each; a smaller block has
    // three, each running its n-tile's four quarters in turn.  Either way every
    // quarter's partial is formed alone and the four are added in the same
    // order, so the result does not depend on the block size.
    const bool split = (blockDim.x >> 5) >= 3 * kPsiParts;
    const int ntask = split ? 3 * kPsiParts : 3;
    // warps ntask .. ntask + nbase - 1 form the heading base and hand it to
    // the epilogue through the named barrier (arrive, no wait)
    const int nbase = base_in_psi() ? kBaseWarps : 0;
    const int nbar = 32 * (ntask + nbase);
    const float *arow = sm + S.PS + frag_row4(g, tl.count) * L.qp;
    const uint2 z = make_uint2(0u, 0u);
    if (warp < ntask) {
        const int nt = warp % 3;
        const int col = nt * 8 + g;
        // columns 22, 23 give discarded outputs: read columns of the same parity
        const uint2 *bcol = col < NV ? reinterpret_cast<const uint2 *>(sm + S.cst + L.off_wcol2) + col * L.qp
                                     : reinterpret_cast<const uint2 *>(sm + S.cst + L.off_pcol2) +
                                           (col < NS ? col - NV : col - NV - 8) * L.qp;
        // one quarter's partial of this warp's n-tile
        auto quarter = [&](int part) {
            float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f}, d2[4] = {0.f, 0.f, 0.f, 0.f};
            const int k0 = part * per, k1 = min(nks, k0 + per);
#pragma unroll 2
            for (int ks = k0; ks < k1; ++ks) {
                const int c0 = ks * 8 + 2 * tq;
                const float2 av = *reinterpret_cast<const float2 *>(arow + c0);
                uint2 a[4], b0, b1;
                split_tf32(av.x, a[0].x, a[0].y);
                split_tf32(av.y, a[2].x, a[2].y);
                a[1] = z;
                a[3] = z;
                ld_pair2(bcol + c0, b0, b1);
                mma_pairs<PR>(d0, d1, d2, a, b0, b1);
            }
            if (g < tl.count) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int c = nt * 8 + 2 * tq + e;
                    if (c < NS) sm[S.psp + (part * kMaxTile + g) * 24 + (c < NV ? c : c + 1)] = d0[e] + d1[e] + d2[e];
                }
            }
        };
        if (split) {
            quarter(warp / 3);
        } else {
#pragma unroll 1
            for (int part = 0; part < kPsiParts; ++part) quarter(part);
        }
        // the task and base warps only (barrier 0 is the block's)
        asm volatile("bar.sync 1, %0;\n" :: "r"(nbar) : "memory");
        for (int i = threadIdx.x; i < tl.count * NS; i += 32 * ntask) {
            const int tt = i / NS, c = i - NS * tt, o = c < NV ? c : c + 1;
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < kPsiParts; ++k) v += sm[S.psp + (k * kMaxTile + tt) * 24 + o];
            psi_apply(p, sm, S, tt, c, v, cur2);
        }
    } else if (warp < ntask + nbase) {
        const int i = int(threadIdx.x) - 32 * ntask;
        if (i < tl.count * NV) heading_base(p, sm, S, i, cur2);
        __threadfence_block();
        asm volatile("bar.arrive 1, %0;\n" :: "r"(nbar) : "memory");
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
// boundary-consistent reference), else from r as well.  x2 holds the heading
// coefficients to use.  RES also accumulates the step's squared residual and
// cost; FIN the smallest squared ellipse distance.
template <int M, bool LIT, bool RES, bool FIN, bool PRO>
__device__ __forceinline__ void sweep(float *sm, const Smem &S, const ConstLayout &L,
                                      const float (&x2)[12], int t, int tt,
                                      const float (&Prow)[12], StepRegs &r, const StepRegs &ref)
{
    const float *cst = sm + S.cst;
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
    const float *obt = cst + L.off_obt;
    const int n = L.n;
    // One (circle, obstacle) pair of this step.
    auto pair = [&](int j) {
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
    };
    if (!LIT && !FIN) {
        // In the default alpha form the row correction of a circle outside
        // the ellipse is exactly zero (max(1, 1/d) - 1 = 0).  Every circle
        // lies within r_max max(1/a, 1/b) of the robot centre in the
        // ellipse-scaled frame, so obstacle j matters only when the centre is
        // near it.  The warp keeps the list of obstacles near any of its steps
        // (formed with a threshold widened by kNearMargin) and forms it again
        // only when one of its centres has moved farther than the margin;
        // then only the pairs of listed obstacles are visited.
        const unsigned act = __activemask();
        float2 *ref = reinterpret_cast<float2 *>(sm + S.NR) + tt * L.q + t;
        unsigned *list = reinterpret_cast<unsigned *>(sm + S.NM) + 2 * (threadIdx.x >> 5);
        const float2 c0 = *ref;
        const float mx = r.x - c0.x, my = r.y - c0.y;
        if (__any_sync(act, fmaf(mx, mx, my * my) > kNearMargin * kNearMargin)) {
            for (int j0 = 0; j0 < n; j0 += 32) {
                const int jn = min(32, n - j0);
                unsigned near = 0u;
                for (int jj = 0; jj < jn; ++jj) {
                    const int j = j0 + jj;
                    const float2 o = obs[j * L.qs + t];
                    const float4 c = obc[j];
                    const float u0 = fmaf(r.x, c.x, -o.x), v0 = fmaf(r.y, c.y, -o.y);
                    near |= (fmaf(u0, u0, v0 * v0) < obt[j] ? 1u : 0u) << jj;
                }
                near = __reduce_or_sync(act, near);
                if ((threadIdx.x & 31) == 0) list[j0 >> 5] = near;
            }
            *ref = make_float2(r.x, r.y);
            __syncwarp(act);
        }
        for (int j0 = 0; j0 < n; j0 += 32) {
            unsigned near = list[j0 >> 5];
            while (near) {
                const int jj = __ffs(near) - 1;
                near &= near - 1u;
                pair(j0 + jj);
            }
        }
    } else {
        for (int j = 0; j < n; ++j) pair(j);
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
    const int qs = L.qs;
    float *Gx = sm + S.G2 + tt * S.RS + t;   // side x: row tt
    float *Gy = Gx + S.T * S.RS;             // side y: row T + tt
    const float svm = sv - 1.f, sam = sa - 1.f;
    // v and a rows: projected value - F xi1 value
    const int qp = L.qp;
    Gx[0] = PRO ? fmaf(r.xd, svm, r.xd - ref.xd) : r.xd * svm;
    Gx[qp] = PRO ? fmaf(r.xdd, sam, r.xdd - ref.xdd) : r.xdd * sam;
    Gx[2 * qp] = r0x;
    Gx[3 * qp] = r1x + dcx;
    Gy[0] = PRO ? fmaf(r.yd, svm, r.yd - ref.yd) : r.yd * svm;
    Gy[qp] = PRO ? fmaf(r.ydd, sam, r.ydd - ref.ydd) : r.ydd * sam;
    Gy[2 * qp] = r0y;
    Gy[3 * qp] = r1y + dsy;
    float *GX = sm + S.GX + tt * 4 * qs + t;
    if (RES) {
        GX[0] = v2 * svm * svm + a2 * sam * sam + rob + dcx * dcx + dsy * dsy;
        const float dp = psi - r.psi_t;
        GX[qs] = dp * dp;
        GX[2 * qs] = fmaf(r.xdd, r.xdd, fmaf(r.ydd, r.ydd, psidd * psidd));
    }
    if (FIN) GX[3 * qs] = dmin;
    r.psi_prev = psi;
    r.psi_cur = psi;
}

template <int M, bool LIT>
__device__ void sweep_dispatch(float *sm, const Smem &S, const ConstLayout &L, const float (&x2)[12],
                               int tt, int t, const float (&Prow)[12], StepRegs &r, bool res,
                               bool fin)
{
    if (fin) sweep<M, LIT, true, true, false>(sm, S, L, x2, t, tt, Prow, r, r);
    else if (res) sweep<M, LIT, true, false, false>(sm, S, L, x2, t, tt, Prow, r, r);
    else sweep<M, LIT, false, false, false>(sm, S, L, x2, t, tt, Prow, r, r);
}

// Stage a problem's constant block into shared memory with one bulk async
// copy and zero the rest of the dynamic area (the padding of the per-step
// arrays past q, and the unused rows of the MMA tiles, must read as zero).
// The wait on the mbarrier is bounded, and the block agrees on its outcome
// before anyone leaves, so no thread is left waiting at a barrier.
__device__ bool stage_constants(const KParams &p, float *sm, const Smem &S, uint64_t *bar,
                                uint32_t parity)
{
    if (threadIdx.x == 0) {
        const uint32_t bytes = uint32_t(p.L.total - p.L.off_fused) * 4u;
        // order the block's earlier generic-proxy accesses of this area
        // before the asynchronous copy overwrites it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
        if (!p.L.diag_stall) bulk_load(sm + S.cst + p.L.off_fused, p.cblob + p.L.off_fused, bytes, bar);
    }
    for (int i = S.xi1 + threadIdx.x; i < S.total; i += blockDim.x) sm[i] = 0.f;
    int ok = 0;
    const uint64_t t0 = global_ns();
    for (int spin = 0; spin < (1 << 26) && !ok; ++spin) {
        ok = mbar_try_wait(bar, parity) ? 1 : 0;
        if (!ok && global_ns() - t0 > kWaitLimitNs) break;
    }
    return __syncthreads_and(ok) != 0;
}

__device__ void init_barrier(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
}

// All iterations of the AM loop for one tile of trajectories of one problem
// whose constants are staged in shared memory.
template <int M, bool LIT, int PR = 0>
__device__ void run_tile(const KParams &p, float *sm, const Smem &S, const Tile &tl)
{
    const ConstLayout &L = p.L;
    const int Tn = tl.count;
    // The tile's state: xi1, xi2 as given into buffer 1, multipliers into buffer 0.
    for (int i = threadIdx.x; i < Tn * STATE; i += blockDim.x) {
        const int tt = i / STATE, e = i - STATE * tt;
        const float v = p.state[(size_t)tl.first * STATE + i];
        if (e < 44) sm[S.xi1 + (p.T + tt) * 48 + (e / NV) * 12 + e % NV] = v;
        else if (e < 55) sm[S.xi2 + (p.T + tt) * 12 + (e - 44)] = v;
        else if (e < 99) sm[S.lam + tt * 48 + ((e - 55) / NV) * 12 + (e - 55) % NV] = v;
        else sm[S.lps + tt * 12 + (e - 99)] = v;
    }
    for (int i = threadIdx.x; i < kRParts * p.T * 48; i += blockDim.x) sm[S.rb + i] = 0.f;
    // no near lists yet: a reference far away makes every warp form its list
    for (int i = threadIdx.x; i < 2 * p.T * L.q; i += blockDim.x) sm[S.NR + i] = 3.0e18f;
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
    // The thread's basis row P[t, :] is reloaded where it is used, so it does
    // not occupy registers through the tensor-core phases.
    const float *prow = sm + S.cst + L.off_prow + t * 12;
    StepRegs r;
    r.psi_t = 0.f;
    int cur = 0, cur2 = 0;

    // Step 1 of Sec. III-D: xi3, xi4 and g from the initial samples, the
    // residual against the reference.
    if (stepper) {
        StepRegs ref;
        float x2[12], Prow[12];
        load12(Prow, prow);
        eval_xy(sm, S, L, sm + S.xi1 + (p.T + tt) * 48, t, Prow, r);
        eval_xy(sm, S, L, sm + S.xi1 + tt * 48, t, Prow, ref);
        load12(x2, sm + S.xi2 + (p.T + tt) * 12);
        sweep<M, LIT, false, false, true>(sm, S, L, x2, t, tt, Prow, r, ref);
        load12(x2, sm + S.xi2 + tt * 12);
        r.psi_cur = dot11(Prow, x2);  // heading of the reference c_psi
    }
    __syncthreads();
    phase_dot<PR>(p, sm, S, tl);
    __syncthreads();

    for (int k = 0; k < p.iters; ++k) {
        const bool res = (p.hist != nullptr) || (k == p.iters - 1);
        const bool prev_res = (p.hist != nullptr) && k > 0;
        phase_xi1(p, sm, S, tl, cur, k == 0, true, prev_res, false, k - 1);
        cur ^= 1;
        __syncthreads();
        if (stepper) {
            float Prow[12];
            load12(Prow, prow);
            eval_xy(sm, S, L, sm + S.xi1 + (cur * p.T + tt) * 48, t, Prow, r);
            // psi_t = psi + wrap(atan2(s, c) - psi), psi the previous heading;
            // the heading step works on delta = psi_t - P xi2
            r.psi_t = r.psi_prev + wrap_pi(atan2_heading(r.s, r.c) - r.psi_prev);
            sm[S.PS + tt * L.qp + t] = r.psi_t - r.psi_cur;
        }
        if (!base_in_psi())
            for (int i = threadIdx.x; i < Tn * NV; i += blockDim.x) heading_base(p, sm, S, i, cur2);
        __syncthreads();
        phase_psi<PR>(p, sm, S, tl, cur2);
        __syncthreads();
        if (stepper) {
            float x2[12];
            load12(x2, sm + S.xi2 + ((cur2 ^ 1) * p.T + tt) * 12);  // xi2' from the PSI phase
            float Prow[12];
            load12(Prow, prow);
            sweep_dispatch<M, LIT>(sm, S, L, x2, tt, t, Prow, r, res, k == p.iters - 1);
        }
        cur2 ^= 1;
        __syncthreads();
        phase_dot<PR>(p, sm, S, tl);
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

template <int M, bool LIT, int PR>
__global__ void __launch_bounds__(kMaxThreads, 1) am_fused_kernel(KParams p)
{
    extern __shared__ __align__(128) float sm[];
    const Smem S = smem_layout(p.L, p.T);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S.bar);
    init_barrier(bar);
    if (!stage_constants(p, sm, S, bar, 0)) {
        if (threadIdx.x == 0) atomicExch(p.err, 1);
        return;
    }
    for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x)
        run_tile<M, LIT, PR>(p, sm, S, tile_of(tile, p.B, p.ntiles));
}

// Uneven batching: persistent launches over the tiles of many problems of
// different batch size, horizon, obstacle and circle counts, one kernel per
// variant (circle count M, alpha form LIT) so that each is compiled on its
// own (the variants inlined into one kernel spill registers).  The variant
// kernels of one solve run concurrently; CTAs take work items (problem,
// tile) of their variant from a list in order, through one atomic counter
// per variant, and re-stage constants whenever they move to another problem.
// The lists, their lengths and offsets live in device memory, so a captured
// launch stays valid when the set of problems it advances changes.
//   head[v]: number of items of variant v; head[8 + v]: offset of its list
//   ctl[2 v]: its work counter (zeroed before the launch); ctl[2 v + 1]: status
template <int M, bool LIT>
__global__ void __launch_bounds__(kMaxThreads, 1)
am_group_kernel(const KParams *probs, const int *items, const int *head, int *ctl)
{
    constexpr int v = M * 2 + (LIT ? 1 : 0) - 2;
    int *counter = ctl + 2 * v;
    const int nitems = head[v];
    const int *list = items + 2 * head[8 + v];
    extern __shared__ __align__(128) float sm[];
    __shared__ KParams kp;
    __shared__ int s_item;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);  // fixed: the layout below starts past it
    init_barrier(bar);
    int cur = -1;
    uint32_t parity = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 item = make_int2(list[2 * it], list[2 * it + 1]);
        if (item.x != cur) {
            if (threadIdx.x == 0) kp = probs[item.x];
            __syncthreads();
            if (!stage_constants(kp, sm, smem_layout(kp.L, kp.T), bar, parity)) {
                if (threadIdx.x == 0) {
                    atomicExch(kp.err, 1);
                    atomicExch(ctl + 2 * v + 1, 1);
                }
                return;
            }
            parity ^= 1u;
            cur = item.x;
        }
        run_tile<M, LIT>(kp, sm, smem_layout(kp.L, kp.T), tile_of(item.y, kp.B, kp.ntiles));
        __syncthreads();
    }
}

}  // namespace

// The group kernel's static shared memory (its problem descriptor) comes out
// of the same 227 KB as the dynamic area.
constexpr size_t kGroupSmemMax = 227 * 1024 - 512;

size_t fused_smem_bytes(const ConstLayout &L, int tile)
{
    return size_t(smem_layout(L, tile).total) * sizeof(float);
}

int fused_max_tile(const ConstLayout &L)
{
    int tmax = kMaxThreads / (L.q > 88 ? L.q : 88);
    if (tmax > kMaxTile) tmax = kMaxTile;
    while (tmax > 1 && fused_smem_bytes(L, tmax) > 227 * 1024) --tmax;
    return tmax < 1 ? 1 : tmax;
}

int fused_max_threads() { return kMaxThreads; }

int group_tile(const ConstLayout &L, int threads)
{
    int t = threads / (L.q > 88 ? L.q : 88);
    if (t > kMaxTile) t = kMaxTile;
    while (t >= 1 && fused_smem_bytes(L, t) > kGroupSmemMax) --t;
    return t < 1 ? 0 : t;
}

int launch_group(const GroupLaunch &g, void *stream, int *launches, const char **why)
{
    *why = nullptr;
    if (g.threads < 32 || g.threads > kMaxThreads || g.smem > kGroupSmemMax || g.grid < 1 ||
        g.variant < 0 || g.variant >= kGroupVariants)
        return -1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the variant's work counter and status word start at zero every solve
    cudaError_t e = cudaMemsetAsync(g.d_ctl + 2 * g.variant, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return -2;
    }
    switch (g.variant) {
#define AM_GCASE(MM, LL)                                                                        \
    case MM * 2 + LL - 2:                                                                       \
        e = cudaFuncSetAttribute(am_group_kernel<MM, LL>,                                       \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem));     \
        if (e != cudaSuccess) {                                                                 \
            *why = cudaGetErrorString(e);                                                       \
            return -2;                                                                          \
        }                                                                                       \
        am_group_kernel<MM, LL><<<g.grid, g.threads, g.smem, st>>>(g.d_probs, g.d_items, g.d_head, \
                                                                   g.d_ctl);                   \
        break;
        AM_GCASE(1, 0)
        AM_GCASE(1, 1)
        AM_GCASE(2, 0)
        AM_GCASE(2, 1)
        AM_GCASE(3, 0)
        AM_GCASE(3, 1)
        AM_GCASE(4, 0)
        AM_GCASE(4, 1)
#undef AM_GCASE
    default:
        return -1;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return -2;
    }
    if (launches) ++*launches;
    return 0;
}

int group_variant(const ConstLayout &L) { return L.m * 2 + (L.alpha_mode ? 1 : 0) - 2; }

int fused_auto_tile(const ConstLayout &L, int B, int num_sms)
{
    // Largest tile that fits one CTA per SM, then shrink so every SM gets work.
    const int tmax = fused_max_tile(L);
    int want = (B + num_sms - 1) / num_sms;
    if (want < 1) want = 1;
    return want < tmax ? want : tmax;
}

namespace {

// Launch configuration of the single-problem kernels, formed once and kept:
// the SM count per device, and per kernel variant the shared-memory limit
// (set to the 227 KB maximum) and the resident CTAs per SM for each (block,
// shared memory) size.  A solve then costs one launch and no driver queries.
std::mutex g_launch_mu;

int device_sms(int dev)
{
    static int cached_dev = -1, count = 0;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    if (cached_dev != dev) {
        if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cached_dev = dev;
    }
    return count;
}

template <int M, bool LIT, int PR>
int launch_variant(const KParams &p, int threads, size_t smem, int dev, int sms, cudaStream_t st)
{
    static int attr_dev = -1;
    static std::map<std::pair<int, size_t>, int> resident;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(g_launch_mu);
        if (attr_dev != dev) {
            if (cudaFuncSetAttribute(am_fused_kernel<M, LIT, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024) != cudaSuccess)
                return -2;
            resident.clear();
            attr_dev = dev;
        }
        const auto key = std::make_pair(threads, smem);
        const auto it = resident.find(key);
        if (it != resident.end()) {
            per_sm = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, am_fused_kernel<M, LIT, PR>, threads, smem) !=
                    cudaSuccess ||
                per_sm < 1)
                return -2;
            resident[key] = per_sm;
        }
    }
    // persistent CTAs: as many as can be resident at once (one per SM for the
    // large tiles; more when a smaller tile lets several share an SM)
    const int grid = p.ntiles < sms * per_sm ? p.ntiles : sms * per_sm;
    am_fused_kernel<M, LIT, PR><<<grid, threads, smem, st>>>(p);
    return 0;
}

}  // namespace

int launch_fused(const SolveArgs &a, void *stream, int *launches)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = device_sms(dev);
    if (sms < 1) return -2;
    const ConstLayout &L = a.L;
    int T = a.tile > 0 ? a.tile : fused_auto_tile(L, a.B, sms);
    const int tq = T * (L.q > 88 ? L.q : 88);
    if (tq > kMaxThreads || T < 1 || T > kMaxTile) return -1;
    const size_t smem = fused_smem_bytes(L, T);
    if (smem > 227 * 1024) return -1;
    const int threads = (tq + 31) & ~31;
    const int ntiles = (a.B + T - 1) / T;
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
    int rc = -1;
    const int sel = (L.precision * 8 + (L.m - 1) * 2) + (L.alpha_mode ? 1 : 0);
    switch (sel) {
#define AM_CASE(MM, LL, PP)                                                                   \
    case PP * 8 + (MM - 1) * 2 + LL:                                                          \
        rc = launch_variant<MM, LL, PP>(p, threads, smem, dev, sms, st);                      \
        break;
#define AM_CASES(PP)                                                                          \
        AM_CASE(1, 0, PP)                                                                     \
        AM_CASE(2, 0, PP)                                                                     \
        AM_CASE(3, 0, PP)                                                                     \
        AM_CASE(4, 0, PP)                                                                     \
        AM_CASE(1, 1, PP)                                                                     \
        AM_CASE(2, 1, PP)                                                                     \
        AM_CASE(3, 1, PP)                                                                     \
        AM_CASE(4, 1, PP)
        AM_CASES(0)
        AM_CASES(1)
        AM_CASES(2)
#undef AM_CASES
#undef AM_CASE
    default:
        return -1;
    }
    if (rc) return rc;
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam
