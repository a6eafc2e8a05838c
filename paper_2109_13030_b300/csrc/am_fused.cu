// Fused persistent kernel of the batched alternating-minimization loop
// (Sec. III-D, steps 1-5, and the batch solution of Sec. III-E).
//
// One CTA stays resident on each SM and works through tiles of T <= 8
// trajectories.  It stages the constant block into shared memory once (bulk
// async copies, completion on an mbarrier), keeps xi1, xi2, lambda,
// lambda_psi and the residual contraction R = F^T (g - F xi1) of every
// trajectory of the tile in shared memory for all iterations, and writes the
// state back only after the last one.  Nothing per element (alpha, d, g) is
// ever stored.
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
// Per-step work (the trajectory values of Eq. param, the heading target and
// the closed-form alpha/d steps) runs on one thread per pair of consecutive
// steps (t, t + 1) of a trajectory.  The thread keeps the basis rows P, Pd,
// Pdd of its two steps in registers for the whole tile and evaluates both
// steps with paired FP32 instructions (fma/mul/add on float2, each component
// rounded exactly like its scalar form); the coefficients it reads are kept
// duplicated, (c, c), beside xi1 and xi2 so that one 128-bit load gives two
// paired operands.
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
//   EVAL  x, xdot, xddot, y, ..., c, s at the thread's two steps (Eq. param);
//         heading target psi_t and delta = psi_t - P xi2; Mpsi lam_psi -
//         Mpsi H xi2 for the heading step
//   PSI   W^T delta and P^T delta on the tensor cores, then
//         xi2 += Mpsi (lam_psi - H xi2) + rho W^T delta
//   SWEEP psi = P xi2; the closed-form alpha/d steps for every circle and
//         obstacle (Eq. zeta_2 - compute_da) in the trig-free form (xt, yt)
//         max(1, 1/sqrt(xt^2/a^2 + yt^2/b^2)), the velocity and acceleration
//         projections, and the per-step residual vectors of R
//   DOT   R on the tensor cores
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "am_async.cuh"
#include "am_heading.cuh"
#include "am_internal.h"

namespace trajam {
namespace {

constexpr int kMaxThreads = 384;  // twelve warps: every tensor-core task of a phase at once
constexpr int kMaxTile = 8;       // rows (side, trajectory) of one 16-row MMA tile
constexpr int kDotParts = 2;      // parts of the steps per segment of R in the DOT phase
constexpr int kRParts = 3 * kDotParts;  // partials of R: (rv | ra | r0 segment) x part of the steps
constexpr int kMinPairThreads = 44;  // threads per trajectory at least (short horizons)


// Threads per trajectory: one per pair of consecutive steps.
__host__ __device__ inline int pair_threads(int q)
{
    const int np = (q + 1) / 2;
    return np > kMinPairThreads ? np : kMinPairThreads;
}

struct Smem {
    int cst, cob, xi1, lam, rb, xi2, dx2, lps, ptp, G2, RS, GX, U, PTD, XD, X2D, bar, total, T;
};

// Debug build (-DAM_DEBUG_BOUNDS, libtrajam_debug.so): every checked index
// outside its array sets the block's flag and the access is skipped; at the
// end of a tile the flag becomes bit 2 of the problem's status word, which
// the host reports as AM_ERR_STATE.  There is no trap.  In the release build
// the checks compile to nothing.
#ifdef AM_DEBUG_BOUNDS
__shared__ int g_oob;
#define AM_BOUND(cond) ((cond) ? true : (g_oob = 1, false))
#else
#define AM_BOUND(cond) true
#endif

// Shared-memory layout (float offsets).
//   cst region [off_fused, off_obs) of the constant block (shape sections);
//   cob region [off_obt, total) (near thresholds, paired obstacle sections)
//   xi1, lam  [2][T][48]   double-buffered, padded blocks of 12 per polynomial
//   rb        [3D][T][48]  partials of R per side (c_pos rows 0..10, c_slack rows
//                          12..22), D = kDotParts: (rv, ra, r0 segment) x part of
//                          the steps; the c_slack rows in the first D (R is the sum of all)
//   xi2       [2][T][12]   double-buffered c_psi;  dx2 [T][12] last increment
//   lps       [T][12]      lambda_psi
//   ptp       [8][12]      P^T delta of the last heading step
//   G2        [2T][RS]     residual vectors, row = side*T + trajectory; segments
//                          rv | ra | r0 | r1 of qp steps
//   GX        [T][4][qs]   per-step squared residual, heading residual, cost, distance
//   U         [T][48]      lam + coef R per side (padded), the position step's input
//   PTD       [T][np][12]  P^T delta over the two steps of each stepper thread
//   XD        [2][T][12][4][2] xi1 duplicated per coefficient k: (cx, cx, cy, cy,
//                          cc, cc, cs, cs), both buffers
//   X2D       [2][T][12][2] xi2 duplicated, both buffers
// The constant block's shape sections are staged so that sm + cst + off_x
// addresses section x; the obstacle region starts at cob (off_obt there).
__host__ __device__ inline Smem smem_layout(const ConstLayout &L, int T)
{
    Smem s;
    int o = 0;
    s.T = T;
    s.bar = o; o += 4;  // one 8-byte mbarrier at a fixed offset, 16-byte aligned
    s.cst = o - L.off_fused; o += L.off_obs - L.off_fused;
    s.cob = o; o += L.total - L.off_obt;
    s.xi1 = o; o += 2 * T * 48;
    s.lam = o; o += 2 * T * 48;
    s.rb = o; o += kRParts * T * 48;
    s.xi2 = o; o += 2 * T * 12;
    s.dx2 = o; o += T * 12;
    s.lps = o; o += T * 12;
    s.ptp = o; o += kMaxTile * 12;
    // RS = 8 mod 32 and qp = 8 mod 16: the 64-bit fragment loads of four
    // neighbouring rows fall on distinct banks
    s.RS = 4 * L.qp + 8;
    s.G2 = o; o += 2 * T * s.RS;
    s.GX = o; o += T * 4 * L.qs;
    s.U = o; o += T * 48;
    s.PTD = o; o += T * ((L.q + 1) / 2) * 12;
    s.XD = o; o += 2 * T * 12 * 8;
    s.X2D = o; o += 2 * T * 12 * 2;
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

// Split BF16 (AM_SPLIT_BF16): x = hi + lo with hi = bf16(x), lo = bf16(x - hi)
// (16 significant bits), two values packed per register as the mma operands
// want them (the first value in the low half).
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    hi = pack_bf16(x0, x1);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
    lo = pack_bf16(x0 - h0, x1 - h1);
}

// D += A B, m16n8k16 with BF16 operands (a: rows g, g + 8 at k 2t, 2t + 1,
// then at k 2t + 8, 2t + 9; b: k 2t, 2t + 1, then 2t + 8, 2t + 9 at column g).
__device__ __forceinline__ void mma_bf16_k16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                             uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// The same with K = 8 (a: rows g, g + 8 at k 2t, 2t + 1; b: k 2t, 2t + 1).
__device__ __forceinline__ void mma_bf16_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
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

// Row of a fragment lane for 64-bit loads, whose 16-lane wavefronts hold four
// rows: lanes past the tile read the row equal to the lane's modulo 4 where the
// tile has one (their results are discarded; MMA rows are independent).
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

// Side-row r (0..21) of (c_pos, c_slack) -> padded index within a 24-float side block.
__device__ __forceinline__ int rowpad(int r) { return r < NV ? r : r + 1; }

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

// Position of polynomial block blk (0 c_x, 1 c_c, 2 c_y, 3 c_s) within a
// duplicated xi1 entry (cx, cx, cy, cy, cc, cc, cs, cs).
__device__ __forceinline__ int dpos(int blk) { return blk == 0 ? 0 : blk == 2 ? 1 : blk == 1 ? 2 : 3; }

// Writes entry o (padded index blk * 12 + k) of trajectory tt's xi1 into
// buffer buf, and its duplicate.
__device__ __forceinline__ void put_xi1(float *sm, const Smem &S, int buf, int tt, int o, float v)
{
    if (!AM_BOUND(buf >= 0 && buf < 2 && tt >= 0 && tt < S.T && o >= 0 && o < 48)) return;
    sm[S.xi1 + (buf * S.T + tt) * 48 + o] = v;
    const int blk = o / 12, k = o - 12 * blk;
    reinterpret_cast<float2 *>(sm + S.XD)[((buf * S.T + tt) * 12 + k) * 4 + dpos(blk)] = make_float2(v, v);
}

// The same for coefficient k of trajectory tt's xi2.
__device__ __forceinline__ void put_xi2(float *sm, const Smem &S, int buf, int tt, int k, float v)
{
    if (!AM_BOUND(buf >= 0 && buf < 2 && tt >= 0 && tt < S.T && k >= 0 && k < 12)) return;
    sm[S.xi2 + (buf * S.T + tt) * 12 + k] = v;
    reinterpret_cast<float2 *>(sm + S.X2D)[(buf * S.T + tt) * 12 + k] = make_float2(v, v);
}

// XI1 phase: the multiplier update of the finished iteration, the next xi1 in
// increment form, the lambda_psi update and the per-trajectory sums.
//   first: lam' = lam,          xi1' = xi1 + Minv (lam + rho R) - MQ xi1
//   later: lam' = lam + rho R,  xi1' = xi1 + Minv (lam + 2 rho R) - MQ xi1
//   post (no solve): lam' = lam + rho R, xi1' = xi1
// A first pass forms u = lam + coef R and lam' for every (trajectory, side,
// row), updates lambda_psi (Eq. update_lambda_psi) and reduces the sums of
// the last sweep; after a block barrier one thread per output row evaluates
// xi1' = xi1 + Minv u - MQ xi1 in FP32 (44 x 48 per trajectory: far too small
// for the tensor cores to pay for their operand traffic).
__device__ void phase_xi1(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur,
                          bool first, bool solve, bool sums, bool final_out, int kprev)
{
    const ConstLayout &L = p.L;
    const float *cst = sm + S.cst;
    const float rho = L.rho, coef = first ? rho : 2.f * rho;
    const int Tn = tl.count;
    const int n_op = Tn * 48, n_lp = first ? 0 : Tn * NV, n_sc = sums ? Tn * 4 : 0;
    const int ntask = n_op + n_lp + n_sc;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        if (task < n_op) {
            const int tt = task / 48, o = task - 48 * tt;
            const int src = (cur * p.T + tt) * 48 + o;
            const float lam = sm[S.lam + src], R = rsum(sm, S, tt * 48 + o);
            sm[S.lam + ((cur ^ 1) * p.T + tt) * 48 + o] = first ? lam : fmaf(rho, R, lam);
            if (solve) sm[S.U + tt * 48 + o] = fmaf(coef, R, lam);
            else put_xi1(sm, S, cur ^ 1, tt, o, sm[S.xi1 + src]);
        } else if (task < n_op + n_lp) {
            // P^T (P xi2' - psi_t) = P^T P dxi2 - P^T delta, delta = psi_t - P xi2
            const int s = task - n_op, tt = s / NV, k = s - NV * tt;
            const float *dx2 = sm + S.dx2 + tt * 12;
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < NV; ++c) a = fmaf(cst[L.off_ptp + c * 12 + k], dx2[c], a);
            float *lp = sm + S.lps + tt * 12;
            lp[k] -= L.psi_sign * L.rho_psi * (a - sm[S.ptp + tt * 12 + k]);
        } else {
            const int s = task - n_op - n_lp, tt = s >> 2, w = s & 3;
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
    if (!solve) return;
    __syncthreads();
    // one thread per (trajectory, side, row): Minv u - MQ xi1 on the side's
    // 22 unknowns, both read from their padded blocks (u, xi1 broadcast;
    // Minv^T and (MQ)^T rows contiguous over the outputs)
    for (int i = threadIdx.x; i < Tn * 2 * NS; i += blockDim.x) {
        const int tt = i / (2 * NS), rem = i - 2 * NS * tt, side = rem / NS, row = rem - NS * side;
        const float *u = sm + S.U + tt * 48 + 24 * side;
        const float *xi = sm + S.xi1 + (cur * p.T + tt) * 48 + 24 * side;
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int c = 0; c < NS; ++c) {
            const int cp = rowpad(c);
            a0 = fmaf(cst[L.off_mt + c * 24 + row], u[cp], a0);
            a1 = fmaf(cst[L.off_mq + c * 24 + row], xi[cp], a1);
        }
        const int rp = rowpad(row);
        put_xi1(sm, S, cur ^ 1, tt, 24 * side + rp, xi[rp] + (a0 - a1));
    }
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
        if (!AM_BOUND(8 * nks <= L.qp && row < S.T)) continue;  // operand columns within a segment
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
        if constexpr (PR == 3) {
            // split BF16: pairs of k-steps as one K = 16 product; lane tq takes
            // the four consecutive steps 4 tq .. 4 tq + 3 of the pair (k 2tq,
            // 2tq + 1 and 2tq + 8, 2tq + 9 of the product), in A and B alike
            int ks = k0;
#pragma unroll 1
            for (; ks + 2 <= k1; ks += 2) {
                const int c = ks * 8 + 4 * tq;
                const float4 x0 = *reinterpret_cast<const float4 *>(a_lo + c);  // row g (side x)
                const float4 x1 = *reinterpret_cast<const float4 *>(a_hi + c);  // row g + 8 (side y)
                uint32_t ah[4], al[4];
                split_bf16x2(x0.x, x0.y, ah[0], al[0]);
                split_bf16x2(x1.x, x1.y, ah[1], al[1]);
                split_bf16x2(x0.z, x0.w, ah[2], al[2]);
                split_bf16x2(x1.z, x1.w, ah[3], al[3]);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    // the basis column as stored: TF32 (hi, lo) pairs; their sum is exact in FP32
                    const uint4 p0 = *reinterpret_cast<const uint4 *>((nt ? bc1 : bc0) + c);
                    const uint4 p1 = *reinterpret_cast<const uint4 *>((nt ? bc1 : bc0) + c + 2);
                    const float b0 = __uint_as_float(p0.x) + __uint_as_float(p0.y);
                    const float b1 = __uint_as_float(p0.z) + __uint_as_float(p0.w);
                    const float b2 = __uint_as_float(p1.x) + __uint_as_float(p1.y);
                    const float b3 = __uint_as_float(p1.z) + __uint_as_float(p1.w);
                    uint32_t bh0, bl0, bh1, bl1;
                    split_bf16x2(b0, b1, bh0, bl0);
                    split_bf16x2(b2, b3, bh1, bl1);
                    float (&dc)[4] = nt ? e0 : d0;
                    float (&dh)[4] = nt ? e2 : d2;
                    mma_bf16_k16(dc, al[0], al[1], al[2], al[3], bh0, bh1);
                    mma_bf16_k16(dc, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
                    mma_bf16_k16(dh, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
                }
            }
            if (ks < k1) {
                // an odd last k-step: one K = 8 product per split term
                const int c0 = ks * 8 + 2 * tq;
                const float2 lo = *reinterpret_cast<const float2 *>(a_lo + c0);
                const float2 hi = *reinterpret_cast<const float2 *>(a_hi + c0);
                uint32_t ah0, al0, ah1, al1;
                split_bf16x2(lo.x, lo.y, ah0, al0);
                split_bf16x2(hi.x, hi.y, ah1, al1);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const uint4 p0 = *reinterpret_cast<const uint4 *>((nt ? bc1 : bc0) + c0);
                    uint32_t bh, bl;
                    split_bf16x2(__uint_as_float(p0.x) + __uint_as_float(p0.y),
                                 __uint_as_float(p0.z) + __uint_as_float(p0.w), bh, bl);
                    float (&dc)[4] = nt ? e0 : d0;
                    float (&dh)[4] = nt ? e2 : d2;
                    mma_bf16_k8(dc, al0, al1, bh);
                    mma_bf16_k8(dc, ah0, ah1, bl);
                    mma_bf16_k8(dh, ah0, ah1, bh);
                }
            }
        } else {
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


// PSI phase: the heading step of Eq. compute_convex_surrogate in increment
// form.  With W = P Mpsi^T, W^T delta = Mpsi P^T delta, so the step needs
// only P^T delta, which every stepper thread has already formed over its two
// steps in EVAL (its basis rows are in registers).  Warp tt sums trajectory
// tt's partials in a fixed order (lanes 2k, 2k + 1: the two halves of the
// steps for coefficient k) and applies
//   xi2' = xi2 + Mpsi (lam_psi + rho P^T delta) - Mpsi H xi2,
// writing xi2', the increment and P^T delta (for the lambda_psi update).
__device__ void phase_psi(const KParams &p, float *sm, const Smem &S, const Tile &tl, int cur2)
{
    const ConstLayout &L = p.L;
    const float *cst = sm + S.cst;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = (L.q + 1) >> 1, nh = (np + 1) >> 1;
    for (int tt = warp; tt < tl.count; tt += blockDim.x >> 5) {
        const int k = lane >> 1, half = lane & 1;
        float s = 0.f;
        if (k < NV) {
            const float *pt = sm + S.PTD + (tt * np) * 12 + k;
            const int j1 = half ? np : nh;
            for (int j = half ? nh : 0; j < j1; ++j) s += pt[j * 12];
        }
        const float ptp = s + __shfl_xor_sync(0xffffffffu, s, 1);  // same sum in both lanes
        const float *lp = sm + S.lps + tt * 12;
        const float *x2 = sm + S.xi2 + (cur2 * p.T + tt) * 12;
        float b0 = 0.f, b1 = 0.f;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const float pc = __shfl_sync(0xffffffffu, ptp, 2 * c);
            if (lane < NV) {
                b0 = fmaf(cst[L.off_mpsi + c * 12 + lane], fmaf(L.rho, pc, lp[c]), b0);
                b1 = fmaf(cst[L.off_mpsih + c * 12 + lane], x2[c], b1);
            }
        }
        if (lane < NV) {
            const float d = b0 - b1;
            put_xi2(sm, S, cur2 ^ 1, tt, lane, x2[lane] + d);
            sm[S.dx2 + tt * 12 + lane] = d;
        }
        if (half == 0 && k < NV) sm[S.ptp + tt * 12 + k] = ptp;
    }
}

// ------------------------------------------------------- paired step work
//
// Each stepper thread owns steps t0 = 2 j and t0 + 1 of one trajectory and
// holds every per-step quantity as a float2 (value at t0, value at t0 + 1).
// The paired instructions round each component exactly like the scalar
// instruction would.  When q is odd the last pair has no second step: its
// basis row is zero and every value it stores for that step is zero.

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// Stores (v.x at t0, v.y at t0 + 1), the second as zero past the horizon.
__device__ __forceinline__ void st2(float *p, float2 v, bool v1)
{
    *reinterpret_cast<float2 *>(p) = make_float2(v.x, v1 ? v.y : 0.f);
}

// Basis rows of the thread's two steps (Eq. param), kept in registers.
struct Basis {
    float2 P[NV], Pd[NV], Pdd[NV];
};

__device__ __forceinline__ void load_basis(const float *sm, const Smem &S, const ConstLayout &L, int t0,
                                           bool v1, Basis &b)
{
    const float *r = sm + S.cst + L.off_prow;  // [3][q][12]
    const int q = L.q, t1 = v1 ? t0 + 1 : t0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        b.P[k] = f2(r[t0 * 12 + k], v1 ? r[t1 * 12 + k] : 0.f);
        b.Pd[k] = f2(r[(q + t0) * 12 + k], v1 ? r[(q + t1) * 12 + k] : 0.f);
        b.Pdd[k] = f2(r[(2 * q + t0) * 12 + k], v1 ? r[(2 * q + t1) * 12 + k] : 0.f);
    }
}

struct Pair {
    float2 x, xd, xdd, y, yd, ydd, c, s;
    float2 psi_t;     // heading target atan2(s, c), unwrapped
    float2 psi_prev;  // heading the unwrap refers to (the previous P xi2)
    float2 psi_cur;   // P xi2 of the current coefficients
};

// Near-obstacle list of the thread's warp (the same in every lane) and the
// robot centres of the thread's two steps when it was formed.
struct Near {
    float2 rx, ry;
    unsigned list0, list1;  // obstacles 0..31, 32..63
};

// EVAL: trajectory values at the thread's two steps from trajectory tt's
// duplicated xi1 in buffer buf.
__device__ __forceinline__ void eval_pair(const float *sm, const Smem &S, int buf, int tt, const Basis &b,
                                          Pair &r)
{
    const float4 *xd = reinterpret_cast<const float4 *>(sm + S.XD) + (buf * S.T + tt) * 24;
    float2 x = f2(0.f, 0.f), vx = x, ax = x, c = x, y = x, vy = x, ay = x, s = x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float4 u = xd[2 * k], w = xd[2 * k + 1];  // (cx, cx, cy, cy), (cc, cc, cs, cs)
        const float2 cx = f2(u.x, u.y), cy = f2(u.z, u.w), cc = f2(w.x, w.y), cs = f2(w.z, w.w);
        x = ffma2(b.P[k], cx, x);
        vx = ffma2(b.Pd[k], cx, vx);
        ax = ffma2(b.Pdd[k], cx, ax);
        c = ffma2(b.P[k], cc, c);
        y = ffma2(b.P[k], cy, y);
        vy = ffma2(b.Pd[k], cy, vy);
        ay = ffma2(b.Pdd[k], cy, ay);
        s = ffma2(b.P[k], cs, s);
    }
    r.x = x;
    r.xd = vx;
    r.xdd = ax;
    r.c = c;
    r.y = y;
    r.yd = vy;
    r.ydd = ay;
    r.s = s;
}

// A basis row pair times trajectory tt's duplicated xi2 in buffer buf.
__device__ __forceinline__ float2 psi_pair(const float *sm, const Smem &S, int buf, int tt, const float2 (&b)[NV])
{
    const float4 *x2 = reinterpret_cast<const float4 *>(sm + S.X2D) + (buf * S.T + tt) * 6;
    float2 s = f2(0.f, 0.f);
#pragma unroll
    for (int k2 = 0; k2 < 6; ++k2) {
        const float4 u = x2[k2];
        s = ffma2(b[2 * k2], f2(u.x, u.y), s);
        if (2 * k2 + 1 < NV) s = ffma2(b[2 * k2 + 1], f2(u.z, u.w), s);
    }
    return s;
}

// Printed alpha = atan2(yt, xt) (alpha_mode = 1) for one step: the offset
// (a d cos, b d sin) - (xt, yt) with d = max(1, rho (a xt^2 + b yt^2) /
// (a^2 xt^2 + b^2 yt^2)), rho = |(xt, yt)|, scaled back by (1/a, 1/b).
__device__ __forceinline__ void literal_offset(float xh, float yh, float a, float b, float ia, float ib,
                                               float &tx, float &ty)
{
    const float xt = a * xh, yt = b * yh;
    const float r2 = fmaf(xt, xt, yt * yt);
    const float u = a * xt, v = b * yt;
    const float den = fmaf(u, u, v * v);
    if (r2 > 0.f) {
        const float ir = rsqrtf(r2);
        const float d = fmaxf(1.f, r2 * ir * fmaf(a, xt * xt, b * yt * yt) / den);
        tx = (d * ir * u - xt) * ia;
        ty = (d * ir * v - yt) * ib;
    } else {
        tx = 1.f;  // alpha = atan2(0, 0) = 0, d = 1: point (a, 0)
        ty = 0.f;
    }
}

// SWEEP: heading at the thread's steps, the closed-form xi3/xi4 steps for
// every (circle, obstacle) pair and the bounds, and the per-step residual
// vectors (g - F xi1 summed per row block).  g is built from r; F xi1 from
// ref when PRO (first step of a solve: g from the initial samples, F xi1 from
// the boundary-consistent reference), else from r as well.  x2buf selects the
// heading coefficients to use.  RES also writes the steps' squared residual
// and cost; FIN the smallest squared ellipse distance.
template <int M, bool LIT, bool RES, bool FIN, bool PRO>
__device__ __forceinline__ void sweep_pair(float *sm, const Smem &S, const ConstLayout &L, const Basis &b,
                                           int x2buf, int tt, int t0, bool v1, Pair &r, const Pair &ref,
                                           Near &nl)
{
    const float2 psi = psi_pair(sm, S, x2buf, tt, b.P);
    float2 psidd = f2(0.f, 0.f);
    if (RES) psidd = psi_pair(sm, S, x2buf, tt, b.Pdd);
    float2 pr;
    pr.x = psi.x - kTwoPi * rintf(psi.x * (1.0f / kTwoPi));
    pr.y = psi.y - kTwoPi * rintf(psi.y * (1.0f / kTwoPi));
    const float2 cp = f2(__cosf(pr.x), __cosf(pr.y)), sp = f2(__sinf(pr.x), __sinf(pr.y));
    const float2 cf = PRO ? ref.c : r.c, sf = PRO ? ref.s : r.s;  // slack values of F xi1

    // velocity and acceleration: project onto the disc of radius v_max / a_max
    const float2 v2 = ffma2(r.xd, r.xd, fmul2(r.yd, r.yd));
    const float2 sv = f2(fminf(1.f, L.v_max * rsqrtf(v2.x)), fminf(1.f, L.v_max * rsqrtf(v2.y)));
    const float2 a2 = ffma2(r.xdd, r.xdd, fmul2(r.ydd, r.ydd));
    const float2 sa = f2(fminf(1.f, L.a_max * rsqrtf(a2.x)), fminf(1.f, L.a_max * rsqrtf(a2.y)));

    float2 X[M], Y[M], ax[M], ay[M], ee[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const float2 ri = dup2(L.r[i]);
        X[i] = ffma2(ri, cp, r.x);
        Y[i] = ffma2(ri, sp, r.y);
        ax[i] = f2(0.f, 0.f);
        ay[i] = f2(0.f, 0.f);
        ee[i] = f2(0.f, 0.f);
    }
    float2 dmin = f2(3.0e38f, 3.0e38f);
    const float *obt = sm + S.cob;
    const int hq = L.qs >> 1;
    const float4 *obs2 = reinterpret_cast<const float4 *>(sm + S.cob + (L.off_obs2 - L.off_obt)) + (t0 >> 1);
    const float4 *obc2 = reinterpret_cast<const float4 *>(sm + S.cob + (L.off_obc2 - L.off_obt));
    const int n = L.n;
    // One (circle, obstacle) pair at both steps.
    auto pair = [&](int j) {
        const float4 o = obs2[j * hq];                          // -x/a at t0, t1; -y/b at t0, t1
        const float4 ci = obc2[2 * j], ca = obc2[2 * j + 1];    // (1/a, 1/a, 1/b, 1/b), (a, a, b, b)
        const float2 ox = f2(o.x, o.y), oy = f2(o.z, o.w);
        const float2 ia = f2(ci.x, ci.y), ib = f2(ci.z, ci.w), aa = f2(ca.x, ca.y), bb = f2(ca.z, ca.w);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float2 xh = ffma2(X[i], ia, ox);  // (x + r_i cos psi - x_j) / a_j
            const float2 yh = ffma2(Y[i], ib, oy);
            const float2 D = ffma2(xh, xh, ffma2(yh, yh, dup2(kTinyD)));
            float2 tx, ty;
            if (!LIT) {
                const float2 h = f2(fmaxf(rsqrtf(D.x), 1.f) - 1.f, fmaxf(rsqrtf(D.y), 1.f) - 1.f);  // max(1, 1/d) - 1
                tx = fmul2(fadd2(xh, dup2(kCoincideT)), h);  // see kCoincideT
                ty = fmul2(yh, h);
            } else {
                literal_offset(xh.x, yh.x, ca.x, ca.z, ci.x, ci.z, tx.x, ty.x);
                literal_offset(xh.y, yh.y, ca.x, ca.z, ci.x, ci.z, tx.y, ty.y);
            }
            if (RES) {
                const float2 ex = fmul2(aa, tx), ey = fmul2(bb, ty);
                ax[i] = fadd2(ax[i], ex);
                ay[i] = fadd2(ay[i], ey);
                ee[i] = ffma2(ex, ex, ffma2(ey, ey, ee[i]));
            } else {
                ax[i] = ffma2(aa, tx, ax[i]);  // e_ij = projected point - (xt, yt)
                ay[i] = ffma2(bb, ty, ay[i]);
            }
            if (FIN) {
                dmin.x = fminf(dmin.x, D.x);
                dmin.y = fminf(dmin.y, D.y);
            }
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
        const float2 mx = fsub2(r.x, nl.rx), my = fsub2(r.y, nl.ry);
        const float2 m2 = ffma2(mx, mx, fmul2(my, my));
        constexpr float lim = kNearMargin * kNearMargin;
        if (__any_sync(act, m2.x > lim || (v1 && m2.y > lim))) {
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                const int j0 = 32 * blk, jn = min(32, n - j0);
                unsigned near = 0u;
                for (int jj = 0; jj < jn; ++jj) {
                    const int j = j0 + jj;
                    const float4 o = obs2[j * hq];
                    const float4 ci = obc2[2 * j];
                    const float2 u0 = ffma2(r.x, f2(ci.x, ci.y), f2(o.x, o.y));
                    const float2 w0 = ffma2(r.y, f2(ci.z, ci.w), f2(o.z, o.w));
                    const float2 d2 = ffma2(u0, u0, fmul2(w0, w0));
                    const float th = obt[j];
                    near |= (d2.x < th || (v1 && d2.y < th) ? 1u : 0u) << jj;
                }
                near = __reduce_or_sync(act, near);
                if (blk == 0) nl.list0 = near;
                else nl.list1 = near;
            }
            nl.rx = r.x;
            nl.ry = r.y;
        }
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
            unsigned near = blk == 0 ? nl.list0 : nl.list1;
            while (near) {
                const int jj = __ffs(near) - 1;
                near &= near - 1u;
                pair(32 * blk + jj);
            }
        }
    } else {
        for (int j = 0; j < n; ++j) pair(j);
    }
    // Obstacle rows: g_ij - (x + r_i c) = r_i (cos psi - c) + e_ij (+ x - x_ref in PRO)
    const float2 fn = dup2(float(n));
    const float2 dxp = PRO ? fsub2(r.x, ref.x) : f2(0.f, 0.f), dyp = PRO ? fsub2(r.y, ref.y) : f2(0.f, 0.f);
    const float2 dcx = fsub2(cp, cf), dsy = fsub2(sp, sf);
    float2 r0x = f2(0.f, 0.f), r1x = r0x, r0y = r0x, r1y = r0x, rob = r0x;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const float2 ri = dup2(L.r[i]);
        const float2 bx = ffma2(fn, ffma2(ri, dcx, dxp), ax[i]);
        const float2 by = ffma2(fn, ffma2(ri, dsy, dyp), ay[i]);
        r0x = fadd2(r0x, bx);
        r0y = fadd2(r0y, by);
        r1x = ffma2(ri, bx, r1x);
        r1y = ffma2(ri, by, r1y);
        if (RES) {
            // sum_j (r_i (c - cos psi) - e_ij)^2, expanded
            const float2 dx = fmul2(ri, dcx), dy = fmul2(ri, dsy);
            const float2 sq = fmul2(fn, ffma2(dx, dx, fmul2(dy, dy)));
            const float2 cr = fmul2(dup2(2.f), ffma2(dx, ax[i], fmul2(dy, ay[i])));
            rob = fadd2(rob, fadd2(fadd2(sq, cr), ee[i]));
        }
    }
    const int qs = L.qs, qp = L.qp;
    if (!AM_BOUND(tt >= 0 && tt < S.T && t0 >= 0 && t0 + 1 < qp && t0 + 1 < qs)) return;
    float *Gx = sm + S.G2 + tt * S.RS + t0;   // side x: row tt
    float *Gy = Gx + S.T * S.RS;              // side y: row T + tt
    const float2 svm = f2(sv.x - 1.f, sv.y - 1.f), sam = f2(sa.x - 1.f, sa.y - 1.f);
    // v and a rows: projected value - F xi1 value
    st2(Gx, PRO ? ffma2(r.xd, svm, fsub2(r.xd, ref.xd)) : fmul2(r.xd, svm), v1);
    st2(Gx + qp, PRO ? ffma2(r.xdd, sam, fsub2(r.xdd, ref.xdd)) : fmul2(r.xdd, sam), v1);
    st2(Gx + 2 * qp, r0x, v1);
    st2(Gx + 3 * qp, fadd2(r1x, dcx), v1);
    st2(Gy, PRO ? ffma2(r.yd, svm, fsub2(r.yd, ref.yd)) : fmul2(r.yd, svm), v1);
    st2(Gy + qp, PRO ? ffma2(r.ydd, sam, fsub2(r.ydd, ref.ydd)) : fmul2(r.ydd, sam), v1);
    st2(Gy + 2 * qp, r0y, v1);
    st2(Gy + 3 * qp, fadd2(r1y, dsy), v1);
    float *GX = sm + S.GX + tt * 4 * qs + t0;
    if (RES) {
        const float2 bnd = ffma2(fmul2(v2, svm), svm, fmul2(fmul2(a2, sam), sam));
        const float2 sl = ffma2(dcx, dcx, fmul2(dsy, dsy));
        st2(GX, fadd2(fadd2(bnd, rob), sl), v1);
        const float2 dp = fsub2(psi, r.psi_t);
        st2(GX + qs, fmul2(dp, dp), v1);
        st2(GX + 2 * qs, ffma2(r.xdd, r.xdd, ffma2(r.ydd, r.ydd, fmul2(psidd, psidd))), v1);
    }
    if (FIN) st2(GX + 3 * qs, dmin, v1);
    r.psi_prev = psi;
    r.psi_cur = psi;
}

template <int M, bool LIT>
__device__ void sweep_dispatch(float *sm, const Smem &S, const ConstLayout &L, const Basis &b, int x2buf,
                               int tt, int t0, bool v1, Pair &r, Near &nl, bool res, bool fin)
{
    if (fin) sweep_pair<M, LIT, true, true, false>(sm, S, L, b, x2buf, tt, t0, v1, r, r, nl);
    else if (res) sweep_pair<M, LIT, true, false, false>(sm, S, L, b, x2buf, tt, t0, v1, r, r, nl);
    else sweep_pair<M, LIT, false, false, false>(sm, S, L, b, x2buf, tt, t0, v1, r, r, nl);
}

// Stage a problem's constant block into shared memory with two bulk async
// copies (the shape sections, then the near thresholds and the paired
// obstacle sections) and zero the rest of the dynamic area (the padding of
// the per-step arrays past q, and the unused rows of the MMA tiles, must read
// as zero).  The wait on the mbarrier is bounded, and the block agrees on its
// outcome before anyone leaves, so no thread is left waiting at a barrier.
__device__ bool stage_constants(const KParams &p, float *sm, const Smem &S, uint64_t *bar,
                                uint32_t parity)
{
    if (threadIdx.x == 0) {
        const ConstLayout &L = p.L;
        const uint32_t b0 = uint32_t(L.off_obs - L.off_fused) * 4u, b1 = uint32_t(L.total - L.off_obt) * 4u;
        // order the block's earlier generic-proxy accesses of this area
        // before the asynchronous copies overwrite it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     :: "r"(smem_u32(bar)), "r"(b0 + b1) : "memory");
        if (!L.diag_stall) {
            bulk_load(sm + S.cst + L.off_fused, p.cblob + L.off_fused, b0, bar);
            if (b1) bulk_load(sm + S.cob, p.cblob + L.off_obt, b1, bar);
        }
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
#ifdef AM_DEBUG_BOUNDS
    if (threadIdx.x == 0) g_oob = 0;
    __syncthreads();
#endif
    for (int i = threadIdx.x; i < Tn * STATE; i += blockDim.x) {
        const int tt = i / STATE, e = i - STATE * tt;
        if (!AM_BOUND(tl.first >= 0 && tl.first + Tn <= p.B && Tn <= p.T)) break;
        const float v = p.state[(size_t)tl.first * STATE + i];
        if (e < 44) put_xi1(sm, S, 1, tt, (e / NV) * 12 + e % NV, v);
        else if (e < 55) put_xi2(sm, S, 1, tt, e - 44, v);
        else if (e < 99) sm[S.lam + tt * 48 + ((e - 55) / NV) * 12 + (e - 55) % NV] = v;
        else sm[S.lps + tt * 12 + (e - 99)] = v;
    }
    for (int i = threadIdx.x; i < kRParts * p.T * 48; i += blockDim.x) sm[S.rb + i] = 0.f;
    __syncthreads();
    // Reference xi1, xi2 into buffer 0: boundary control points from the
    // boundary conditions on every block that has boundary rows, the rest as given.
    for (int i = threadIdx.x; i < Tn * 55; i += blockDim.x) {
        const int tt = i / 55, e = i - 55 * tt, blk = e / NV, k = e - NV * blk;
        const bool has_bc = (blk == 0 || blk == 2 || blk == 4 || L.cs_boundary);
        float v = blk < 4 ? sm[S.xi1 + (p.T + tt) * 48 + blk * 12 + k] : sm[S.xi2 + (p.T + tt) * 12 + k];
        if (has_bc && k <= 2) v = sm[S.cst + L.off_ends + blk * 8 + k];
        if (has_bc && k >= 8) v = sm[S.cst + L.off_ends + blk * 8 + (k - 5)];
        if (blk < 4) put_xi1(sm, S, 0, tt, blk * 12 + k, v);
        else put_xi2(sm, S, 0, tt, k, v);
    }
    __syncthreads();

    // Stepper threads: trajectory tt, steps t0 and t0 + 1.
    const int tpt = pair_threads(L.q), np = (L.q + 1) >> 1;
    const int tt = int(threadIdx.x) / tpt, jp = int(threadIdx.x) - tt * tpt;
    const bool stepper = tt < Tn && jp < np;
    const int t0 = 2 * jp;
    const bool v1 = stepper && t0 + 1 < L.q;
    Basis b;
    Pair r;
    Near nl;
    int cur = 0, cur2 = 0;

    // Step 1 of Sec. III-D: xi3, xi4 and g from the initial samples, the
    // residual against the reference.
    if (stepper) {
        load_basis(sm, S, L, t0, v1, b);
        nl.rx = nl.ry = f2(3.0e18f, 3.0e18f);  // no near list yet: every warp forms one
        nl.list0 = nl.list1 = 0u;
        Pair ref;
        eval_pair(sm, S, 1, tt, b, r);
        eval_pair(sm, S, 0, tt, b, ref);
        r.psi_t = f2(0.f, 0.f);
        sweep_pair<M, LIT, false, false, true>(sm, S, L, b, 1, tt, t0, v1, r, ref, nl);
        r.psi_cur = psi_pair(sm, S, 0, tt, b.P);  // heading of the reference c_psi
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
            eval_pair(sm, S, cur, tt, b, r);
            // psi_t = psi + wrap(atan2(s, c) - psi), psi the previous heading;
            // the heading step works on delta = psi_t - P xi2
            r.psi_t.x = r.psi_prev.x + wrap_pi(atan2_heading(r.s.x, r.c.x) - r.psi_prev.x);
            r.psi_t.y = r.psi_prev.y + wrap_pi(atan2_heading(r.s.y, r.c.y) - r.psi_prev.y);
            const float2 dl = fsub2(r.psi_t, r.psi_cur);
            const float2 dd = f2(dl.x, v1 ? dl.y : 0.f);
            // this pair's share of P^T delta (the second step's basis row is zero past q)
            float pk[12];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const float2 m = fmul2(b.P[k], dd);
                pk[k] = m.x + m.y;
            }
            pk[11] = 0.f;
            if (AM_BOUND(tt < S.T && jp < np)) {
                float4 *dst = reinterpret_cast<float4 *>(sm + S.PTD + (tt * np + jp) * 12);
                dst[0] = make_float4(pk[0], pk[1], pk[2], pk[3]);
                dst[1] = make_float4(pk[4], pk[5], pk[6], pk[7]);
                dst[2] = make_float4(pk[8], pk[9], pk[10], pk[11]);
            }
        }
        __syncthreads();
        phase_psi(p, sm, S, tl, cur2);
        __syncthreads();
        if (stepper) sweep_dispatch<M, LIT>(sm, S, L, b, cur2 ^ 1, tt, t0, v1, r, nl, res, k == p.iters - 1);
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
        if (!AM_BOUND(tl.first >= 0 && tl.first + Tn <= p.B && Tn <= p.T)) break;
        float v;
        if (e < 44) v = sm[S.xi1 + (cur * p.T + tq) * 48 + (e / NV) * 12 + e % NV];
        else if (e < 55) v = sm[S.xi2 + (cur2 * p.T + tq) * 12 + (e - 44)];
        else if (e < 99) v = sm[S.lam + (cur * p.T + tq) * 48 + ((e - 55) / NV) * 12 + (e - 55) % NV];
        else v = sm[S.lps + tq * 12 + (e - 99)];
        p.state[(size_t)tl.first * STATE + i] = v;
    }
    __syncthreads();
#ifdef AM_DEBUG_BOUNDS
    if (threadIdx.x == 0 && g_oob) atomicOr(p.err, 2);
#endif
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
// variant (precision form PR, circle count M, alpha form LIT) so that each is
// compiled on its own (the variants inlined into one kernel spill registers).
// PR selects the DOT phase's tensor-core products as in the single-problem
// kernel, so a problem gives the same bits alone and in a group.  The variant
// kernels of one solve run concurrently; CTAs take work items (problem,
// tile) of their variant from a list in order, through one atomic counter
// per variant, and re-stage constants whenever they move to another problem.
// The lists, their lengths and offsets live in device memory, so a captured
// launch stays valid when the set of problems it advances changes.
//   head[v]: number of items of variant v; head[kGroupVariants + v]: offset of its list
//   ctl[2 v]: its work counter (zeroed before the launch); ctl[2 v + 1]: status
template <int M, bool LIT, int PR>
__global__ void __launch_bounds__(kMaxThreads, 1)
am_group_kernel(const KParams *probs, const int *items, const int *head, int *ctl)
{
    constexpr int v = PR * 8 + M * 2 + (LIT ? 1 : 0) - 2;
    int *counter = ctl + 2 * v;
    const int nitems = head[v];
    const int *list = items + 2 * head[kGroupVariants + v];
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
        run_tile<M, LIT, PR>(kp, sm, smem_layout(kp.L, kp.T), tile_of(item.y, kp.B, kp.ntiles));
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
    int tmax = kMaxThreads / pair_threads(L.q);
    if (tmax > kMaxTile) tmax = kMaxTile;
    while (tmax > 1 && fused_smem_bytes(L, tmax) > kFusedSmemMax) --tmax;
    return tmax < 1 ? 1 : tmax;
}

int fused_max_threads() { return kMaxThreads; }

int group_tile(const ConstLayout &L, int threads)
{
    int t = threads / pair_threads(L.q);
    if (t > kMaxTile) t = kMaxTile;
    while (t >= 1 && fused_smem_bytes(L, t) > kGroupSmemMax) --t;
    return t < 1 ? 0 : t;
}

int launch_group(const GroupLaunch &g, void *stream, int *launches, const char **why)
{
    if (g.variant >= kGroupWarpVariant0) return launch_group_warp(g, stream, launches, why);
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
#define AM_GCASE(MM, LL, PP)                                                                    \
    case PP * 8 + MM * 2 + LL - 2:                                                              \
        e = cudaError_t(raise_smem_limit(reinterpret_cast<const void *>(am_group_kernel<MM, LL, PP>), g.smem)); \
        if (e != cudaSuccess) {                                                                 \
            *why = cudaGetErrorString(e);                                                       \
            return -2;                                                                          \
        }                                                                                       \
        am_group_kernel<MM, LL, PP><<<g.grid, g.threads, g.smem, st>>>(g.d_probs, g.d_items,    \
                                                                       g.d_head, g.d_ctl);      \
        break;
#define AM_GCASES(PP)                                                                           \
        AM_GCASE(1, 0, PP)                                                                      \
        AM_GCASE(1, 1, PP)                                                                      \
        AM_GCASE(2, 0, PP)                                                                      \
        AM_GCASE(2, 1, PP)                                                                      \
        AM_GCASE(3, 0, PP)                                                                      \
        AM_GCASE(3, 1, PP)                                                                      \
        AM_GCASE(4, 0, PP)                                                                      \
        AM_GCASE(4, 1, PP)
        AM_GCASES(0)
        AM_GCASES(1)
        AM_GCASES(2)
        AM_GCASES(3)
#undef AM_GCASES
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

int group_variant(const ConstLayout &L) { return L.precision * 8 + L.m * 2 + (L.alpha_mode ? 1 : 0) - 2; }

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
                                     int(kFusedSmemMax)) != cudaSuccess)
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
    const int tq = T * pair_threads(L.q);
    if (tq > kMaxThreads || T < 1 || T > kMaxTile) return -1;
    const size_t smem = fused_smem_bytes(L, T);
    if (smem > kFusedSmemMax) return -1;
    // twelve warps whatever the tile: the tensor-core phases run all their tasks at once
    const int threads = kMaxThreads;
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
        AM_CASES(3)
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
