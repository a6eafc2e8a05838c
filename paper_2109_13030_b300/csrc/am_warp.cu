// Warp-pair-per-trajectory kernel of the batched alternating-minimization
// loop (Sec. III-D, steps 1-5; the batch solution of Sec. III-E), for batches
// of a few trajectories per SM, such as the paper's B = 1000.
//
// At such batch sizes an SM holds about seven trajectories.  A kernel that
// advances them together through the phases of an iteration (position step,
// trajectory values, heading step, sweep, contraction) waits at a block
// barrier after every phase for its slowest warp.  Here each trajectory
// belongs to two warps (its "halves") for all its iterations, and the halves
// of different trajectories never wait for one another: after the constants
// are staged, a pair of warps runs its trajectory's whole loop, synchronising
// only with each other (a 64-thread named barrier), writes the state back and
// takes the next trajectory.  Different trajectories sit in different phases
// at any moment, so the scheduler fills one warp's dependency stalls with
// another's work.
//
// Lane l of half h owns the pair of consecutive steps j = h nh + l (steps 2j
// and 2j + 1), with nh = ceil(np / 2) pairs per half, np = ceil(q / 2) and
// q <= 128.  It keeps the basis row P of its two steps in registers for the
// life of the kernel, reads Pd and Pdd from a copy in shared memory laid out
// per pair of steps, and evaluates both steps with paired FP32 instructions.
// The steps' contributions to the two contractions over time -- R = F^T (g -
// F xi1) for the position step and P^T delta for the heading step -- are
// formed per lane and summed over the 64 lanes through a transpose in shared
// memory: lane l of half h stores its partial of output o at red[o][32 h + l],
// and after the pair's barrier the lane that owns output o sums row o with
// 128-bit loads.  Half h owns the position-step outputs of side h (x or y),
// which need only that side's u and xi1, so the position step needs no
// barrier between the halves until its result is complete.
//
// The arithmetic is that of the small-tile fused kernel: the position step
// in the increment form xi1' = xi1 + Minv (lam + coef R) - MQ xi1, the
// multiplier update lam' = lam + rho R (Eq. update_lambda_1), the heading
// step xi2' = xi2 + Mpsi (lam_psi + rho P^T delta) - Mpsi H xi2 and the
// lambda_psi update of Eq. update_lambda_psi, the trig-free closed form of
// the alpha/d steps (Eq. zeta_2 - compute_da) with a list of near obstacles
// per warp, and the sums of the last sweep (residuals, cost) in FP64.  The
// contraction R is FP32 SIMT here (the FP32 precision form).  A solve starts
// from the reference whose boundary control points come from the boundary
// conditions, exactly as in that kernel.
//
// Per iteration of one trajectory (B = the pair's barrier, w = a warp's own):
//   XI1   owner lanes: R from its row, lam' and u; u to shared memory  w
//         xi1' = xi1 + Minv u - MQ xi1 for the half's side  B
//   EVAL  x ... s at the lane's steps; heading target psi_t and delta;
//         the lane's partial of P^T delta to the transpose rows  B
//   PSI   half 0, lanes 0..10: P^T delta, lam_psi + rho P^T delta  w
//         xi2' = xi2 + Mpsi (.) - Mpsi H xi2  B
//   SWEEP psi = P xi2', the closed-form steps, the residual rows (registers)
//   DOT   the lane's partial of R to the transpose rows  B
//
// The kernel covers the default alpha form and the FP32 precision form,
// 1..4 circles, up to 64 obstacles and q <= 128; history is supported.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "am_async.cuh"
#include "am_heading.cuh"
#include "am_internal.h"

namespace trajam {
namespace {

constexpr int kWMaxQ = 256;       // 128 pairs: one per lane of four warps
constexpr int kWMaxWarps = 16;    // warps per CTA (128 registers each: four per scheduler)
// Floats per pair of steps in the pair-interleaved copy of Pd, Pdd: 11
// float2 entries (B(t, k), B(t + 1, k)) and padding; 28 = 4 x 7, so the
// 128-bit loads of eight neighbouring pairs fall on distinct banks.  Pair
// 32 NW is all zero: lanes without a pair read it.
constexpr int kPB = 28;
// Row stride of the Minv and MQ rows (24 padded columns): 28, for the same
// reason, so the owner lanes' 128-bit row loads do not share banks.
constexpr int kMR = 28;

// Per-trajectory shared-memory area (float offsets from the trajectory's
// base); NW warps per trajectory, C = 32 NW lane columns.
constexpr int kWxd = 0;       // [2][12][8] xi1 duplicated per coefficient k:
                              //            (cx, cx, cy, cy, cc, cc, cs, cs), both buffers
constexpr int kWx2d = 192;    // [2][12][2] xi2 duplicated, both buffers
constexpr int kWxi = 240;     // [2][48]    xi1, blocks of 12 (c_x, c_c | c_y, c_s), both buffers
constexpr int kWx2 = 336;     // [2][12]    xi2, both buffers
constexpr int kWu = 360;      // [48]       lam + coef R, the position step's input
constexpr int kWv = 408;      // [12]       lam_psi + rho P^T delta, the heading step's input
constexpr int kWdx2 = 420;    // [12]       the last increment of xi2
constexpr int kWsum = 432;    // [NW][4] double: per warp, the sums of the last sweep (res, res_psi, cost, dmin)
constexpr int kWsdx2 = 464;   // [12]       the sum of the heading increments over the iterations
constexpr int kWacc = 480;    // [4][C] float4: per lane, its residual rows summed over the iterations
// then  eb  [5][C] float4: per lane, the boundary control points' share of its
//                          values (x, xd | xdd, c | y, yd | ydd, s | psi, psidd)
//       red [44][C + 4]    transpose rows of the reductions over the steps
//                          (the stride is 4 mod 32 banks)
template <int NW>
struct WS {
    static constexpr int kThreads = 32 * NW;              // threads per trajectory
    static constexpr int kCols = 32 * NW;                 // lane columns of the transpose rows
    static constexpr int kRS = kCols + 4;                 // their row stride
    static constexpr int kMaxTraj = kWMaxWarps / NW;      // trajectories in flight per CTA
    static constexpr int kPairs = 32 * NW + 1;            // pairs of the Pd, Pdd copy, the last all zero
    static constexpr int kEb = kWacc + 16 * kCols;
    static constexpr int kRed = kEb + 20 * kCols;
    static constexpr int kTrajFloats = kRed + 44 * kRS;
};

// Warps per trajectory for a horizon of q steps: one pair of steps per lane.
__host__ __device__ constexpr int warps_for_q(int q) { return q <= 128 ? 2 : q <= 192 ? 3 : 4; }

// Interior control points.  Every polynomial block has boundary rows (the
// slack blocks too, with cs_boundary): they fix control points 0, 1, 2 and
// 8, 9, 10, so the null space of the constraint rows is spanned by points
// 3..7, and the KKT inverse blocks Minv = N (N^T Qbar N)^-1 N^T and Mpsi
// vanish on the other rows and columns.  The position and heading steps
// therefore move only the interior points and read only the interior
// components of R and P^T delta: 20 of R's 44 components (state order o' =
// 5 blk + k - 3) and 5 of P^T delta's 11 are formed per iteration.  The
// multipliers' boundary components change no trajectory; the state keeps
// them exact through the linearity of their updates (the residual rows and
// delta are summed over the iterations and contracted once at the end).
constexpr int kI0 = 3;        // first interior control point
constexpr int kNI = 5;        // interior control points per block
__device__ __forceinline__ bool interior(int k) { return k >= kI0 && k < kI0 + kNI; }

// Debug build (-DAM_DEBUG_BOUNDS): a failed index check sets the block's
// flag and skips the access; the flag becomes bit 2 of the status word.
#ifdef AM_DEBUG_BOUNDS
__shared__ int g_woob;
#define AM_WBOUND(cond) ((cond) ? true : (g_woob = 1, false))
#else
#define AM_WBOUND(cond) true
#endif

// CTA shared-memory layout (float offsets).
//   bar    the staging mbarrier (16 bytes)
//   cst    region [off_mt, off_obs) of the constant block (Minv^T, (MQ)^T,
//          boundary control points, Mpsi^T, (Mpsi H)^T, P^T P), placed so
//          that sm + cst + off_x addresses section x
//   cob    region [off_obt, total) (near thresholds, paired obstacle sections)
//   mir    [22][kMR] Minv by rows, columns in blocks of 12 per polynomial
//   mqr    [22][kMR] MQ by rows, the same columns
//   mpr    [11][12] Mpsi by rows;  mhr [11][12] Mpsi H by rows;  ptr [11][12] P^T P by rows
//   pb     [2][32 NW + 1][kPB] Pd, Pdd per pair of steps j: (B(2j, k), B(2j + 1, k))
//          for k = 0..10, zero past the horizon
//   traj   T x WS<NW>::kTrajFloats
struct WSmem {
    int bar, cst, cob, mir, mqr, mpr, mhr, ptr, pb, traj, total;
};

template <int NW>
__host__ __device__ inline WSmem wsmem_layout(const ConstLayout &L, int T)
{
    WSmem s;
    int o = 0;
    s.bar = o; o += 4;
    s.cst = o - L.off_mt; o += L.off_obs - L.off_mt;
    s.cob = o; o += L.total - L.off_obt;
    o = (o + 3) & ~3;
    s.mir = o; o += NS * kMR;
    s.mqr = o; o += NS * kMR;
    s.mpr = o; o += NV * 12;
    s.mhr = o; o += NV * 12;
    s.ptr = o; o += NV * 12;
    s.pb = o; o += 2 * WS<NW>::kPairs * kPB;
    s.traj = o; o += T * WS<NW>::kTrajFloats;
    s.total = o;
    return s;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// The NW warps of a trajectory meet: named barrier id (1..8) of 32 NW threads.
template <int NW>
__device__ __forceinline__ void pair_sync(int id)
{
    __syncwarp();
    asm volatile("bar.sync %0, %1;\n" :: "r"(id), "r"(WS<NW>::kThreads) : "memory");
}

// Padded index (blocks of 12) of state entry o = blk * 11 + k of xi1 or lam.
__device__ __forceinline__ int pidx(int o) { return o + o / NV; }

// Position of polynomial block blk (0 c_x, 1 c_c, 2 c_y, 3 c_s) within a
// duplicated xi1 entry (cx, cx, cy, cy, cc, cc, cs, cs).
__device__ __forceinline__ int dpos(int blk) { return blk == 0 ? 0 : blk == 2 ? 1 : blk == 1 ? 2 : 3; }

// Writes entry p (padded index blk * 12 + k) of xi1 into buffer buf, and its duplicate.
__device__ __forceinline__ void put_xi1(float *ta, int buf, int p, float v)
{
    if (!AM_WBOUND(buf >= 0 && buf < 2 && p >= 0 && p < 48)) return;
    ta[kWxi + buf * 48 + p] = v;
    const int blk = p / 12, k = p - 12 * blk;
    reinterpret_cast<float2 *>(ta + kWxd)[(buf * 12 + k) * 4 + dpos(blk)] = make_float2(v, v);
}

__device__ __forceinline__ void put_xi2(float *ta, int buf, int k, float v)
{
    if (!AM_WBOUND(buf >= 0 && buf < 2 && k >= 0 && k < 12)) return;
    ta[kWx2 + buf * 12 + k] = v;
    reinterpret_cast<float2 *>(ta + kWx2d)[buf * 12 + k] = make_float2(v, v);
}

// Basis row P of the lane's pair of steps (Eq. param), kept in registers; the
// rows Pd, Pdd are read from the pair-interleaved copy in shared memory (pd,
// pdd: float4 pointers to the pair's (B(t, k), B(t + 1, k), B(t, k + 1), B(t +
// 1, k + 1)) entries).
struct WBasis {
    float2 P[NV];
    const float4 *pd, *pdd;
};

// Trajectory values of one pair of steps.
struct WVals {
    float2 x, xd, xdd, y, yd, ydd, c, s;
};

// Residual rows g - F xi1 of one pair of steps, per side: velocity,
// acceleration, the circles' position rows summed (r0) and weighted by the
// circle offsets plus the slack row (r1).
struct WRes {
    float2 vx, ax, r0x, r1x, vy, ay, r0y, r1y;
};

// Per pair of steps: heading target, the heading the unwrap refers to and
// the current P xi2; the warp's near-obstacle list (the same in every lane)
// and the robot centres it was formed at.
struct WSlot {
    float2 psi_t, psi_prev, psi_cur;
    float2 nrx, nry;
    unsigned near0, near1;
};

// rows: [3][q][12] P, Pd, Pdd in global memory (P read once per warp); pb:
// the shared-memory copy of Pd, Pdd per pair (jb: the lane's pair, or the
// zero pair 64 for a lane without one).
template <int NW>
__device__ __forceinline__ void load_basis(const float *rows, const float *pb, int jb, bool valid, bool v1,
                                           WBasis &b)
{
    const int t0 = 2 * jb, t1 = v1 ? t0 + 1 : t0;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        b.P[k] = valid ? f2(__ldg(rows + t0 * 12 + k), v1 ? __ldg(rows + t1 * 12 + k) : 0.f) : f2(0.f, 0.f);
    b.pd = reinterpret_cast<const float4 *>(pb + jb * kPB);
    b.pdd = reinterpret_cast<const float4 *>(pb + (WS<NW>::kPairs + jb) * kPB);
}

// Pd or Pdd entry k of a pair from its float4 copy (two k per float4).
__device__ __forceinline__ float2 brow(const float4 &v, int k) { return (k & 1) ? f2(v.z, v.w) : f2(v.x, v.y); }

// x, xdot, ..., c, s at the pair of steps from the duplicated xi1 (Eq. param).
__device__ __forceinline__ void eval_pair(const float4 *xd, const WBasis &b, WVals &r)
{
    const float2 z = f2(0.f, 0.f);
    r = WVals{z, z, z, z, z, z, z, z};
    float4 d, e;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if ((k & 1) == 0) {
            d = b.pd[k >> 1];
            e = b.pdd[k >> 1];
        }
        const float4 u = xd[2 * k], w = xd[2 * k + 1];  // (cx, cx, cy, cy), (cc, cc, cs, cs)
        const float2 cx = f2(u.x, u.y), cy = f2(u.z, u.w), cc = f2(w.x, w.y), cs = f2(w.z, w.w);
        const float2 pd = brow(d, k), pdd = brow(e, k);
        r.x = ffma2(b.P[k], cx, r.x);
        r.xd = ffma2(pd, cx, r.xd);
        r.xdd = ffma2(pdd, cx, r.xdd);
        r.c = ffma2(b.P[k], cc, r.c);
        r.y = ffma2(b.P[k], cy, r.y);
        r.yd = ffma2(pd, cy, r.yd);
        r.ydd = ffma2(pdd, cy, r.ydd);
        r.s = ffma2(b.P[k], cs, r.s);
    }
}

// Heading (and with DD its second derivative) at the pair from the duplicated xi2.
template <bool DD>
__device__ __forceinline__ void heading_pair(const float4 *x2, const WBasis &b, float2 &p, float2 &dd)
{
    p = dd = f2(0.f, 0.f);
#pragma unroll
    for (int k2 = 0; k2 < 6; ++k2) {
        const float4 u = x2[k2];
        const float2 ca = f2(u.x, u.y), cb = f2(u.z, u.w);
        p = ffma2(b.P[2 * k2], ca, p);
        if (2 * k2 + 1 < NV) p = ffma2(b.P[2 * k2 + 1], cb, p);
        if (DD) {
            const float4 w = b.pdd[k2];
            dd = ffma2(f2(w.x, w.y), ca, dd);
            if (2 * k2 + 1 < NV) dd = ffma2(f2(w.z, w.w), cb, dd);
        }
    }
}

// The boundary control points' share of the trajectory values and of the
// heading (and its second derivative) at the pair: constant over the
// iterations, since those points never move.  Formed once per trajectory
// from the reference (buffer 0) into the lane's slots of eb.
template <int NW>
__device__ __forceinline__ void eval_boundary(const float4 *xd, const float4 *x2, const WBasis &b, float4 *eb)
{
    constexpr int C = WS<NW>::kCols;
    const float2 z = f2(0.f, 0.f);
    WVals r{z, z, z, z, z, z, z, z};
    float2 ps = z, pdd = z;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (interior(k)) continue;
        const float2 pd = brow(b.pd[k >> 1], k), pe = brow(b.pdd[k >> 1], k);
        const float4 u = xd[2 * k], w = xd[2 * k + 1];
        const float2 cx = f2(u.x, u.y), cy = f2(u.z, u.w), cc = f2(w.x, w.y), cs = f2(w.z, w.w);
        r.x = ffma2(b.P[k], cx, r.x);
        r.xd = ffma2(pd, cx, r.xd);
        r.xdd = ffma2(pe, cx, r.xdd);
        r.c = ffma2(b.P[k], cc, r.c);
        r.y = ffma2(b.P[k], cy, r.y);
        r.yd = ffma2(pd, cy, r.yd);
        r.ydd = ffma2(pe, cy, r.ydd);
        r.s = ffma2(b.P[k], cs, r.s);
        const float4 v = x2[k >> 1];
        const float2 c2 = (k & 1) ? f2(v.z, v.w) : f2(v.x, v.y);
        ps = ffma2(b.P[k], c2, ps);
        pdd = ffma2(pe, c2, pdd);
    }
    eb[0] = make_float4(r.x.x, r.x.y, r.xd.x, r.xd.y);
    eb[C] = make_float4(r.xdd.x, r.xdd.y, r.c.x, r.c.y);
    eb[2 * C] = make_float4(r.y.x, r.y.y, r.yd.x, r.yd.y);
    eb[3 * C] = make_float4(r.ydd.x, r.ydd.y, r.s.x, r.s.y);
    eb[4 * C] = make_float4(ps.x, ps.y, pdd.x, pdd.y);
}

// Trajectory values at the pair: the boundary share plus the interior
// control points 3..7 of the duplicated xi1.
template <int NW>
__device__ __forceinline__ void eval_interior(const float4 *xd, const WBasis &b, const float4 *eb, WVals &r)
{
    constexpr int C = WS<NW>::kCols;
    const float4 e0 = eb[0], e1 = eb[C], e2 = eb[2 * C], e3 = eb[3 * C];
    r = WVals{f2(e0.x, e0.y), f2(e0.z, e0.w), f2(e1.x, e1.y), f2(e2.x, e2.y),
              f2(e2.z, e2.w), f2(e3.x, e3.y), f2(e1.z, e1.w), f2(e3.z, e3.w)};
    float4 d, e;
#pragma unroll
    for (int k = kI0; k < kI0 + kNI; ++k) {
        if (k == kI0 || (k & 1) == 0) {
            d = b.pd[k >> 1];
            e = b.pdd[k >> 1];
        }
        const float4 u = xd[2 * k], w = xd[2 * k + 1];
        const float2 cx = f2(u.x, u.y), cy = f2(u.z, u.w), cc = f2(w.x, w.y), cs = f2(w.z, w.w);
        const float2 pd = brow(d, k), pdd = brow(e, k);
        r.x = ffma2(b.P[k], cx, r.x);
        r.xd = ffma2(pd, cx, r.xd);
        r.xdd = ffma2(pdd, cx, r.xdd);
        r.c = ffma2(b.P[k], cc, r.c);
        r.y = ffma2(b.P[k], cy, r.y);
        r.yd = ffma2(pd, cy, r.yd);
        r.ydd = ffma2(pdd, cy, r.ydd);
        r.s = ffma2(b.P[k], cs, r.s);
    }
}

// Heading (and with DD its second derivative) at the pair: the boundary
// share plus the interior control points of the duplicated xi2.
template <int NW, bool DD>
__device__ __forceinline__ void heading_interior(const float4 *x2, const WBasis &b, const float4 *eb, float2 &p,
                                                 float2 &dd)
{
    const float4 e4 = eb[4 * WS<NW>::kCols];
    p = f2(e4.x, e4.y);
    dd = f2(e4.z, e4.w);
    float4 v, w;
#pragma unroll
    for (int k = kI0; k < kI0 + kNI; ++k) {
        if (k == kI0 || (k & 1) == 0) {
            v = x2[k >> 1];
            if (DD) w = b.pdd[k >> 1];
        }
        const float2 c2 = brow(v, k);
        p = ffma2(b.P[k], c2, p);
        if (DD) dd = ffma2(brow(w, k), c2, dd);
    }
}

// Per-step sums of the last sweep: squared residual, squared heading
// residual, cost, smallest squared ellipse distance (both steps of a pair).
struct WSums {
    float2 res, rpsi, cost, dmin;
};

// SWEEP of the lane's pair of steps: the closed-form alpha/d steps of every
// (circle, obstacle) pair in the trig-free form and the velocity and
// acceleration projections, giving the residual rows.  PRO: first step of a
// solve (g from the initial samples r, F xi1 from the boundary-consistent
// reference ref).  RES: the per-step sums; FIN: also the smallest distance,
// every obstacle visited.  A lane without a pair takes part in the warp's
// votes with no vote of its own; its basis rows are zero, so its residual
// rows are zero.
template <int M, bool RES, bool FIN, bool PRO>
__device__ __forceinline__ void sweep_pair(const float *cob, const ConstLayout &L, float2 psi, float2 psidd,
                                           int jp, bool valid, bool v1, const WVals &r, const WVals &ref,
                                           WSlot &st, WRes &o, WSums &sums)
{
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
    const float *obt = cob;
    const int hq = L.qs >> 1;
    const float4 *obs2 = reinterpret_cast<const float4 *>(cob + (L.off_obs2 - L.off_obt)) + jp;
    const float4 *obc2 = reinterpret_cast<const float4 *>(cob + (L.off_obc2 - L.off_obt));
    const int n = L.n;
    auto pair = [&](int j) {
        const float4 ob = obs2[j * hq];                        // -x/a at t0, t1; -y/b at t0, t1
        const float4 ci = obc2[2 * j], ca = obc2[2 * j + 1];   // (1/a, 1/a, 1/b, 1/b), (a, a, b, b)
        const float2 ox = f2(ob.x, ob.y), oy = f2(ob.z, ob.w);
        const float2 ia = f2(ci.x, ci.y), ib = f2(ci.z, ci.w), aa = f2(ca.x, ca.y), bb = f2(ca.z, ca.w);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float2 xh = ffma2(X[i], ia, ox);  // (x + r_i cos psi - x_j) / a_j
            const float2 yh = ffma2(Y[i], ib, oy);
            const float2 D = ffma2(xh, xh, ffma2(yh, yh, dup2(kTinyD)));
            const float2 h = f2(fmaxf(rsqrtf(D.x), 1.f) - 1.f, fmaxf(rsqrtf(D.y), 1.f) - 1.f);  // max(1, 1/d) - 1
            const float2 tx = fmul2(fadd2(xh, dup2(kCoincideT)), h), ty = fmul2(yh, h);  // see kCoincideT
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
    if (!FIN) {
        // The row correction of a circle outside the ellipse is exactly zero
        // (max(1, 1/d) - 1 = 0), and every circle lies within r_max max(1/a,
        // 1/b) of the robot centre in the ellipse-scaled frame, so obstacle j
        // matters only when the centre is near it.  The list of obstacles
        // near any step of the warp (formed with a threshold widened by
        // kNearMargin) is formed again only when one of its centres has
        // moved farther than the margin since.
        const float2 mx = fsub2(r.x, st.nrx), my = fsub2(r.y, st.nry);
        const float2 m2 = ffma2(mx, mx, fmul2(my, my));
        constexpr float lim = kNearMargin * kNearMargin;
        if (__any_sync(0xffffffffu, valid && (m2.x > lim || (v1 && m2.y > lim)))) {
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                const int j0 = 32 * blk, jn = min(32, n - j0);
                unsigned near = 0u;
                for (int jj = 0; jj < jn; ++jj) {
                    const int j = j0 + jj;
                    const float4 ob = obs2[j * hq];
                    const float4 ci = obc2[2 * j];
                    const float2 u0 = ffma2(r.x, f2(ci.x, ci.y), f2(ob.x, ob.y));
                    const float2 w0 = ffma2(r.y, f2(ci.z, ci.w), f2(ob.z, ob.w));
                    const float2 d2 = ffma2(u0, u0, fmul2(w0, w0));
                    const float th = obt[j];
                    near |= (valid && (d2.x < th || (v1 && d2.y < th)) ? 1u : 0u) << jj;
                }
                near = __reduce_or_sync(0xffffffffu, near);
                if (blk == 0) st.near0 = near;
                else st.near1 = near;
            }
            st.nrx = r.x;
            st.nry = r.y;
        }
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
            unsigned near = blk == 0 ? st.near0 : st.near1;
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
    const float2 svm = f2(sv.x - 1.f, sv.y - 1.f), sam = f2(sa.x - 1.f, sa.y - 1.f);
    // v and a rows: projected value - F xi1 value
    o.vx = PRO ? ffma2(r.xd, svm, fsub2(r.xd, ref.xd)) : fmul2(r.xd, svm);
    o.ax = PRO ? ffma2(r.xdd, sam, fsub2(r.xdd, ref.xdd)) : fmul2(r.xdd, sam);
    o.r0x = r0x;
    o.r1x = fadd2(r1x, dcx);
    o.vy = PRO ? ffma2(r.yd, svm, fsub2(r.yd, ref.yd)) : fmul2(r.yd, svm);
    o.ay = PRO ? ffma2(r.ydd, sam, fsub2(r.ydd, ref.ydd)) : fmul2(r.ydd, sam);
    o.r0y = r0y;
    o.r1y = fadd2(r1y, dsy);
    if (RES) {
        const float2 bnd = ffma2(fmul2(v2, svm), svm, fmul2(fmul2(a2, sam), sam));
        const float2 sl = ffma2(dcx, dcx, fmul2(dsy, dsy));
        const float2 dp = fsub2(psi, st.psi_t);
        const float2 e0 = fadd2(fadd2(bnd, rob), sl), e1 = fmul2(dp, dp);
        const float2 e2 = ffma2(r.xdd, r.xdd, ffma2(r.ydd, r.ydd, fmul2(psidd, psidd)));
        sums.res = f2(valid ? e0.x : 0.f, v1 ? e0.y : 0.f);
        sums.rpsi = f2(valid ? e1.x : 0.f, v1 ? e1.y : 0.f);
        sums.cost = f2(valid ? e2.x : 0.f, v1 ? e2.y : 0.f);
    }
    if (FIN) sums.dmin = f2(valid ? dmin.x : 3.0e38f, v1 ? dmin.y : 3.0e38f);
    st.psi_prev = psi;
    st.psi_cur = psi;
}

// Sum over the warp of a double held per lane (every lane gets the sum).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum of transpose row o (the 64 lane partials) in a fixed order.
// Sum of F float4s of partials of transpose row o (row stride rs) from
// column c0 (a multiple of 4), in a fixed order: two running sums over the
// float4s, or for F = 4 a tree.
template <int F>
__device__ __forceinline__ float row_part(const float *red, int o, int c0, int rs)
{
    const float4 *r = reinterpret_cast<const float4 *>(red + o * rs + c0);
    if constexpr (F == 4) {
        const float4 a = r[0], b = r[1], c = r[2], d = r[3];
        return (((a.x + b.x) + (c.x + d.x)) + ((a.y + b.y) + (c.y + d.y))) +
               (((a.z + b.z) + (c.z + d.z)) + ((a.w + b.w) + (c.w + d.w)));
    } else {
        float4 a = r[0], b = r[1];
#pragma unroll
        for (int i = 2; i < F; i += 2) {
            const float4 v = r[i];
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
            a.w += v.w;
            if (i + 1 < F) {
                const float4 w = r[i + 1];
                b.x += w.x;
                b.y += w.y;
                b.z += w.z;
                b.w += w.w;
            }
        }
        return ((a.x + b.x) + (a.y + b.y)) + ((a.z + b.z) + (a.w + b.w));
    }
}

// Sum of the 32 NW partials of transpose row o.
template <int NW>
__device__ __forceinline__ float row_sum(const float *red, int o)
{
    return row_part<8 * NW>(red, o, 0, WS<NW>::kRS);
}

// R for the owner lanes 0..9 of warps 0 and 1 (side x, side y): each row
// is summed by lanes l and l + 16 (the two halves of the columns), joined
// by one shuffle.  Every lane of the warp takes part in the shuffle; other
// warps own no component.
template <int NW>
__device__ __forceinline__ float r_rows(const float *red, int w, int lane)
{
    if (w >= 2) return 0.f;
    const int l = lane & 15;
    const float s = l < 2 * kNI ? row_part<4 * NW>(red, 2 * kNI * w + l, 16 * NW * (lane >> 4), WS<NW>::kRS) : 0.f;
    return s + __shfl_xor_sync(0xffffffffu, s, 16);
}

// P^T delta for lanes 0..4 (rows 0..4, interior k = 3..7): each row is
// summed by lanes k, k + 8, k + 16, k + 24 (a quarter of the columns each),
// joined by two shuffles.  Every lane of the warp takes part.
template <int NW>
__device__ __forceinline__ float ptd_rows(const float *red, int lane)
{
    const int l = lane & 7;
    float s = l < kNI ? row_part<2 * NW>(red, l, 8 * NW * (lane >> 3), WS<NW>::kRS) : 0.f;
    s += __shfl_xor_sync(0xffffffffu, s, 8);
    return s + __shfl_xor_sync(0xffffffffu, s, 16);
}

// The lane's partial of R = F^T (g - F xi1) over its two steps, to column c
// of the transpose rows: R_pos[side][k] = Pd^T rv + Pdd^T ra + P^T r0 and
// R_slack[side][k] = P^T r1 (state order o = 11 blk + k: c_x pos, c_c slack,
// c_y pos, c_s slack).
template <int NW>
__device__ __forceinline__ void dot_partials(float *red, int c, const WBasis &b, const WRes &g)
{
    constexpr int kRS = WS<NW>::kRS;
    float4 d, e;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if ((k & 1) == 0) {
            d = b.pd[k >> 1];
            e = b.pdd[k >> 1];
        }
        float2 px = fmul2(brow(d, k), g.vx), py = fmul2(brow(d, k), g.vy);
        px = ffma2(brow(e, k), g.ax, px);
        py = ffma2(brow(e, k), g.ay, py);
        px = ffma2(b.P[k], g.r0x, px);
        py = ffma2(b.P[k], g.r0y, py);
        const float2 sx = fmul2(b.P[k], g.r1x), sy = fmul2(b.P[k], g.r1y);
        red[k * kRS + c] = px.x + px.y;
        red[(NV + k) * kRS + c] = sx.x + sx.y;
        red[(2 * NV + k) * kRS + c] = py.x + py.y;
        red[(3 * NV + k) * kRS + c] = sy.x + sy.y;
    }
}

// The interior components of the lane's partial of R (k = 3..7 of each
// block), to column c of transpose rows 0..19 (o' = 5 blk + k - 3).
template <int NW>
__device__ __forceinline__ void dot_interior(float *red, int c, const WBasis &b, const WRes &g)
{
    constexpr int kRS = WS<NW>::kRS;
    float4 d, e;
#pragma unroll
    for (int k = kI0; k < kI0 + kNI; ++k) {
        if (k == kI0 || (k & 1) == 0) {
            d = b.pd[k >> 1];
            e = b.pdd[k >> 1];
        }
        float2 px = fmul2(brow(d, k), g.vx), py = fmul2(brow(d, k), g.vy);
        px = ffma2(brow(e, k), g.ax, px);
        py = ffma2(brow(e, k), g.ay, py);
        px = ffma2(b.P[k], g.r0x, px);
        py = ffma2(b.P[k], g.r0y, py);
        const float2 sx = fmul2(b.P[k], g.r1x), sy = fmul2(b.P[k], g.r1y);
        const int i = k - kI0;
        red[i * kRS + c] = px.x + px.y;
        red[(kNI + i) * kRS + c] = sx.x + sx.y;
        red[(2 * kNI + i) * kRS + c] = py.x + py.y;
        red[(3 * kNI + i) * kRS + c] = sy.x + sy.y;
    }
}

// Adds the lane's residual rows to its running sums (slot-major float4s,
// consecutive lanes on consecutive words).
template <int NW>
__device__ __forceinline__ void acc_rows(float *ta, int col, const WRes &g)
{
    constexpr int C = WS<NW>::kCols;
    float4 *a = reinterpret_cast<float4 *>(ta + kWacc) + col;
    const float4 a0 = a[0], a1 = a[C], a2 = a[2 * C], a3 = a[3 * C];
    a[0] = make_float4(a0.x + g.vx.x, a0.y + g.vx.y, a0.z + g.ax.x, a0.w + g.ax.y);
    a[C] = make_float4(a1.x + g.r0x.x, a1.y + g.r0x.y, a1.z + g.r1x.x, a1.w + g.r1x.y);
    a[2 * C] = make_float4(a2.x + g.vy.x, a2.y + g.vy.y, a2.z + g.ay.x, a2.w + g.ay.y);
    a[3 * C] = make_float4(a3.x + g.r0y.x, a3.y + g.r0y.y, a3.z + g.r1y.x, a3.w + g.r1y.y);
}

template <int NW>
__device__ __forceinline__ WRes acc_load(const float *ta, int col)
{
    constexpr int C = WS<NW>::kCols;
    const float4 *a = reinterpret_cast<const float4 *>(ta + kWacc) + col;
    const float4 a0 = a[0], a1 = a[C], a2 = a[2 * C], a3 = a[3 * C];
    return WRes{f2(a0.x, a0.y), f2(a0.z, a0.w), f2(a1.x, a1.y), f2(a1.z, a1.w),
                f2(a2.x, a2.y), f2(a2.z, a2.w), f2(a3.x, a3.y), f2(a3.z, a3.w)};
}

// The whole AM loop for one trajectory on its NW warps.  wi: the warp's index
// within the trajectory (0, 1: the sides of the position step; 0: the
// heading step); b: the lane's basis rows; bid: the trajectory's named
// barrier.
template <int M, int NW>
__device__ void traj_solve(const FusedProblem &p, const float *sm, const WSmem &S, float *ta, int traj, int wi,
                           int lane, int bid, const WBasis &b, int jp, bool valid, bool v1)
{
    const ConstLayout &L = p.L;
    const float *cst = sm + S.cst;
    const float *cob = sm + S.cob;
    float *red = ta + WS<NW>::kRed;
    const int col = 32 * wi + lane;        // the lane's column of the transpose rows
    // lanes 0..9 of warp h < 2 own the interior position-step outputs of
    // side h: block 2h + lane / 5, control point 3 + lane % 5
    const bool owner = wi < 2 && lane < 2 * kNI;
    const int oblk = 2 * wi + lane / kNI, ok = kI0 + lane % kNI;
    const int o = NV * oblk + ok, pp = 12 * oblk + ok, orow = NV * (oblk & 1) + ok;
    // lanes 0..4 of warp 0 own the interior heading coefficients k = 3 + lane
    const bool psi_lane = wi == 0 && lane < kNI;
    const int pk = kI0 + lane;
    const float rho = L.rho;

    // ---- state: xi1, xi2 as given into buffer 1 (wi 0), lam and lam_psi
    // to the owner lanes' registers, then the reference into buffer 0
    if (!AM_WBOUND(traj >= 0 && traj < p.B)) return;
    const float *gs = p.state + (size_t)traj * STATE;
    if (wi == 0) {
        for (int e = lane; e < 55; e += 32) {
            const float v = gs[e];
            if (e < 44) put_xi1(ta, 1, pidx(e), v);
            else put_xi2(ta, 1, e - 44, v);
        }
    }
    float lam = owner ? gs[55 + o] : 0.f;
    float lps = psi_lane ? gs[99 + pk] : 0.f;
    {
        constexpr int C = WS<NW>::kCols;
        float4 *a = reinterpret_cast<float4 *>(ta + kWacc) + col;
        a[0] = a[C] = a[2 * C] = a[3 * C] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (wi == 0 && lane < 12) ta[kWsdx2 + lane] = 0.f;
    }
    float2 dsum = f2(0.f, 0.f);  // the lane's delta summed over the iterations
    pair_sync<NW>(bid);
    // boundary control points from the boundary conditions on every block with
    // boundary rows, the rest as given (entries split between the halves)
    for (int e = col; e < 55; e += WS<NW>::kThreads) {
        const int blk = e / NV, k = e - NV * blk;
        const bool has_bc = (blk == 0 || blk == 2 || blk == 4 || L.cs_boundary);
        float v = blk < 4 ? ta[kWxi + 48 + blk * 12 + k] : ta[kWx2 + 12 + k];
        if (has_bc && k <= 2) v = cst[L.off_ends + blk * 8 + k];
        if (has_bc && k >= 8) v = cst[L.off_ends + blk * 8 + (k - 5)];
        if (blk < 4) put_xi1(ta, 0, blk * 12 + k, v);
        else put_xi2(ta, 0, k, v);
    }
    pair_sync<NW>(bid);

    WSlot st;
    st.nrx = st.nry = f2(3.0e18f, 3.0e18f);  // no near list yet
    st.near0 = st.near1 = 0u;
    st.psi_t = f2(0.f, 0.f);
    WRes g;
    WSums sums;
    const float2 z2 = f2(0.f, 0.f);
    // Step 1 of Sec. III-D: the projections of the initial samples, the
    // residual against the reference.
    {
        const float4 *xdg = reinterpret_cast<const float4 *>(ta + kWxd) + 24;   // buffer 1: given
        const float4 *xdr = reinterpret_cast<const float4 *>(ta + kWxd);        // buffer 0: reference
        float2 pg, pr, dd;
        heading_pair<false>(reinterpret_cast<const float4 *>(ta + kWx2d) + 6, b, pg, dd);
        heading_pair<false>(reinterpret_cast<const float4 *>(ta + kWx2d), b, pr, dd);
        WVals r, f;
        eval_pair(xdg, b, r);
        eval_pair(xdr, b, f);
        sweep_pair<M, false, false, true>(cob, L, pg, z2, jp, valid, v1, r, f, st, g, sums);
        st.psi_cur = pr;
    }
    dot_interior<NW>(red, col, b, g);
    pair_sync<NW>(bid);
    float R = r_rows<NW>(red, wi, lane);  // owner lanes: their component of R
    // The boundary points never move from here on: both buffers take the
    // reference's (buffer 1 held the given samples for the first step).
    if (wi == 0) {
        for (int e = lane; e < 30; e += 32) {
            const int blk = e / 6, i = e - 6 * blk, k = i < 3 ? i : i + 5;
            if (blk < 4) put_xi1(ta, 1, blk * 12 + k, ta[kWxi + blk * 12 + k]);
            else put_xi2(ta, 1, k, ta[kWx2 + k]);
        }
    }
    const float4 *eb = reinterpret_cast<const float4 *>(ta + WS<NW>::kEb) + col;
    eval_boundary<NW>(reinterpret_cast<const float4 *>(ta + kWxd), reinterpret_cast<const float4 *>(ta + kWx2d), b,
                  reinterpret_cast<float4 *>(ta + WS<NW>::kEb) + col);

    float ptp = 0.f;  // heading lanes: P^T delta of the last heading step
    int cur = 0, cur2 = 0;

    for (int it = 0; it <= p.iters; ++it) {
        const bool post = it == p.iters;  // multipliers of the last iteration only
        const bool first = it == 0;
        // ---- XI1: lam' = lam + rho R (not in the first step); u = lam + coef R
        {
            const float u = fmaf(first ? rho : 2.f * rho, R, lam);
            if (!first) {
                lam = fmaf(rho, R, lam);
                // lambda_psi (Eq. update_lambda_psi): P^T (P xi2' - psi_t) = P^T P dxi2 - P^T delta
                if (psi_lane) {
                    const float *dx2 = ta + kWdx2;  // zero at the boundary points
                    const float *pr = sm + S.ptr + pk * 12;
                    float a = 0.f;
#pragma unroll
                    for (int c = kI0; c < kI0 + kNI; ++c) a = fmaf(pr[c], dx2[c], a);
                    lps -= L.psi_sign * L.rho_psi * (a - ptp);
                }
            }
            if (post) break;
            if (owner) ta[kWu + pp] = u;  // the boundary entries of u stay zero
            __syncwarp();
            // xi1' = xi1 + Minv u - MQ xi1 on the interior rows of the side's
            // 22 unknowns (rows of Minv and MQ with columns in blocks of 12; the
            // padding is zero)
            if (owner) {
                const float4 *mr = reinterpret_cast<const float4 *>(sm + S.mir + orow * kMR);
                const float4 *qr = reinterpret_cast<const float4 *>(sm + S.mqr + orow * kMR);
                const float4 *uu = reinterpret_cast<const float4 *>(ta + kWu + 24 * wi);
                const float4 *xx = reinterpret_cast<const float4 *>(ta + kWxi + cur * 48 + 24 * wi);
                // Minv u over the interior columns 3..7 and 15..19 (u is zero
                // elsewhere); MQ xi1 over every column, in order
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int c4 = 0; c4 < 6; ++c4) {
                    const float4 qq = qr[c4], x = xx[c4];
                    if (c4 == 0 || c4 == 3) {
                        a0 = fmaf(mr[c4].w, uu[c4].w, a0);
                    } else if (c4 == 1 || c4 == 4) {
                        const float4 m = mr[c4], uv = uu[c4];
                        a0 = fmaf(m.x, uv.x, a0);
                        a0 = fmaf(m.y, uv.y, a0);
                        a0 = fmaf(m.z, uv.z, a0);
                        a0 = fmaf(m.w, uv.w, a0);
                    }
                    a1 = fmaf(qq.x, x.x, a1);
                    a1 = fmaf(qq.y, x.y, a1);
                    a1 = fmaf(qq.z, x.z, a1);
                    a1 = fmaf(qq.w, x.w, a1);
                }
                put_xi1(ta, cur ^ 1, pp, ta[kWxi + cur * 48 + pp] + (a0 - a1));
            }
            cur ^= 1;
            pair_sync<NW>(bid);
        }
        const bool res = (p.hist != nullptr) || (it == p.iters - 1);
        const bool fin = it == p.iters - 1;
        // ---- EVAL: trajectory values, heading target, the lane's P^T delta
        WVals r;
        {
            eval_interior<NW>(reinterpret_cast<const float4 *>(ta + kWxd) + cur * 24, b, eb, r);
            // psi_t = psi + wrap(atan2(s, c) - psi), psi the previous heading;
            // the heading step works on delta = psi_t - P xi2
            st.psi_t.x = st.psi_prev.x + wrap_pi(atan2_heading(r.s.x, r.c.x) - st.psi_prev.x);
            st.psi_t.y = st.psi_prev.y + wrap_pi(atan2_heading(r.s.y, r.c.y) - st.psi_prev.y);
            const float2 dl = fsub2(st.psi_t, st.psi_cur);
            const float2 dd = f2(valid ? dl.x : 0.f, v1 ? dl.y : 0.f);
            dsum = fadd2(dsum, dd);
#pragma unroll
            for (int k = kI0; k < kI0 + kNI; ++k) {
                const float2 m = fmul2(b.P[k], dd);
                red[(k - kI0) * WS<NW>::kRS + col] = m.x + m.y;
            }
            pair_sync<NW>(bid);
        }
        // ---- PSI: the heading step of Eq. compute_convex_surrogate in increment form
        if (wi == 0) {
            ptp = ptd_rows<NW>(red, lane);
            if (psi_lane) ta[kWv + pk] = fmaf(rho, ptp, lps);  // the boundary entries of v stay zero
            __syncwarp();
            if (psi_lane) {
                const float4 *mr = reinterpret_cast<const float4 *>(sm + S.mpr + pk * 12);
                const float4 *hr = reinterpret_cast<const float4 *>(sm + S.mhr + pk * 12);
                const float4 *vv = reinterpret_cast<const float4 *>(ta + kWv);
                const float4 *xx = reinterpret_cast<const float4 *>(ta + kWx2 + cur2 * 12);
                // Mpsi (.) over the interior columns 3..7 (v is zero elsewhere);
                // Mpsi H xi2 over every column, in order
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int c4 = 0; c4 < 3; ++c4) {
                    const float4 hh = hr[c4], x = xx[c4];
                    if (c4 == 0) a0 = fmaf(mr[0].w, vv[0].w, a0);
                    if (c4 == 1) {
                        const float4 m = mr[1], w = vv[1];
                        a0 = fmaf(m.x, w.x, a0);
                        a0 = fmaf(m.y, w.y, a0);
                        a0 = fmaf(m.z, w.z, a0);
                        a0 = fmaf(m.w, w.w, a0);
                    }
                    a1 = fmaf(hh.x, x.x, a1);
                    a1 = fmaf(hh.y, x.y, a1);
                    a1 = fmaf(hh.z, x.z, a1);
                    if (c4 < 2) a1 = fmaf(hh.w, x.w, a1);
                }
                const float d = a0 - a1;
                put_xi2(ta, cur2 ^ 1, pk, ta[kWx2 + cur2 * 12 + pk] + d);
                ta[kWdx2 + pk] = d;
                ta[kWsdx2 + pk] += d;
            }
        }
        cur2 ^= 1;
        pair_sync<NW>(bid);
        // ---- SWEEP and DOT
        {
            const float4 *x2d = reinterpret_cast<const float4 *>(ta + kWx2d) + cur2 * 6;
            float2 ps, pdd;
            if (res) heading_interior<NW, true>(x2d, b, eb, ps, pdd);
            else heading_interior<NW, false>(x2d, b, eb, ps, pdd);
            if (fin) sweep_pair<M, true, true, false>(cob, L, ps, pdd, jp, valid, v1, r, r, st, g, sums);
            else if (res) sweep_pair<M, true, false, false>(cob, L, ps, pdd, jp, valid, v1, r, r, st, g, sums);
            else sweep_pair<M, false, false, false>(cob, L, ps, pdd, jp, valid, v1, r, r, st, g, sums);
            acc_rows<NW>(ta, col, g);
            dot_interior<NW>(red, col, b, g);
            double *hs = reinterpret_cast<double *>(ta + kWsum);
            if (res) {
                // the sums over the steps of the residuals and the cost in FP64
                const double a_res = warp_sum(double(sums.res.x) + double(sums.res.y));
                const double a_psi = warp_sum(double(sums.rpsi.x) + double(sums.rpsi.y));
                const double a_cost = warp_sum(double(sums.cost.x) + double(sums.cost.y));
                float dm = 3.0e38f;
                if (fin) {
                    dm = fminf(sums.dmin.x, sums.dmin.y);
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) dm = fminf(dm, __shfl_xor_sync(0xffffffffu, dm, off));
                }
                if (lane == 0) {
                    hs[4 * wi] = a_res;
                    hs[4 * wi + 1] = a_psi;
                    hs[4 * wi + 2] = a_cost;
                    hs[4 * wi + 3] = dm;
                }
            }
            pair_sync<NW>(bid);
            if (res && wi == 0 && lane == 0) {
                double sr = hs[0], sp = hs[1], sc = hs[2], sdm = hs[3];
#pragma unroll
                for (int k = 1; k < NW; ++k) {
                    sr += hs[4 * k];
                    sp += hs[4 * k + 1];
                    sc += hs[4 * k + 2];
                    sdm = fmin(sdm, hs[4 * k + 3]);
                }
                const float vr = float(sqrt(sr)), vp = float(sqrt(sp));
                const float vc = float(sc);
                if (p.hist) {
                    float *hd = p.hist + ((size_t)traj * p.iters + it) * 3;
                    hd[0] = vr;
                    hd[1] = vp;
                    hd[2] = vc;
                }
                if (fin) {
                    p.res[traj] = vr;
                    p.res_psi[traj] = vp;
                    p.cost[traj] = vc;
                    p.mind[traj] = sqrtf(float(sdm));
                }
            }
            R = r_rows<NW>(red, wi, lane);
        }
    }
    // ---- the state back: xi1 (cur), xi2 (cur2), lam, lam_psi.  The
    // multipliers' boundary components: lam_b' = lam_b + rho F_b^T (sum of
    // the residual rows of the iterations), and lam_psi_b' = lam_psi_b -
    // sign rho_psi (P^T P sum(dxi2) - P^T sum(delta))_b (Eq. update_lambda_1
    // and update_lambda_psi summed over the iterations; both are linear).
    float *gd = p.state + (size_t)traj * STATE;
    pair_sync<NW>(bid);  // every R row read before the rows are reused
    dot_partials<NW>(red, col, b, acc_load<NW>(ta, col));
    pair_sync<NW>(bid);
    if (wi < 2 && lane < NS) {
        const int ob = NS * wi + lane;
        if (!interior(ob % NV)) gd[55 + ob] = fmaf(rho, row_sum<NW>(red, ob), gs[55 + ob]);
    }
    pair_sync<NW>(bid);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float2 m = fmul2(b.P[k], dsum);
        red[k * WS<NW>::kRS + col] = m.x + m.y;
    }
    pair_sync<NW>(bid);
    if (wi == 0) {
        if (lane < NV && !interior(lane)) {
            const float *pr = sm + S.ptr + lane * 12;
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < NV; ++c) a = fmaf(pr[c], ta[kWsdx2 + c], a);
            gd[99 + lane] = gs[99 + lane] - L.psi_sign * L.rho_psi * (a - row_sum<NW>(red, lane));
        }
        for (int e = lane; e < 55; e += 32)
            gd[e] = e < 44 ? ta[kWxi + cur * 48 + pidx(e)] : ta[kWx2 + cur2 * 12 + (e - 44)];
        if (psi_lane) gd[99 + pk] = lps;
    }
    if (owner) gd[55 + o] = lam;
    pair_sync<NW>(bid);  // the area is free for the next trajectory
}

// Stages a problem's small matrices and obstacle sections into shared memory
// (two bulk copies on one mbarrier, waited on with a bound) while zeroing the
// rest of the area, then forms the row-major copies of Minv, MQ, Mpsi, Mpsi H
// and P^T P and the pair-interleaved Pd, Pdd.  Every thread of the block
// calls it; false (for every thread) when the wait ran out.
template <int NW>
__device__ bool stage_problem(const FusedProblem &p, float *sm, const WSmem &S, uint64_t *bar, uint32_t parity)
{
    const ConstLayout &L = p.L;
    if (threadIdx.x == 0) {
        const uint32_t b0 = uint32_t(L.off_obs - L.off_mt) * 4u, b1 = uint32_t(L.total - L.off_obt) * 4u;
        // order the block's earlier generic-proxy accesses of this area
        // before the asynchronous copies overwrite it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     :: "r"(smem_u32(bar)), "r"(b0 + b1) : "memory");
        if (!L.diag_stall) {
            bulk_load(sm + S.cst + L.off_mt, p.cblob + L.off_mt, b0, bar);
            if (b1) bulk_load(sm + S.cob, p.cblob + L.off_obt, b1, bar);
        }
    }
    for (int i = S.mir + threadIdx.x; i < S.total; i += blockDim.x) sm[i] = 0.f;
    int ok = 0;
    {
        const uint64_t t0 = global_ns();
        for (int spin = 0; spin < (1 << 26) && !ok; ++spin) {
            ok = mbar_try_wait(bar, parity) ? 1 : 0;
            if (!ok && global_ns() - t0 > kWaitLimitNs) break;
        }
    }
    if (__syncthreads_and(ok) == 0) return false;
    const float *cst = sm + S.cst;
    for (int i = threadIdx.x; i < NS * NS; i += blockDim.x) {
        const int row = i / NS, c = i - NS * row, cp = c < NV ? c : c + 1;
        sm[S.mir + row * kMR + cp] = cst[L.off_mt + c * 24 + row];
        sm[S.mqr + row * kMR + cp] = cst[L.off_mq + c * 24 + row];
    }
    for (int i = threadIdx.x; i < NV * NV; i += blockDim.x) {
        const int k = i / NV, c = i - NV * k;
        sm[S.mpr + k * 12 + c] = cst[L.off_mpsi + c * 12 + k];
        sm[S.mhr + k * 12 + c] = cst[L.off_mpsih + c * 12 + k];
        sm[S.ptr + k * 12 + c] = cst[L.off_ptp + c * 12 + k];
    }
    // Pd, Pdd per pair of steps (global rows [3][q][12]); entries past the
    // horizon, and the last pair, stay zero
    const float *rows = p.cblob + L.off_prow;
    for (int i = threadIdx.x; i < 2 * L.q * NV; i += blockDim.x) {
        const int ty = i / (L.q * NV), rem = i - ty * L.q * NV, t = rem / NV, k = rem - NV * t;
        sm[S.pb + (ty * WS<NW>::kPairs + (t >> 1)) * kPB + 2 * k + (t & 1)] =
            __ldg(rows + ((1 + ty) * L.q + t) * 12 + k);
    }
    __syncthreads();
    return true;
}

// The lane's pair of steps and its basis rows for a problem of horizon q.
struct WLane {
    WBasis b;
    int jp;
    bool valid, v1;
};

template <int NW>
__device__ __forceinline__ void lane_setup(const FusedProblem &p, const float *sm, const WSmem &S, int wi,
                                           int lane, WLane &w)
{
    const int q = p.L.q, np = (q + 1) >> 1, nh = (np + NW - 1) / NW;
    const int j = wi * nh + lane;
    w.valid = lane < nh && j < np;
    w.v1 = w.valid && 2 * j + 1 < q;
    load_basis<NW>(p.cblob + p.L.off_prow, sm + S.pb, w.valid ? j : WS<NW>::kPairs - 1, w.valid, w.v1, w.b);
    w.jp = w.valid ? j : 0;  // obstacle-track pair (in range for every lane)
}

__device__ __forceinline__ void init_stage_barrier(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
}

template <int M, int NW>
__global__ void __launch_bounds__(kWMaxWarps * 32, 1) am_warp_kernel(FusedProblem p)
{
    extern __shared__ __align__(128) float sm[];
    const int T = blockDim.x / WS<NW>::kThreads;
    const WSmem S = wsmem_layout<NW>(p.L, T);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S.bar);
#ifdef AM_DEBUG_BOUNDS
    if (threadIdx.x == 0) g_woob = 0;
#endif
    init_stage_barrier(bar);
    if (!stage_problem<NW>(p, sm, S, bar, 0)) {
        if (threadIdx.x == 0) atomicExch(p.err, 1);
        return;
    }
    const int slot = threadIdx.x / WS<NW>::kThreads, wi = (threadIdx.x >> 5) % NW, lane = threadIdx.x & 31;
    float *ta = sm + S.traj + slot * WS<NW>::kTrajFloats;
    WLane w;
    lane_setup<NW>(p, sm, S, wi, lane, w);
    for (int traj = blockIdx.x * T + slot; traj < p.B; traj += gridDim.x * T)
        traj_solve<M, NW>(p, sm, S, ta, traj, wi, lane, 1 + slot, w.b, w.jp, w.valid, w.v1);
#ifdef AM_DEBUG_BOUNDS
    __syncthreads();
    if (threadIdx.x == 0 && g_woob) atomicOr(p.err, 2);
#endif
}

// Uneven batching with the warp-pair kernel: persistent CTAs of up to 16 / NW
// trajectory slots (one count per launch, the most that every problem of
// the variant fits in shared memory) take work items (problem, tile of at most that many
// trajectories) of variant v from a list in order, through one atomic
// counter, and re-stage constants whenever they move to another problem.
// Each slot's NW warps run one trajectory of the tile.  A variant holds the
// problems of one circle count and one NW.  The lists
// live in device memory, as for the small-tile group kernels.
//   head[v]: number of items of variant v; head[kGroupVariants + v]: offset of its list
//   ctl[2 v]: its work counter (zeroed before the launch); ctl[2 v + 1]: status
template <int M, int NW>
__global__ void __launch_bounds__(kWMaxWarps * 32, 1)
am_group_warp_kernel(const FusedProblem *probs, const int *items, const int *head, int *ctl, int v)
{
    int *counter = ctl + 2 * v;
    const int nitems = head[v];
    const int *list = items + 2 * head[kGroupVariants + v];
    extern __shared__ __align__(128) float sm[];
    __shared__ FusedProblem kp;
    __shared__ int s_item;
    // the barrier sits at the start of the area, as in every layout below
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
#ifdef AM_DEBUG_BOUNDS
    if (threadIdx.x == 0) g_woob = 0;
#endif
    init_stage_barrier(bar);
    const int TM = blockDim.x / WS<NW>::kThreads;  // trajectory slots
    const int slot = threadIdx.x / WS<NW>::kThreads, wi = (threadIdx.x >> 5) % NW, lane = threadIdx.x & 31;
    int cur = -1;
    uint32_t parity = 0;
    WLane w;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int pi = list[2 * it], tile = list[2 * it + 1];
        if (pi != cur) {
            if (threadIdx.x == 0) kp = probs[pi];
            __syncthreads();
            if (!stage_problem<NW>(kp, sm, wsmem_layout<NW>(kp.L, TM), bar, parity)) {
                if (threadIdx.x == 0) {
                    atomicExch(kp.err, 1);
                    atomicExch(ctl + 2 * v + 1, 1);
                }
                return;
            }
            parity ^= 1u;
            cur = pi;
            lane_setup<NW>(kp, sm, wsmem_layout<NW>(kp.L, TM), wi, lane, w);
        }
        const WSmem S = wsmem_layout<NW>(kp.L, TM);
        const long long lo = (long long)tile * kp.B / kp.ntiles, hi = (long long)(tile + 1) * kp.B / kp.ntiles;
        const int traj = int(lo) + slot;
        if (traj < hi)
            traj_solve<M, NW>(kp, sm, S, sm + S.traj + slot * WS<NW>::kTrajFloats, traj, wi, lane, 1 + slot, w.b,
                              w.jp, w.valid, w.v1);
        __syncthreads();
    }
#ifdef AM_DEBUG_BOUNDS
    __syncthreads();
    if (threadIdx.x == 0 && g_woob) atomicOr(kp.err, 2);
#endif
}

std::mutex g_warp_mu;

template <int M, int NW>
int launch_warp_mn(const FusedProblem &p, int T, size_t smem, int grid, cudaStream_t st)
{
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_warp_mu);
        if (attr_dev != dev) {
            if (cudaFuncSetAttribute(am_warp_kernel<M, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(kFusedSmemMax)) != cudaSuccess)
                return -2;
            attr_dev = dev;
        }
    }
    am_warp_kernel<M, NW><<<grid, T * WS<NW>::kThreads, smem, st>>>(p);
    return 0;
}

template <int M, int NW>
cudaError_t launch_group_warp_mn(const GroupLaunch &g, cudaStream_t st)
{
    cudaError_t r = cudaError_t(raise_smem_limit(reinterpret_cast<const void *>(am_group_warp_kernel<M, NW>), g.smem));
    if (r != cudaSuccess) return r;
    am_group_warp_kernel<M, NW><<<g.grid, g.slots * WS<NW>::kThreads, g.smem, st>>>(
        g.d_probs, g.d_items, g.d_head, g.d_ctl, g.variant);
    return cudaPeekAtLastError();
}

int max_traj(int nw) { return nw == 2 ? WS<2>::kMaxTraj : nw == 3 ? WS<3>::kMaxTraj : WS<4>::kMaxTraj; }

}  // namespace

size_t warp_smem_bytes(const ConstLayout &L, int T)
{
    const int nw = warps_for_q(L.q);
    const int total = nw == 2 ? wsmem_layout<2>(L, T).total : nw == 3 ? wsmem_layout<3>(L, T).total
                                                                      : wsmem_layout<4>(L, T).total;
    return size_t(total) * sizeof(float);
}

int warp_supported(const ConstLayout &L)
{
    // every block needs its boundary rows (cs_boundary): the kernel moves
    // only the interior control points
    if (L.precision != 0 || L.alpha_mode != 0 || !L.cs_boundary) return 0;
    if (L.q < 2 || L.q > kWMaxQ || L.m < 1 || L.m > MAXM || L.n > 64) return 0;
    return warp_smem_bytes(L, 1) <= kFusedSmemMax ? 1 : 0;
}

int warp_max_traj(const ConstLayout &L) { return max_traj(warps_for_q(L.q)); }

int warp_auto_traj(const ConstLayout &L, int B, int sms)
{
    // fewest rounds of trajectories per CTA slot, then the fewest
    // trajectories per CTA that keep that number of rounds
    const int tmax = warp_max_traj(L);
    const long long slots = (long long)sms * tmax;
    const long long rounds = (B + slots - 1) / slots;
    long long T = (B + (long long)sms * rounds - 1) / ((long long)sms * rounds);
    if (T < 1) T = 1;
    if (T > tmax) T = tmax;
    while (T > 1 && warp_smem_bytes(L, int(T)) > kFusedSmemMax) --T;
    return int(T);
}

int warp_group_traj(const ConstLayout &L)
{
    if (!warp_supported(L)) return 0;
    int T = warp_max_traj(L);
    while (T > 0 && warp_smem_bytes(L, T) > kGroupSmemLimit) --T;
    return T;
}

int warp_group_variant(const ConstLayout &L) { return kGroupWarpVariant0 + 4 * (warps_for_q(L.q) - 2) + L.m - 1; }

int launch_group_warp(const GroupLaunch &g, void *stream, int *launches, const char **why)
{
    *why = nullptr;
    const int k = g.variant - kGroupWarpVariant0, M = k % 4 + 1, NW = k / 4 + 2;
    if (k < 0 || NW > 4 || g.grid < 1 || g.smem > kGroupSmemLimit || g.slots < 1 || g.slots > max_traj(NW))
        return -1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(g.d_ctl + 2 * g.variant, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return -2;
    }
    switch (4 * (NW - 2) + M - 1) {
#define AM_WG(MM, NN)                                                                                        \
    case 4 * (NN - 2) + MM - 1:                                                                              \
        e = launch_group_warp_mn<MM, NN>(g, st);                                                             \
        break;
        AM_WG(1, 2) AM_WG(2, 2) AM_WG(3, 2) AM_WG(4, 2)
        AM_WG(1, 3) AM_WG(2, 3) AM_WG(3, 3) AM_WG(4, 3)
        AM_WG(1, 4) AM_WG(2, 4) AM_WG(3, 4) AM_WG(4, 4)
#undef AM_WG
    default:
        return -1;
    }
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return -2;
    }
    if (launches) ++*launches;
    return 0;
}

int launch_warp(const SolveArgs &a, void *stream, int *launches)
{
    const ConstLayout &L = a.L;
    if (!warp_supported(L)) return -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return -2;
    const int T = a.tile > 0 ? a.tile : warp_auto_traj(L, a.B, sms);
    if (T < 1 || T > warp_max_traj(L)) return -1;
    const size_t smem = warp_smem_bytes(L, T);
    if (smem > kFusedSmemMax) return -1;
    FusedProblem p;
    p.cblob = a.cblob;
    p.L = L;
    p.B = a.B;
    p.iters = a.iters;
    p.T = T;
    p.ntiles = (a.B + T - 1) / T;
    p.state = a.state;
    p.res = a.res;
    p.res_psi = a.res_psi;
    p.cost = a.cost;
    p.mind = a.mind;
    p.hist = a.hist;
    p.err = a.err;
    const int grid = p.ntiles < sms ? p.ntiles : sms;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nw = warps_for_q(L.q);
    int rc = -1;
    switch (4 * (nw - 2) + L.m - 1) {
#define AM_W(MM, NN)                                                                                         \
    case 4 * (NN - 2) + MM - 1:                                                                              \
        rc = launch_warp_mn<MM, NN>(p, T, smem, grid, st);                                                   \
        break;
        AM_W(1, 2) AM_W(2, 2) AM_W(3, 2) AM_W(4, 2)
        AM_W(1, 3) AM_W(2, 3) AM_W(3, 3) AM_W(4, 3)
        AM_W(1, 4) AM_W(2, 4) AM_W(3, 4) AM_W(4, 4)
#undef AM_W
    default:
        return -1;
    }
    if (rc) return rc;
    if (launches) ++*launches;
    // peek: the caller reports the launch error's text
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam
