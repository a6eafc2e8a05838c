// Large-batch kernel of the batched alternating-minimization loop (Sec.
// III-D, in the batch matrix form of Sec. III-E, Eq. over_3) on the
// fifth-generation tensor cores.
//
// A persistent CTA per SM works through tiles of 128 trajectories.  A
// trajectory is a row of every batched product and a lane of the tensor
// memory, so each dense product of an iteration is a chain of tcgen05.mma
// instructions (M = 128) over the whole tile:
//   * the position step in increment form, xi1' = xi1 + Minv u - MQ xi1 with
//     u = lam + coef R, per side [128 x 32] x [32 x 32] + [128 x 24] x [24 x 32];
//   * the trajectory values of Eq. param at a chunk of 16 steps, per
//     coefficient block [128 x 16] x [16 x 16 t] (P rows; P, Pd, Pdd rows at
//     once for the position blocks), and the heading step's P^T delta;
//   * the contraction R = F^T (g - F xi1) of the residual rows the sweep
//     writes, per row block [128 x 16 t] x [16 t x 16], accumulated over the
//     chunks in tensor memory.
// Each product keeps FP32 accuracy with three TF32 products (lo*hi + hi*lo +
// hi*hi, x = hi + lo, hi the TF32 rounding of x and lo = x - hi exactly).  The
// operands the threads produce (u, delta, the residual rows) are written to
// tensor memory (tcgen05.st) and read from there by the MMA; the coefficient
// blocks and the constant basis, Minv and MQ operands sit in shared memory
// in the K-major layout without swizzle (8-row x 16-byte core matrices, 128
// bytes apart along K, 8-row groups K/4 core matrices apart).
//
// Threads: 16 warps, four per 32-lane quadrant of the tensor memory (warp w
// reads lanes 32 (w mod 4) .. + 31: trajectories), each taking one quarter
// of the steps of a chunk (two pairs of consecutive steps).  Lane 0 of the
// four warps of the last quarter issues the tensor-core work, each issuer
// its own accumulators, and signals completion through mbarriers that count
// the four issuers (tcgen05.commit, or a plain arrive when it issued
// nothing); every thread waits on them with a bounded wait.  (A separate
// issuing warp would cap the registers at 96: five warps on one scheduler.)  The sweep (closed-form alpha/d steps, velocity and
// acceleration bounds, residual rows) is FP32 SIMT with paired instructions
// as in the small-tile kernel.  Its near-obstacle test compares the bounding
// box of the warp's 32 robot centres (warp-wide min / max) with every
// obstacle at once, one obstacle per lane.
//
// Per iteration:
//   XI1   lam and u from R; the position step on the tensor cores
//   EVAL  c, s, psi at every step (tensor cores, three chunks at a time);
//         psi_t and delta per step; P^T delta (tensor cores)
//   PSI   the heading step and the lambda_psi update (Eq. update_lambda_psi),
//         one thread per trajectory
//   SWEEP per chunk of 16 steps: x ... psi (tensor cores), then the
//         closed-form steps and residual rows (SIMT), then R (tensor cores);
//         the values of chunk c + 1 are formed while chunk c is swept.
// The sums of the last iteration (residuals, cost, smallest distance) are
// formed per thread over its steps in FP64 and combined per trajectory.
//
// The kernel covers the default alpha form, the FP32 precision form and
// horizons of at most 128 steps, without per-iteration history; the host
// checks the shape against the shared-memory limit.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "am_async.cuh"
#include "am_heading.cuh"
#include "am_internal.h"

namespace trajam {
namespace {

constexpr int kLT = 128;                      // trajectories per tile: the MMA's M, one lane each
constexpr int kLThreads = 512;                // 16 warps
constexpr int kIssuers = 4;                   // lane 0 of warps 12..15 issue the tensor-core work
constexpr int kChunk = 16;                    // steps per chunk of the sweep
constexpr int kGroup = 3;                     // chunks per group of the heading-target pass
constexpr int kAK = 76;                       // K extent of the coefficient operand: 6 blocks of 12, + 4
constexpr int kLMaxQ = 128;                   // delta (hi, lo) of every step fits 256 columns
constexpr float kBoxMargin = 0.05f;           // metres added to the reach of the near-obstacle test

// Tensor-memory columns (512 allocated).
constexpr uint32_t kTmR = 0;    // R: per side c_pos (16) | c_slack (16); P^T delta (16) in EVAL
constexpr uint32_t kTmE = 64;   // trajectory values of a chunk (192); xi1 increment (64) in XI1
constexpr uint32_t kTmA = 256;  // residual rows of a chunk, hi (128) | lo (128); delta; u
constexpr uint32_t kTmCols = 512;
// Column of each trajectory value within a sweep chunk (16 steps each).
constexpr int kQx = 0, kQxd = 16, kQxdd = 32, kQy = 48, kQyd = 64, kQydd = 80, kQc = 96, kQs = 112,
              kQpsi = 128, kQpsidd = 160, kQpsio = 176;

// Debug build (-DAM_DEBUG_BOUNDS): a failed index check sets the block's
// flag and skips the access; the flag becomes bit 2 of the status word.
#ifdef AM_DEBUG_BOUNDS
__shared__ int g_loob;
#define AM_LBOUND(cond) ((cond) ? true : (g_loob = 1, false))
#else
#define AM_LBOUND(cond) true
#endif

// Shared-memory layout (byte offsets, 128-byte aligned sections).
//   bar   three mbarriers (constant copy, value products, R products) and
//         the tensor-memory base address
//   ob    the obstacle region [off_obt, total) of the constant block
//   ps    Mpsi^T, (Mpsi H)^T, P^T P, each [NV][12]
//   eb    [2][qc][48][16] value operand B per chunk: rows P | Pd | Pdd at the
//         chunk's 16 steps, K = basis index (hi part, then lo part)
//   rb    [2][3][16][qk]  contraction operand B: rows = basis index, K = step,
//         for P, Pd, Pdd
//   mi    [2][32][32]     Minv (rows and columns in blocks of 16 per side)
//   nq    [2][32][24]     -MQ (rows in blocks of 16, columns in blocks of 12)
//   ae    [2][128][76]    coefficient operand A: blocks of 12 c_x, c_c, c_y,
//         c_s, c_psi, previous c_psi
//   lps   [128][13]       lambda_psi
//   sums  [128][4][3] double + [128][4] float: the last iteration's sums per
//         thread; in the first sweep [128][25] float boundary differences
struct LSmem {
    int bar, ob, ps, eb, rb, mi, nq, ae, lps, sums, total;
    int qc, qk;
};

__host__ __device__ inline int align128(int b) { return (b + 127) & ~127; }

__host__ __device__ inline LSmem lsmem_layout(const ConstLayout &L)
{
    LSmem s;
    s.qc = (L.q + kChunk - 1) / kChunk;
    s.qk = s.qc * kChunk;
    int o = 0;
    s.bar = o; o += 128;
    s.ob = o; o = align128(o + (L.total - L.off_obt) * 4);
    s.ps = o; o = align128(o + 3 * NV * 12 * 4);
    s.eb = o; o = align128(o + 2 * s.qc * 48 * 16 * 4);
    s.rb = o; o = align128(o + 2 * 3 * 16 * s.qk * 4);
    s.mi = o; o = align128(o + 2 * 32 * 32 * 4);
    s.nq = o; o = align128(o + 2 * 32 * 24 * 4);
    s.ae = o; o = align128(o + 2 * kLT * kAK * 4);
    s.lps = o; o = align128(o + kLT * 13 * 4);
    s.sums = o; o = align128(o + kLT * 4 * 3 * 8 + kLT * 4 * 4);
    s.total = o;
    return s;
}

// Float index of element (r, k) of an operand with K extent K (a multiple of
// 4) in the K-major layout without swizzle.
__host__ __device__ inline int kmaj(int r, int k, int K)
{
    return (r >> 3) * (K * 8) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// ---------------------------------------------------------- tcgen05 access

// Shared-memory matrix descriptor: start address, leading (K) byte offset
// 128, stride (8-row group) byte offset sbo, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo)
{
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t(128u >> 4) << 16) | (uint64_t((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// M = 128 and the given N.
__host__ __device__ constexpr uint32_t idesc_tf32(int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kLT >> 4) << 24);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 :: "r"(d), "r"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

// Three TF32 products into one accumulator: lo*hi + hi*lo + hi*hi.
__device__ __forceinline__ void mma3_ss(uint32_t d, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, uint32_t id,
                                        bool acc)
{
    mma_ss(d, al, bh, id, acc ? 1u : 0u);
    mma_ss(d, ah, bl, id, 1u);
    mma_ss(d, ah, bh, id, 1u);
}

__device__ __forceinline__ void mma3_ts(uint32_t d, uint32_t ah, uint32_t al, uint64_t bh, uint64_t bl, uint32_t id,
                                        bool acc)
{
    mma_ts(d, al, bh, id, acc ? 1u : 0u);
    mma_ts(d, ah, bl, id, 1u);
    mma_ts(d, ah, bh, id, 1u);
}

// The mbarrier's phase completes when every tensor-core operation issued so
// far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void tm_ld4(uint32_t ta, float4 &v)
{
    uint32_t a, b, c, d;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "r"(ta));
    v = make_float4(__uint_as_float(a), __uint_as_float(b), __uint_as_float(c), __uint_as_float(d));
}

__device__ __forceinline__ void tm_ld16(uint32_t ta, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(ta));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Values loaded from tensor memory are defined only after the wait: each is
// passed through an empty statement ordered after it.
__device__ __forceinline__ void hold(float &x) { asm volatile("" : "+f"(x)); }
__device__ __forceinline__ void hold(float4 &v)
{
    hold(v.x);
    hold(v.y);
    hold(v.z);
    hold(v.w);
}

__device__ __forceinline__ void tm_st2(uint32_t ta, float a, float b)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n"
                 :: "r"(ta), "r"(__float_as_uint(a)), "r"(__float_as_uint(b)) : "memory");
}

__device__ __forceinline__ void tm_st4(uint32_t ta, const float (&v)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n"
                 :: "r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])) : "memory");
}

__device__ __forceinline__ void tm_st16(uint32_t ta, const float (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                 "%12, %13, %14, %15, %16};\n"
                 :: "r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                    "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                    "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                    "r"(__float_as_uint(v[15]))
                 : "memory");
}

__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// x = hi + lo with hi = x rounded to TF32 (to nearest, ties away from zero,
// on the bit pattern) and lo = x - hi, exact in FP32.
__device__ __forceinline__ void split(float x, float &hi, float &lo)
{
    hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
    lo = x - hi;
}

// ---------------------------------------------------------- paired FP32

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// Steps e, e + 1 of four consecutive steps held as a float4 (e = 0 or 2).
__device__ __forceinline__ float2 pick(const float4 &v, int e) { return e == 0 ? f2(v.x, v.y) : f2(v.z, v.w); }
__device__ __forceinline__ float comp(const float4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

__device__ __forceinline__ float warp_min(float v)
{
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;\n" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float warp_max(float v)
{
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;\n" : "=f"(r) : "f"(v));
    return r;
}

// ---------------------------------------------------------- operands

// Shared-memory byte addresses of the tensor-core operands.
struct LAddr {
    uint32_t eb, eb_lo, rb, rb_lo, mi, mi_lo, nq, nq_lo, ae, ae_lo;
};

__device__ __forceinline__ LAddr laddr(unsigned char *smb, const LSmem &S)
{
    const uint32_t b = smem_u32(smb);
    LAddr a;
    a.eb = b + S.eb;
    a.eb_lo = a.eb + S.qc * 48 * 16 * 4;
    a.rb = b + S.rb;
    a.rb_lo = a.rb + 3 * 16 * S.qk * 4;
    a.mi = b + S.mi;
    a.mi_lo = a.mi + 32 * 32 * 4;
    a.nq = b + S.nq;
    a.nq_lo = a.nq + 32 * 24 * 4;
    a.ae = b + S.ae;
    a.ae_lo = a.ae + kLT * kAK * 4;
    return a;
}

// Entries k0 .. k0 + 11 (k0 a multiple of 4) of row i of the coefficient operand.
__device__ __forceinline__ void ae_get(const unsigned char *smb, const LSmem &S, int i, int k0, float (&v)[12])
{
    const float *hi = reinterpret_cast<const float *>(smb + S.ae), *lo = hi + kLT * kAK;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int o = kmaj(i, k0 + 4 * j, kAK);
        const float4 h = *reinterpret_cast<const float4 *>(hi + o), l = *reinterpret_cast<const float4 *>(lo + o);
        v[4 * j] = h.x + l.x;
        v[4 * j + 1] = h.y + l.y;
        v[4 * j + 2] = h.z + l.z;
        v[4 * j + 3] = h.w + l.w;
    }
}

__device__ __forceinline__ void ae_put(unsigned char *smb, const LSmem &S, int i, int k0, const float (&v)[12])
{
    if (!AM_LBOUND(i >= 0 && i < kLT && k0 >= 0 && k0 + 12 <= kAK)) return;
    float *hi = reinterpret_cast<float *>(smb + S.ae), *lo = hi + kLT * kAK;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int o = kmaj(i, k0 + 4 * j, kAK);
        float4 h, l;
        split(v[4 * j], h.x, l.x);
        split(v[4 * j + 1], h.y, l.y);
        split(v[4 * j + 2], h.z, l.z);
        split(v[4 * j + 3], h.w, l.w);
        *reinterpret_cast<float4 *>(hi + o) = h;
        *reinterpret_cast<float4 *>(lo + o) = l;
    }
}

// The constant operands, split into TF32 (hi, lo), from the constant block in
// global memory; the coefficient operand zeroed (its padding must read 0).
__device__ void build_operands(const FusedProblem &p, unsigned char *smb, const LSmem &S)
{
    const ConstLayout &L = p.L;
    const float *g = p.cblob;
    const int q = L.q, qk = S.qk;
    float *eb = reinterpret_cast<float *>(smb + S.eb), *rb = reinterpret_cast<float *>(smb + S.rb);
    float *mi = reinterpret_cast<float *>(smb + S.mi), *nq = reinterpret_cast<float *>(smb + S.nq);
    float *ps = reinterpret_cast<float *>(smb + S.ps), *ae = reinterpret_cast<float *>(smb + S.ae);
    const int neb = S.qc * 768;
    for (int x = threadIdx.x; x < neb; x += blockDim.x) {
        const int c = x / 768, r = (x % 768) >> 4, k = x & 15, mat = r >> 4, t = kChunk * c + (r & 15);
        const float v = (t < q && k < NV) ? g[L.off_prow + (mat * q + t) * 12 + k] : 0.f;
        const int o = c * 768 + kmaj(r, k, 16);
        split(v, eb[o], eb[neb + o]);
    }
    const int nrb = 3 * 16 * qk;
    for (int x = threadIdx.x; x < nrb; x += blockDim.x) {
        const int mat = x / (16 * qk), rem = x % (16 * qk), r = rem / qk, t = rem % qk;
        const float v = (r < NV && t < q) ? g[L.off_prow + (mat * q + t) * 12 + r] : 0.f;
        const int o = mat * 16 * qk + kmaj(r, t, qk);
        split(v, rb[o], rb[nrb + o]);
    }
    for (int x = threadIdx.x; x < 32 * 32; x += blockDim.x) {
        const int r = x >> 5, c = x & 31, br = r >> 4, kr = r & 15, bc = c >> 4, kc = c & 15;
        const float v = (kr < NV && kc < NV) ? g[L.off_mt + (NV * bc + kc) * 24 + NV * br + kr] : 0.f;
        const int o = kmaj(r, c, 32);
        split(v, mi[o], mi[1024 + o]);
    }
    for (int x = threadIdx.x; x < 32 * 24; x += blockDim.x) {
        const int r = x / 24, c = x % 24, br = r >> 4, kr = r & 15, bc = c / 12, kc = c % 12;
        const float v = (kr < NV && kc < NV) ? -g[L.off_mq + (NV * bc + kc) * 24 + NV * br + kr] : 0.f;
        const int o = kmaj(r, c, 24);
        split(v, nq[o], nq[768 + o]);
    }
    for (int x = threadIdx.x; x < 3 * NV * 12; x += blockDim.x) {
        const int sec = x / (NV * 12), e = x % (NV * 12);
        ps[x] = g[(sec == 0 ? L.off_mpsi : sec == 1 ? L.off_mpsih : L.off_ptp) + e];
    }
    for (int x = threadIdx.x; x < 2 * kLT * kAK; x += blockDim.x) ae[x] = 0.f;
}

// Stage the obstacle region (bulk async copy, completion on an mbarrier)
// while the operands are built; the wait is bounded and the block agrees on
// its outcome.
__device__ bool lstage(const FusedProblem &p, unsigned char *smb, const LSmem &S, uint64_t *bar)
{
    const ConstLayout &L = p.L;
    if (threadIdx.x == 0) {
        const uint32_t bytes = uint32_t(L.total - L.off_obt) * 4u;
        const uint32_t expect = bytes + (L.diag_stall ? 16u : 0u);  // diagnostic: never completes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     :: "r"(smem_u32(bar)), "r"(expect) : "memory");
        if (bytes && !L.diag_stall) bulk_load(smb + S.ob, p.cblob + L.off_obt, bytes, bar);
    }
    build_operands(p, smb, S);
    const bool ok = mbar_wait_bounded(bar, 0);
    proxy_fence();  // the operands written above, before the tensor cores read them
    return __syncthreads_and(ok) != 0;
}

// ---------------------------------------------------------- MMA issue (one thread)

// Values of coefficient block blk at chunk c: rows P (n = 16) or P | Pd | Pdd
// (n = 48) of the chunk's steps, into columns d ...
__device__ __forceinline__ void mma_values(const LAddr &A, uint32_t d, int blk, int n, int c)
{
    const uint32_t id = idesc_tf32(n);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t ao = uint32_t(3 * blk + 2 * h) * 128u, bo = uint32_t(c) * 3072u + uint32_t(h) * 256u;
        mma3_ss(d, sdesc(A.ae + ao, kAK * 32), sdesc(A.ae_lo + ao, kAK * 32), sdesc(A.eb + bo, 512),
                sdesc(A.eb_lo + bo, 512), id, h > 0);
    }
}

// Every value the sweep of chunk c reads, issuer u's share.  First sweep:
// x ... s of the given position coefficients and psi of the given heading
// coefficients (block 5).  Later: psi of the current heading coefficients
// (with psi'' when res) and, when res, psi of the previous ones.
template <bool PRO, bool RES>
__device__ void issue_values(const LAddr &A, uint32_t tm, int c, int u)
{
    if (u == 0) {
        mma_values(A, tm + kTmE + kQx, 0, 48, c);
    } else if (u == 1) {
        mma_values(A, tm + kTmE + kQy, 2, 48, c);
    } else if (u == 2) {
        mma_values(A, tm + kTmE + kQc, 1, 16, c);
        mma_values(A, tm + kTmE + kQs, 3, 16, c);
    } else if (PRO) {
        mma_values(A, tm + kTmE + kQpsi, 5, 16, c);
    } else {
        mma_values(A, tm + kTmE + kQpsi, 4, RES ? 48 : 16, c);
        if (RES) mma_values(A, tm + kTmE + kQpsio, 5, 16, c);
    }
}

// R over chunk c, issuer u's share (side u >> 1): Pd^T rv + Pdd^T ra + P^T r0
// into the c_pos columns (u even) or P^T r1 into the c_slack columns (u
// odd); the first chunk starts each sum.
__device__ void issue_r(const LAddr &A, uint32_t tm, int c, int qk, int u)
{
    const uint32_t id = idesc_tf32(16), sbo = uint32_t(qk) * 32u;
    const int s = u >> 1, seg0 = (u & 1) ? 3 : 0, seg1 = (u & 1) ? 4 : 3;
    const uint32_t d = tm + kTmR + 32 * s + 16 * (u & 1);
    for (int seg = seg0; seg < seg1; ++seg) {
        const int mat = seg == 0 ? 1 : seg == 1 ? 2 : 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = kChunk * c + 8 * h;
            const uint32_t a = tm + kTmA + 16 * (4 * s + seg) + 8 * h;
            const uint32_t bo = uint32_t(mat * 16 * qk) * 4u + uint32_t(t >> 2) * 128u;
            const bool acc = !(c == 0 && h == 0 && seg == seg0);
            mma3_ts(d, a, a + 128, sdesc(A.rb + bo, sbo), sdesc(A.rb_lo + bo, sbo), id, acc);
        }
    }
}

// P^T delta over chunks [c0, c1); the first chunk starts the sum.
__device__ void issue_ptd(const LAddr &A, uint32_t tm, int c0, int c1, int qk)
{
    const uint32_t id = idesc_tf32(16), sbo = uint32_t(qk) * 32u;
    for (int c = c0; c < c1; ++c)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = kChunk * c + 8 * h;
            const uint32_t a = tm + kTmA + t, bo = uint32_t(t >> 2) * 128u;
            mma3_ts(tm + kTmR, a, a + 128, sdesc(A.rb + bo, sbo), sdesc(A.rb_lo + bo, sbo), id, !(c == 0 && h == 0));
        }
}

// c (issuer 0), s (1), psi (2) and, in the first iteration, psi of the given
// heading coefficients (3) at chunks [g0, g1), 64 columns per chunk.  Returns
// whether anything was issued.
__device__ bool issue_heading_values(const LAddr &A, uint32_t tm, int g0, int g1, bool first, int u)
{
    if (u == 3 && !first) return false;
    const int blk = u == 0 ? 1 : u == 1 ? 3 : u == 2 ? 4 : 5;
    for (int c = g0; c < g1; ++c) mma_values(A, tm + kTmE + 64 * (c - g0) + 16 * u, blk, 16, c);
    return true;
}

// Position-step increment of side u (issuers 0, 1): Minv u (u from tensor
// memory) - MQ xi1 (xi1 from the coefficient operand), columns 32 u + 16 b + k.
__device__ void issue_xi1(const LAddr &A, uint32_t tm, int s)
{
    const uint32_t id = idesc_tf32(32);
    const uint32_t d = tm + kTmE + 32 * s;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const uint32_t a = tm + kTmA + 32 * s + 8 * h;
        mma3_ts(d, a, a + 128, sdesc(A.mi + 256 * h, 1024), sdesc(A.mi_lo + 256 * h, 1024), id, h > 0);
    }
#pragma unroll
    for (int h = 0; h < 3; ++h) {
        const uint32_t ao = uint32_t(6 * s + 2 * h) * 128u;
        mma3_ss(d, sdesc(A.ae + ao, kAK * 32), sdesc(A.ae_lo + ao, kAK * 32), sdesc(A.nq + 256 * h, 768),
                sdesc(A.nq_lo + 256 * h, 768), id, true);
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(smem_u32(bar)) : "memory");
}

// ---------------------------------------------------------- per-thread context

struct Ctx {
    unsigned char *smb;
    LSmem S;
    LAddr A;
    uint64_t *bars;      // [0] constant copy, [1] value products, [2] R products
    uint32_t tm;         // tensor-memory base
    uint32_t tl;         // this warp's lane quadrant
    int warp, lane, qd, sl, i;
    int iss;             // issuer index (lane 0 of warps 12..15), else -1
    uint32_t pe, pr;     // phases of bars[1], bars[2] waited for next
};

__device__ __forceinline__ bool wait_values(Ctx &x)
{
    const bool ok = mbar_wait_bounded(&x.bars[1], x.pe);
    x.pe ^= 1u;
    tc_fence_after();
    return ok;
}

__device__ __forceinline__ bool wait_r(Ctx &x)
{
    const bool ok = mbar_wait_bounded(&x.bars[2], x.pr);
    x.pr ^= 1u;
    tc_fence_after();
    return ok;
}

// Block barrier that also orders tensor-core work and agrees on failure.
__device__ __forceinline__ bool barrier_ok(bool ok)
{
    tc_fence_before();
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// ---------------------------------------------------------- sweep of one pair

// Boundary control point index kk (0..5) -> coefficient index 0, 1, 2, 8, 9, 10.
__device__ __forceinline__ int bnd_k(int kk) { return kk < 3 ? kk : kk + 5; }

struct Vals {
    float2 x, xd, xdd, y, yd, ydd, c, s;
};

// The closed-form steps and the residual rows of steps t0, t0 + 1 (Eq. zeta_2
// - compute_da, in the trig-free projection form), as in the small-tile
// kernel: out = rv, ra, r0, r1 per side.  PRO: g from the given samples r,
// F xi1 from the reference ref.  RES: the step's sums; FIN: the smallest
// squared ellipse distance.  Lanes past the tile's trajectories compute
// finite values that nothing reads and stay out of the near-obstacle box.
template <int M, bool PRO, bool RES, bool FIN>
__device__ __forceinline__ void sweep_pair(const ConstLayout &L, const float *ob, int t0, bool v1, bool row_ok,
                                           const Vals &r, const Vals &ref, float2 psi, float2 psidd, float2 psio,
                                           float rmax, float2 (&out)[8], double (&acc)[3], float &dmn)
{
    const float4 *obs2 = reinterpret_cast<const float4 *>(ob + (L.off_obs2 - L.off_obt)) + (t0 >> 1);
    const float4 *obc2 = reinterpret_cast<const float4 *>(ob + (L.off_obc2 - L.off_obt));
    const int hq = L.qs >> 1, n = L.n;
    float2 pr;
    pr.x = psi.x - kTwoPi * rintf(psi.x * (1.0f / kTwoPi));
    pr.y = psi.y - kTwoPi * rintf(psi.y * (1.0f / kTwoPi));
    const float2 cp = f2(__cosf(pr.x), __cosf(pr.y)), sp = f2(__sinf(pr.x), __sinf(pr.y));
    const float2 cf = PRO ? ref.c : r.c, sf = PRO ? ref.s : r.s;

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
    auto pair = [&](int j) {
        const float4 o = obs2[j * hq];
        const float4 ci = obc2[2 * j], ca = obc2[2 * j + 1];
        const float2 ox = f2(o.x, o.y), oy = f2(o.z, o.w);
        const float2 ia = f2(ci.x, ci.y), ib = f2(ci.z, ci.w), aa = f2(ca.x, ca.y), bb = f2(ca.z, ca.w);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float2 xh = ffma2(X[i], ia, ox);
            const float2 yh = ffma2(Y[i], ib, oy);
            const float2 D = ffma2(xh, xh, ffma2(yh, yh, dup2(kTinyD)));
            const float2 h = f2(fmaxf(rsqrtf(D.x), 1.f) - 1.f, fmaxf(rsqrtf(D.y), 1.f) - 1.f);
            const float2 tx = fmul2(fadd2(xh, dup2(kCoincideT)), h), ty = fmul2(yh, h);  // see kCoincideT
            if (RES) {
                const float2 ex = fmul2(aa, tx), ey = fmul2(bb, ty);
                ax[i] = fadd2(ax[i], ex);
                ay[i] = fadd2(ay[i], ey);
                ee[i] = ffma2(ex, ex, ffma2(ey, ey, ee[i]));
            } else {
                ax[i] = ffma2(aa, tx, ax[i]);
                ay[i] = ffma2(bb, ty, ay[i]);
            }
            if (FIN) {
                dmin.x = fminf(dmin.x, D.x);
                dmin.y = fminf(dmin.y, D.y);
            }
        }
    };
    if (FIN) {
        for (int j = 0; j < n; ++j) pair(j);
    } else {
        // Obstacle j matters only when some circle centre of the warp's steps
        // lies inside its ellipse; every circle centre is within r_max of the
        // robot centre, so the bounding box of the warp's robot centres
        // (both steps) widened by r_max (+ a margin) in the ellipse-scaled
        // frame decides.  One obstacle per lane; the list is warp-uniform.
        const float lx0 = row_ok ? (v1 ? fminf(r.x.x, r.x.y) : r.x.x) : 3.0e38f;
        const float lx1 = row_ok ? (v1 ? fmaxf(r.x.x, r.x.y) : r.x.x) : -3.0e38f;
        const float ly0 = row_ok ? (v1 ? fminf(r.y.x, r.y.y) : r.y.x) : 3.0e38f;
        const float ly1 = row_ok ? (v1 ? fmaxf(r.y.x, r.y.y) : r.y.x) : -3.0e38f;
        const float bx0 = warp_min(lx0), bx1 = warp_max(lx1), by0 = warp_min(ly0), by1 = warp_max(ly1);
        const int lane = threadIdx.x & 31;
        auto near = [&](int j) {
            if (j >= n) return false;
            const float4 o = obs2[j * hq];
            const float4 ci = obc2[2 * j];
            const float ox0 = v1 ? fminf(o.x, o.y) : o.x, ox1 = v1 ? fmaxf(o.x, o.y) : o.x;
            const float oy0 = v1 ? fminf(o.z, o.w) : o.z, oy1 = v1 ? fmaxf(o.z, o.w) : o.z;
            const float ulo = fmaf(bx0, ci.x, ox0), uhi = fmaf(bx1, ci.x, ox1);
            const float vlo = fmaf(by0, ci.z, oy0), vhi = fmaf(by1, ci.z, oy1);
            const float du = fmaxf(0.f, fmaxf(ulo, -uhi)), dv = fmaxf(0.f, fmaxf(vlo, -vhi));
            const float reach = fmaf(rmax + kBoxMargin, fmaxf(ci.x, ci.z), 1.f);
            return fmaf(du, du, dv * dv) < reach * reach;
        };
        const unsigned list0 = __ballot_sync(0xffffffffu, near(lane));
        const unsigned list1 = n > 32 ? __ballot_sync(0xffffffffu, near(lane + 32)) : 0u;
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
            unsigned nl = blk == 0 ? list0 : list1;
            while (nl) {
                const int jj = __ffs(nl) - 1;
                nl &= nl - 1u;
                pair(32 * blk + jj);
            }
        }
    }
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
            const float2 dx = fmul2(ri, dcx), dy = fmul2(ri, dsy);
            const float2 sq = fmul2(fn, ffma2(dx, dx, fmul2(dy, dy)));
            const float2 cr = fmul2(dup2(2.f), ffma2(dx, ax[i], fmul2(dy, ay[i])));
            rob = fadd2(rob, fadd2(fadd2(sq, cr), ee[i]));
        }
    }
    const float2 svm = f2(sv.x - 1.f, sv.y - 1.f), sam = f2(sa.x - 1.f, sa.y - 1.f);
    out[0] = PRO ? ffma2(r.xd, svm, fsub2(r.xd, ref.xd)) : fmul2(r.xd, svm);
    out[1] = PRO ? ffma2(r.xdd, sam, fsub2(r.xdd, ref.xdd)) : fmul2(r.xdd, sam);
    out[2] = r0x;
    out[3] = fadd2(r1x, dcx);
    out[4] = PRO ? ffma2(r.yd, svm, fsub2(r.yd, ref.yd)) : fmul2(r.yd, svm);
    out[5] = PRO ? ffma2(r.ydd, sam, fsub2(r.ydd, ref.ydd)) : fmul2(r.ydd, sam);
    out[6] = r0y;
    out[7] = fadd2(r1y, dsy);
    if (!v1) {
#pragma unroll
        for (int g = 0; g < 8; ++g) out[g].y = 0.f;
    }
    if (RES && row_ok) {
        const float2 bnd = ffma2(fmul2(v2, svm), svm, fmul2(fmul2(a2, sam), sam));
        const float2 sl = ffma2(dcx, dcx, fmul2(dsy, dsy));
        const float2 e0 = fadd2(fadd2(bnd, rob), sl);
        // psi_t = psi_prev + wrap(atan2(s, c) - psi_prev), psi_prev the
        // heading before this iteration's heading step
        const float ptx = psio.x + wrap_pi(atan2_heading(r.s.x, r.c.x) - psio.x);
        const float pty = psio.y + wrap_pi(atan2_heading(r.s.y, r.c.y) - psio.y);
        const float2 dp = fsub2(psi, f2(ptx, pty));
        const float2 e1 = fmul2(dp, dp);
        const float2 e2 = ffma2(r.xdd, r.xdd, ffma2(r.ydd, r.ydd, fmul2(psidd, psidd)));
        acc[0] += double(e0.x) + (v1 ? double(e0.y) : 0.0);
        acc[1] += double(e1.x) + (v1 ? double(e1.y) : 0.0);
        acc[2] += double(e2.x) + (v1 ? double(e2.y) : 0.0);
    }
    if (FIN && row_ok) dmn = fminf(dmn, v1 ? fminf(dmin.x, dmin.y) : dmin.x);
}

// ---------------------------------------------------------- phases

// One sweep over the horizon in chunks: the values of chunk c on the tensor
// cores (issued while chunk c - 1 is swept), the closed-form steps on the
// workers, R of chunk c on the tensor cores.
template <int M, bool PRO, bool RES, bool FIN>
__device__ bool sweep(const FusedProblem &p, Ctx &x, int count, double (&acc)[3], float &dmn)
{
    const ConstLayout &L = p.L;
    const float *ob = reinterpret_cast<const float *>(x.smb + x.S.ob);
    const bool row_ok = x.i < count;
    float rmax = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) rmax = fmaxf(rmax, fabsf(L.r[i]));
    if (x.iss >= 0) {
        tc_fence_after();
        issue_values<PRO, RES>(x.A, x.tm, 0, x.iss);
        tc_commit(&x.bars[1]);
    }
    for (int c = 0; c < x.S.qc; ++c) {
        bool ok = true;
        float4 v[11];
        {
            ok = wait_values(x);
            const uint32_t a = x.tl + kTmE + 4 * x.sl;
            tm_ld4(a + kQx, v[0]);
            tm_ld4(a + kQxd, v[1]);
            tm_ld4(a + kQxdd, v[2]);
            tm_ld4(a + kQy, v[3]);
            tm_ld4(a + kQyd, v[4]);
            tm_ld4(a + kQydd, v[5]);
            tm_ld4(a + kQc, v[6]);
            tm_ld4(a + kQs, v[7]);
            tm_ld4(a + kQpsi, v[8]);
            if (RES) {
                tm_ld4(a + kQpsidd, v[9]);
                tm_ld4(a + kQpsio, v[10]);
            }
            tm_wait_ld();
#pragma unroll
            for (int e = 0; e < 9; ++e) hold(v[e]);
            if (RES) {
                hold(v[9]);
                hold(v[10]);
            }
        }
        if (!barrier_ok(ok)) return false;
        if (x.iss >= 0 && c + 1 < x.S.qc) {
            tc_fence_after();
            issue_values<PRO, RES>(x.A, x.tm, c + 1, x.iss);
            tc_commit(&x.bars[1]);
        }
        {
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int e = 2 * pp, j = 4 * x.sl + e, t0 = kChunk * c + j;
                float2 out[8];
#pragma unroll
                for (int g = 0; g < 8; ++g) out[g] = f2(0.f, 0.f);
                if (t0 < L.q) {  // the same for the whole warp
                    const bool v1 = t0 + 1 < L.q;
                    Vals r;
                    r.x = pick(v[0], e);
                    r.xd = pick(v[1], e);
                    r.xdd = pick(v[2], e);
                    r.y = pick(v[3], e);
                    r.yd = pick(v[4], e);
                    r.ydd = pick(v[5], e);
                    r.c = pick(v[6], e);
                    r.s = pick(v[7], e);
                    const float2 psi = pick(v[8], e);
                    const float2 psidd = RES ? pick(v[9], e) : f2(0.f, 0.f);
                    const float2 psio = RES ? pick(v[10], e) : f2(0.f, 0.f);
                    Vals ref = r;
                    if (PRO) {
                        // the reference differs from the given coefficients
                        // only at the boundary control points
                        const float *del = reinterpret_cast<const float *>(x.smb + x.S.sums) + x.i * 25;
                        const float *pr = p.cblob + L.off_prow;
                        const int t1 = v1 ? t0 + 1 : t0;
#pragma unroll
                        for (int kk = 0; kk < 6; ++kk) {
                            const int k = bnd_k(kk);
                            const float2 P = f2(pr[t0 * 12 + k], v1 ? pr[t1 * 12 + k] : 0.f);
                            const float2 Pd = f2(pr[(L.q + t0) * 12 + k], v1 ? pr[(L.q + t1) * 12 + k] : 0.f);
                            const float2 Pdd = f2(pr[(2 * L.q + t0) * 12 + k], v1 ? pr[(2 * L.q + t1) * 12 + k] : 0.f);
                            const float2 d0 = dup2(del[kk]), d1 = dup2(del[6 + kk]);
                            const float2 d2 = dup2(del[12 + kk]), d3 = dup2(del[18 + kk]);
                            ref.x = ffma2(P, d0, ref.x);
                            ref.xd = ffma2(Pd, d0, ref.xd);
                            ref.xdd = ffma2(Pdd, d0, ref.xdd);
                            ref.c = ffma2(P, d1, ref.c);
                            ref.y = ffma2(P, d2, ref.y);
                            ref.yd = ffma2(Pd, d2, ref.yd);
                            ref.ydd = ffma2(Pdd, d2, ref.ydd);
                            ref.s = ffma2(P, d3, ref.s);
                        }
                    }
                    sweep_pair<M, PRO, RES, FIN>(L, ob, t0, v1, row_ok, r, ref, psi, psidd, psio, rmax, out, acc,
                                                 dmn);
                }
                // the previous chunk's R products read the residual columns
                if (pp == 0 && c > 0) ok = wait_r(x) && ok;
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    float h0, l0, h1, l1;
                    split(out[g].x, h0, l0);
                    split(out[g].y, h1, l1);
                    tm_st2(x.tl + kTmA + 16 * g + j, h0, h1);
                    tm_st2(x.tl + kTmA + 128 + 16 * g + j, l0, l1);
                }
            }
            tm_wait_st();
        }
        if (!barrier_ok(ok)) return false;
        if (x.iss >= 0) {
            tc_fence_after();
            issue_r(x.A, x.tm, c, x.S.qk, x.iss);
            tc_commit(&x.bars[2]);
        }
    }
    return true;
}

// XI1: the multiplier update and u = lam + coef R of the finished sweep
//   first: lam' = lam,          u = lam + rho R
//   later: lam' = lam + rho R,  u = lam + 2 rho R
//   post (no solve): lam' = lam + rho R
// then xi1' = xi1 + Minv u - MQ xi1 on the tensor cores.  Thread (trajectory
// i, slice sl) owns coefficient block sl (c_x, c_c, c_y, c_s) and its lambda.
__device__ bool phase_xi1(const FusedProblem &p, Ctx &x, bool first, bool solve, float (&lam)[12])
{
    const int s = x.sl >> 1, b = x.sl & 1;
    bool ok = true;
    {
        ok = wait_r(x);
        float R[16];
        tm_ld16(x.tl + kTmR + 32 * s + 16 * b, R);
        tm_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) hold(R[k]);
        const float rho = p.L.rho, coef = first ? rho : 2.f * rho;
        float uh[16], ul[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float u = 0.f;
            if (k < NV) {
                u = fmaf(coef, R[k], lam[k]);
                if (!first) lam[k] = fmaf(rho, R[k], lam[k]);
            }
            split(u, uh[k], ul[k]);
        }
        if (solve) {
            tm_st16(x.tl + kTmA + 32 * s + 16 * b, uh);
            tm_st16(x.tl + kTmA + 128 + 32 * s + 16 * b, ul);
            tm_wait_st();
        }
    }
    if (!barrier_ok(ok)) return false;
    if (!solve) return true;
    if (x.iss >= 2) {
        mbar_arrive(&x.bars[1]);
    } else if (x.iss >= 0) {
        tc_fence_after();
        issue_xi1(x.A, x.tm, x.iss);
        tc_commit(&x.bars[1]);
    }
    {
        ok = wait_values(x);
        float D[16];
        tm_ld16(x.tl + kTmE + 32 * s + 16 * b, D);
        tm_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) hold(D[k]);
        float c[12];
        ae_get(x.smb, x.S, x.i, 12 * x.sl, c);
#pragma unroll
        for (int k = 0; k < NV; ++k) c[k] += D[k];
        c[11] = 0.f;
        ae_put(x.smb, x.S, x.i, 12 * x.sl, c);
    }
    proxy_fence();
    return barrier_ok(ok);
}

// EVAL: psi_t = psi_prev + wrap(atan2(s, c) - psi_prev) and delta = psi_t -
// P xi2 at every step, three chunks at a time, then P^T delta.
__device__ bool phase_heading_target(const FusedProblem &p, Ctx &x, bool first)
{
    const int qc = x.S.qc, q = p.L.q;
    for (int g0 = 0; g0 < qc; g0 += kGroup) {
        const int g1 = min(qc, g0 + kGroup);
        bool ok = true;
        if (x.iss >= 0) {
            tc_fence_after();
            bool any = issue_heading_values(x.A, x.tm, g0, g1, first, x.iss);
            if (x.iss == 3 && g0 > 0) {
                issue_ptd(x.A, x.tm, g0 - kGroup, g0, x.S.qk);
                any = true;
            }
            if (any) tc_commit(&x.bars[1]);
            else mbar_arrive(&x.bars[1]);
        }
        {
            ok = wait_values(x);
            for (int c = g0; c < g1; ++c) {
                const uint32_t a = x.tl + kTmE + 64 * (c - g0) + 4 * x.sl;
                float4 vc, vs, vp, vq;
                tm_ld4(a, vc);
                tm_ld4(a + 16, vs);
                tm_ld4(a + 32, vp);
                if (first) tm_ld4(a + 48, vq);
                tm_wait_ld();
                hold(vc);
                hold(vs);
                hold(vp);
                if (first) hold(vq);
                else vq = vp;
                float dh[4], dl[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int t = kChunk * c + 4 * x.sl + e;
                    const float pv = comp(vq, e), pc = comp(vp, e);
                    const float pt = pv + wrap_pi(atan2_heading(comp(vs, e), comp(vc, e)) - pv);
                    split(t < q ? pt - pc : 0.f, dh[e], dl[e]);
                }
                tm_st4(x.tl + kTmA + kChunk * c + 4 * x.sl, dh);
                tm_st4(x.tl + kTmA + 128 + kChunk * c + 4 * x.sl, dl);
            }
            tm_wait_st();
        }
        if (!barrier_ok(ok)) return false;
    }
    if (x.iss == 3) {
        tc_fence_after();
        issue_ptd(x.A, x.tm, ((qc - 1) / kGroup) * kGroup, qc, x.S.qk);
        tc_commit(&x.bars[1]);
    } else if (x.iss >= 0) {
        mbar_arrive(&x.bars[1]);
    }
    return true;
}

// PSI: the heading step of Eq. compute_convex_surrogate in increment form,
//   xi2' = xi2 + Mpsi (lam_psi + rho P^T delta) - Mpsi H xi2,
// then lam_psi' = lam_psi - sign rho_psi (P^T P dxi2 - P^T delta)
// (Eq. update_lambda_psi), one thread (slice 0) per trajectory.  Block 5 of
// the coefficient operand keeps the heading coefficients before the step
// (in the first iteration it keeps the given ones).
__device__ bool phase_psi(const FusedProblem &p, Ctx &x, bool first)
{
    const ConstLayout &L = p.L;
    bool ok = true;
    {
        ok = wait_values(x);
        if (x.sl == 0) {
            float ptd[16];
            tm_ld16(x.tl + kTmR, ptd);
            tm_wait_ld();
#pragma unroll
            for (int k = 0; k < 16; ++k) hold(ptd[k]);
            float x2[12];
            ae_get(x.smb, x.S, x.i, 48, x2);
            float *lp = reinterpret_cast<float *>(x.smb + x.S.lps) + x.i * 13;
            const float *ps = reinterpret_cast<const float *>(x.smb + x.S.ps);
            float lv[NV], d[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) lv[k] = lp[k];
#pragma unroll
            for (int o = 0; o < NV; ++o) {
                float b0 = 0.f, b1 = 0.f;
#pragma unroll
                for (int c = 0; c < NV; ++c) {
                    b0 = fmaf(ps[c * 12 + o], fmaf(L.rho, ptd[c], lv[c]), b0);
                    b1 = fmaf(ps[NV * 12 + c * 12 + o], x2[c], b1);
                }
                d[o] = b0 - b1;
            }
            float xn[12];
#pragma unroll
            for (int o = 0; o < NV; ++o) xn[o] = x2[o] + d[o];
            xn[11] = 0.f;
            ae_put(x.smb, x.S, x.i, 48, xn);
            if (!first) ae_put(x.smb, x.S, x.i, 60, x2);
#pragma unroll
            for (int o = 0; o < NV; ++o) {
                float a = 0.f;
#pragma unroll
                for (int c = 0; c < NV; ++c) a = fmaf(ps[2 * NV * 12 + c * 12 + o], d[c], a);
                lp[o] = lv[o] - L.psi_sign * L.rho_psi * (a - ptd[o]);
            }
        }
    }
    proxy_fence();
    return barrier_ok(ok);
}

// All iterations of the AM loop for one tile of 128 trajectories.
template <int M>
__device__ bool run_tile(const FusedProblem &p, Ctx &x, int tile)
{
    const ConstLayout &L = p.L;
    const int first = tile * kLT, count = min(kLT, p.B - first);
    const bool row_ok = x.i < count;
    float lam[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) lam[k] = 0.f;
    const float *ends = p.cblob + L.off_ends;
#ifdef AM_DEBUG_BOUNDS
    if (threadIdx.x == 0) g_loob = 0;
    __syncthreads();
#endif
    // State of the tile: the given coefficients into blocks 0..3 (and c_psi
    // into block 5, its reference into block 4), lambda into registers,
    // lambda_psi into shared memory, the boundary differences of the
    // reference for the first sweep.
    {
        const bool in = row_ok && AM_LBOUND(first >= 0 && first + count <= p.B);
        const float *st = p.state + size_t(first + (in ? x.i : 0)) * STATE;
        const int blk = x.sl;
        float v[12];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v[k] = in ? st[NV * blk + k] : 0.f;
            lam[k] = in ? st[55 + NV * blk + k] : 0.f;
        }
        v[11] = 0.f;
        ae_put(x.smb, x.S, x.i, 12 * blk, v);
        const bool has_bc = blk == 0 || blk == 2 || L.cs_boundary;
        float *del = reinterpret_cast<float *>(x.smb + x.S.sums) + x.i * 25 + 6 * blk;
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
            const int k = bnd_k(kk);
            del[kk] = has_bc ? ends[blk * 8 + (k <= 2 ? k : k - 5)] - v[k] : 0.f;
        }
        if (x.sl == 0) {
            float w[12], wr[12];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                w[k] = in ? st[44 + k] : 0.f;
                wr[k] = k <= 2 ? ends[32 + k] : k >= 8 ? ends[32 + k - 5] : w[k];
            }
            w[11] = wr[11] = 0.f;
            ae_put(x.smb, x.S, x.i, 60, w);
            ae_put(x.smb, x.S, x.i, 48, wr);
        }
        if (x.sl == 1) {
            float *lp = reinterpret_cast<float *>(x.smb + x.S.lps) + x.i * 13;
#pragma unroll
            for (int k = 0; k < NV; ++k) lp[k] = in ? st[99 + k] : 0.f;
        }
    }
    proxy_fence();
    __syncthreads();

    double acc[3] = {0.0, 0.0, 0.0};
    float dmn = 3.0e38f;
    // Step 1 of Sec. III-D: the closed-form steps and g from the initial
    // samples, the residual against the reference.
    if (!sweep<M, true, false, false>(p, x, count, acc, dmn)) return false;
    // The reference becomes the current position coefficients.
    {
        const int blk = x.sl;
        const bool has_bc = blk == 0 || blk == 2 || L.cs_boundary;
        if (has_bc) {
            float v[12];
            ae_get(x.smb, x.S, x.i, 12 * blk, v);
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) {
                const int k = bnd_k(kk);
                v[k] = ends[blk * 8 + (k <= 2 ? k : k - 5)];
            }
            v[11] = 0.f;
            ae_put(x.smb, x.S, x.i, 12 * blk, v);
        }
    }
    proxy_fence();

    for (int k = 0; k < p.iters; ++k) {
        if (!phase_xi1(p, x, k == 0, true, lam)) return false;
        if (!phase_heading_target(p, x, k == 0)) return false;
        if (!phase_psi(p, x, k == 0)) return false;
        const bool ok = k == p.iters - 1 ? sweep<M, false, true, true>(p, x, count, acc, dmn)
                                         : sweep<M, false, false, false>(p, x, count, acc, dmn);
        if (!ok) return false;
    }
    // Multipliers of the last iteration; state and results out.
    if (!phase_xi1(p, x, false, false, lam)) return false;
    double *sums = reinterpret_cast<double *>(x.smb + x.S.sums);
    float *mins = reinterpret_cast<float *>(x.smb + x.S.sums + kLT * 4 * 3 * 8);
    {
        if (row_ok && AM_LBOUND(first + count <= p.B)) {
            float *st = p.state + size_t(first + x.i) * STATE;
            float v[12];
            ae_get(x.smb, x.S, x.i, 12 * x.sl, v);
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                st[NV * x.sl + k] = v[k];
                st[55 + NV * x.sl + k] = lam[k];
            }
            if (x.sl == 0) {
                ae_get(x.smb, x.S, x.i, 48, v);
#pragma unroll
                for (int k = 0; k < NV; ++k) st[44 + k] = v[k];
            }
            if (x.sl == 1) {
                const float *lp = reinterpret_cast<const float *>(x.smb + x.S.lps) + x.i * 13;
#pragma unroll
                for (int k = 0; k < NV; ++k) st[99 + k] = lp[k];
            }
        }
#pragma unroll
        for (int w = 0; w < 3; ++w) sums[(x.i * 4 + x.sl) * 3 + w] = acc[w];
        mins[x.i * 4 + x.sl] = dmn;
    }
    __syncthreads();
    if (x.sl == 0 && row_ok) {
        double a[3] = {0.0, 0.0, 0.0};
        float mn = 3.0e38f;
        for (int s = 0; s < 4; ++s) {
#pragma unroll
            for (int w = 0; w < 3; ++w) a[w] += sums[(x.i * 4 + s) * 3 + w];
            mn = fminf(mn, mins[x.i * 4 + s]);
        }
        const int traj = first + x.i;
        p.res[traj] = float(sqrt(a[0]));
        p.res_psi[traj] = float(sqrt(a[1]));
        p.cost[traj] = float(a[2]);
        p.mind[traj] = sqrtf(mn);
    }
    __syncthreads();
#ifdef AM_DEBUG_BOUNDS
    if (threadIdx.x == 0 && g_loob) atomicOr(p.err, 2);
#endif
    return true;
}

template <int M>
__global__ void __launch_bounds__(kLThreads, 1) am_large_kernel(FusedProblem p)
{
    extern __shared__ __align__(1024) unsigned char smb[];
    Ctx x;
    x.smb = smb;
    x.S = lsmem_layout(p.L);
    x.A = laddr(smb, x.S);
    x.bars = reinterpret_cast<uint64_t *>(smb + x.S.bar);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smb + x.S.bar + 32);
    x.warp = threadIdx.x >> 5;
    x.lane = threadIdx.x & 31;
    x.qd = x.warp & 3;
    x.sl = x.warp >> 2;
    x.i = 32 * x.qd + x.lane;
    x.iss = (x.sl == 3 && x.lane == 0) ? x.qd : -1;
    x.pe = x.pr = 0u;
    if (x.warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(slot)), "r"(kTmCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(&x.bars[0])));
        for (int b = 1; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(&x.bars[b])), "r"(kIssuers));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    x.tm = *reinterpret_cast<volatile uint32_t *>(slot);
    x.tl = x.tm + (uint32_t(32 * x.qd) << 16);
    bool ok = lstage(p, smb, x.S, &x.bars[0]);
    for (int tile = blockIdx.x; ok && tile < p.ntiles; tile += gridDim.x) ok = run_tile<M>(p, x, tile);
    // every tensor-core operation has completed (every thread waited for each
    // commit) unless a wait ran out; the allocating warp frees the columns
    tc_fence_before();
    __syncthreads();
    if (x.warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(x.tm), "r"(kTmCols) : "memory");
    }
    if (!ok && threadIdx.x == 0) atomicExch(p.err, 1);
}

std::mutex g_large_mu;

template <int M>
int launch_large_m(const FusedProblem &p, size_t smem, int grid, cudaStream_t st)
{
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_large_mu);
        if (attr_dev != dev) {
            if (cudaFuncSetAttribute(am_large_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(kFusedSmemMax)) != cudaSuccess)
                return -2;
            attr_dev = dev;
        }
    }
    am_large_kernel<M><<<grid, kLThreads, smem, st>>>(p);
    return 0;
}

}  // namespace

size_t large_smem_bytes(const ConstLayout &L) { return size_t(lsmem_layout(L).total); }

int large_supported(const ConstLayout &L, bool hist)
{
    if (L.precision != 0 || L.alpha_mode != 0 || hist) return 0;
    if (L.q < 2 || L.q > kLMaxQ || L.m < 1 || L.m > MAXM || L.n > 64) return 0;
    return large_smem_bytes(L) <= kFusedSmemMax ? 1 : 0;
}

int launch_large(const SolveArgs &a, void *stream, int *launches)
{
    const ConstLayout &L = a.L;
    if (!large_supported(L, a.hist != nullptr)) return -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return -2;
    FusedProblem p;
    p.cblob = a.cblob;
    p.L = L;
    p.B = a.B;
    p.iters = a.iters;
    p.T = kLT;
    p.ntiles = (a.B + kLT - 1) / kLT;
    p.state = a.state;
    p.res = a.res;
    p.res_psi = a.res_psi;
    p.cost = a.cost;
    p.mind = a.mind;
    p.hist = nullptr;
    p.err = a.err;
    const int grid = p.ntiles < sms ? p.ntiles : sms;
    const size_t smem = large_smem_bytes(L);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = -1;
    switch (L.m) {
    case 1: rc = launch_large_m<1>(p, smem, grid, st); break;
    case 2: rc = launch_large_m<2>(p, smem, grid, st); break;
    case 3: rc = launch_large_m<3>(p, smem, grid, st); break;
    case 4: rc = launch_large_m<4>(p, smem, grid, st); break;
    default: return -1;
    }
    if (rc) return rc;
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam
