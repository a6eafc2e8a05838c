// Small kernels around the AM loop: initial state, obstacle preparation and
// the best-trajectory selection.
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>

#include "am_internal.h"
#include "am_rng.cuh"

namespace trajam {
namespace {

// state = (xi1 = (c_x, c_c, c_y, c_s), xi2 = c_psi, lambda, lambda_psi) from B x 3 x 11
// initial coefficients and optional B x 55 warm multipliers.  The first xi1
// step does not depend on the slack coefficients (Sec. III-D, step 2 uses only
// g), so they start at cos / sin of the heading control points: a reference
// close to the slacks the first step will produce, which keeps the
// incremental position update of the kernels well scaled.
// With out (4 B floats: res, res_psi, cost, mind) and err, the same launch
// clears the results and the status word.
__global__ void init_state_kernel(float *state, const float *init, const float *warm, int B, float *out,
                                  int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (out && i < 4 * B) out[i] = 0.f;  // 4 B < B * STATE threads
    if (err && i == 0) *err = 0;
    if (i >= B * STATE) return;
    const int l = i / STATE, e = i - STATE * l;
    float v = 0.f;
    if (e < 11) v = init[l * 33 + e];
    else if (e < 22) v = cosf(init[l * 33 + 22 + (e - 11)]);
    else if (e < 33) v = init[l * 33 + 11 + (e - 22)];
    else if (e < 44) v = sinf(init[l * 33 + 22 + (e - 33)]);
    else if (e < 55) v = init[l * 33 + 22 + (e - 44)];
    else if (warm) v = warm[l * 55 + (e - 55)];
    state[i] = v;
}

// Batch re-draw (am_resample): one thread per trajectory.  Ten standard
// normals from five Box-Muller pairs (draws 2p, 2p + 1), z_x = 0..4 and
// z_y = 5..9; trajectory 0 takes none.  Control points 3..7 of c_x, c_y are the
// straight line plus sigma L z; the heading is the straight line between its
// boundary values and the slacks its cos, sin (as init_state_kernel).  The
// multipliers (state entries 55..109) are left as they are.
__global__ void resample_kernel(float *state, ResampleArgs a)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.B) return;
    double z[10];
    for (int p = 0; p < 5; ++p) {
        z[2 * p] = z[2 * p + 1] = 0.0;
        if (l > 0) normal_pair(a.seed, (unsigned long long)l, p, z[2 * p], z[2 * p + 1]);
    }
    float *st = state + (size_t)l * STATE;
    for (int k = 0; k < NV; ++k) {
        const float w = fminf(fmaxf((k - 2) / 6.f, 0.f), 1.f);
        float cx = fmaf(a.line[1] - a.line[0], w, a.line[0]);
        float cy = fmaf(a.line[3] - a.line[2], w, a.line[2]);
        const float cp = fmaf(a.line[5] - a.line[4], w, a.line[4]);
        if (k >= 3 && k <= 7) {
            const int i = k - 3;
            double dx = 0.0, dy = 0.0;
            for (int j = 0; j <= i; ++j) {
                dx += double(a.Lc[i * 5 + j]) * z[j];
                dy += double(a.Lc[i * 5 + j]) * z[5 + j];
            }
            cx += a.sigma * float(dx);
            cy += a.sigma * float(dy);
        }
        st[k] = cx;
        st[11 + k] = cosf(cp);
        st[22 + k] = cy;
        st[33 + k] = sinf(cp);
        st[44 + k] = cp;
    }
}

// Re-timing (am_shift): one thread per (trajectory, polynomial); the five
// polynomials of a trajectory are state entries 0, 11, 22, 33, 44 on.
__global__ void shift_kernel(float *state, ShiftArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.B * 5) return;
    float *c = state + (size_t)(i / 5) * STATE + 11 * (i % 5);
    float in[NV];
    for (int k = 0; k < NV; ++k) in[k] = c[k];
    for (int k = 0; k < NV; ++k) {
        float v = 0.f;
        for (int j = 0; j < NV; ++j) v = fmaf(a.S[k * NV + j], in[j], v);
        c[k] = v;
    }
}

// Multiplier decay between re-plans: state entries 55..109 of every trajectory.
__global__ void scale_multipliers_kernel(float *state, int B, float factor)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 55) return;
    float &v = state[(size_t)(i / 55) * STATE + 55 + i % 55];
    v *= factor;
}

// Obstacle sections of the constant block: centre tracks in ellipse-scaled
// coordinates (x_j(t)/a_j, y_j(t)/b_j) and per-obstacle (1/a_j, 1/b_j, a_j, b_j),
// with the semi-axes inflated by the robot circle radius.  The same values in
// the fused kernel's paired form: per pair of steps (t, t + 1) the negated
// scaled centre coordinates, and every per-obstacle constant twice, so that
// one 128-bit load gives the operands of paired FP32 instructions.
__global__ void prep_obstacles_kernel(float *cblob, ConstLayout L, const float *xo, const float *yo,
                                      const float *a, const float *b, float r_c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L.n * L.q) {
        const int j = i / L.q, t = i - L.q * j;
        const float aj = a[j] + r_c, bj = b[j] + r_c;
        float2 *obs = reinterpret_cast<float2 *>(cblob + L.off_obs);
        const float u = xo[i] / aj, v = yo[i] / bj;
        obs[j * L.qs + t] = make_float2(u, v);
        float *o2 = cblob + L.off_obs2 + j * 2 * L.qs + 4 * (t >> 1) + (t & 1);
        o2[0] = -u;
        o2[2] = -v;
    }
    if (i < L.n) {
        const float aj = a[i] + r_c, bj = b[i] + r_c;
        const float ia = 1.f / aj, ib = 1.f / bj;
        reinterpret_cast<float4 *>(cblob + L.off_obc)[i] = make_float4(ia, ib, aj, bj);
        float4 *c2 = reinterpret_cast<float4 *>(cblob + L.off_obc2) + 2 * i;
        c2[0] = make_float4(ia, ia, ib, ib);
        c2[1] = make_float4(aj, aj, bj, bj);
        // Every circle centre lies within r_max max(1/a, 1/b) of the robot
        // centre in the ellipse-scaled frame; a centre at squared distance
        // above this threshold (with a relative margin for rounding) has every
        // circle outside the ellipse, and keeps that property while it moves
        // by at most kNearMargin (m).
        float rmax = 0.f;
        for (int k = 0; k < L.m; ++k) rmax = fmaxf(rmax, fabsf(L.r[k]));
        const float reach = fmaf(rmax + kNearMargin, fmaxf(1.f / aj, 1.f / bj), 1.f);
        cblob[L.off_obt + i] = reach * reach * (1.f + 1e-4f) + 1e-6f;
    }
}

struct Key {
    int coll;
    float cost;
    int idx;
};

__device__ __forceinline__ bool better(const Key &a, const Key &b)
{
    if (a.coll != b.coll) return a.coll < b.coll;
    if (a.cost != b.cost) return a.cost < b.cost;
    return a.idx < b.idx;
}

// Lexicographic minimum over the batch of (collides, cost, index), where a
// trajectory collides when its smallest ellipse distance is below 0.99; a
// non-finite cost ranks last.  With select = 1, colliding trajectories rank
// by their smallest distance, largest first, instead of by cost.  Writes
// {index, cost, residual, c_x, c_y, c_psi}; the whole block takes part, out
// gets 36 floats.
__device__ void select_best(int select, const float *state, const float *cost, const float *res,
                            const float *mind, int B, float *out, Key *sk)
{
    Key best{2, FLT_MAX, 0x7fffffff};
    for (int l = threadIdx.x; l < B; l += blockDim.x) {
        float c = cost[l];
        const bool coll = mind[l] < 0.99f;
        const float v = coll && select == 1 ? -mind[l] : c;
        Key k{coll ? 1 : 0, isfinite(v) ? v : FLT_MAX, l};
        if (!isfinite(c)) k.coll = 2;
        if (better(k, best)) best = k;
    }
    sk[threadIdx.x] = best;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s && better(sk[threadIdx.x + s], sk[threadIdx.x]))
            sk[threadIdx.x] = sk[threadIdx.x + s];
        __syncthreads();
    }
    const Key w = sk[0];
    if (w.idx >= B) return;
    const float *st = state + (size_t)w.idx * STATE;
    if (threadIdx.x == 0) {
        out[0] = float(w.idx);
        out[1] = cost[w.idx];
        out[2] = res[w.idx];
    }
    if (threadIdx.x < 33) {
        const int e = threadIdx.x;
        out[3 + e] = e < 11 ? st[e] : e < 22 ? st[22 + (e - 11)] : st[44 + (e - 22)];
    }
}

__global__ void argmin_kernel(int select, const float *state, const float *cost, const float *res,
                              const float *mind, int B, float *out)
{
    __shared__ Key sk[1024];
    select_best(select, state, cost, res, mind, B, out, sk);
}

__global__ void group_argmin_kernel(const FusedProblem *probs, const int *list, float *out)
{
    __shared__ Key sk[1024];
    const FusedProblem &p = probs[list[blockIdx.x]];
    select_best(p.L.select, p.state, p.cost, p.res, p.mind, p.B, out + 36 * blockIdx.x, sk);
}

}  // namespace

int raise_smem_limit(const void *kernel, size_t smem)
{
    // the current limit is read back each time (a device reset clears it);
    // the lock keeps two threads from lowering each other's setting
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return int(e);
    if (smem <= size_t(fa.maxDynamicSharedSizeBytes)) return 0;
    return int(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
}

int launch_init_state(float *state, const float *init, const float *warm, int B, void *stream,
                      int *launches, float *out, int *err)
{
    const int n = B * STATE;
    init_state_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(state, init,
                                                                                      warm, B, out, err);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_resample(float *state, const ResampleArgs &a, void *stream, int *launches)
{
    if (a.B < 1) return 0;
    resample_kernel<<<(a.B + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(state, a);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_shift(float *state, const ShiftArgs &a, void *stream, int *launches)
{
    if (a.B < 1) return 0;
    const int n = 5 * a.B;
    shift_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(state, a);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_scale_multipliers(float *state, int B, float factor, void *stream, int *launches)
{
    if (B < 1) return 0;
    const int n = 55 * B;
    scale_multipliers_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(state, B, factor);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_prep_obstacles(float *cblob, const ConstLayout &L, const float *xo, const float *yo,
                          const float *a, const float *b, float r_c, void *stream, int *launches)
{
    const int n = L.n * L.q > L.n ? L.n * L.q : L.n;
    if (n == 0) return 0;
    prep_obstacles_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        cblob, L, xo, yo, a, b, r_c);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_group_argmin(const FusedProblem *d_probs, const int *d_list, int count, float *d_out,
                        void *stream, int *launches)
{
    if (count < 1) return 0;
    group_argmin_kernel<<<count, 1024, 0, static_cast<cudaStream_t>(stream)>>>(d_probs, d_list, d_out);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_argmin(int select, const float *state, const float *cost, const float *res, const float *mind,
                  int B, float *best_out, void *stream, int *launches)
{
    argmin_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(select, state, cost, res, mind, B,
                                                                     best_out);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam
