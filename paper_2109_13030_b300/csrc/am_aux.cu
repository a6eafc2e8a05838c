// Small kernels around the AM loop: initial state, obstacle preparation and
// the best-trajectory selection.
#include <cuda_runtime.h>

#include <cfloat>

#include "am_internal.h"

namespace trajam {
namespace {

// state = (xi1 = (c_x, c_c, c_y, c_s), xi2 = c_psi, lambda, lambda_psi) from B x 3 x 11
// initial coefficients and optional B x 55 warm multipliers.  The first xi1
// step does not depend on the slack coefficients (Sec. III-D, step 2 uses only
// g), so they start at cos / sin of the heading control points: a reference
// close to the slacks the first step will produce, which keeps the
// incremental position update of the kernels well scaled.
__global__ void init_state_kernel(float *state, const float *init, const float *warm, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
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

// Obstacle sections of the constant block: centre tracks in ellipse-scaled
// coordinates (x_j(t)/a_j, y_j(t)/b_j) and per-obstacle (1/a_j, 1/b_j, a_j, b_j),
// with the semi-axes inflated by the robot circle radius.
__global__ void prep_obstacles_kernel(float *cblob, ConstLayout L, const float *xo, const float *yo,
                                      const float *a, const float *b, float r_c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L.n * L.q) {
        const int j = i / L.q, t = i - L.q * j;
        const float aj = a[j] + r_c, bj = b[j] + r_c;
        float2 *obs = reinterpret_cast<float2 *>(cblob + L.off_obs);
        obs[j * L.qs + t] = make_float2(xo[i] / aj, yo[i] / bj);
    }
    if (i < L.n) {
        const float aj = a[i] + r_c, bj = b[i] + r_c;
        reinterpret_cast<float4 *>(cblob + L.off_obc)[i] = make_float4(1.f / aj, 1.f / bj, aj, bj);
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
// non-finite cost ranks last.  Writes {index, cost, residual, c_x, c_y, c_psi}.
// Lexicographic best over B trajectories (collision-free first, then cost,
// then index); the whole block takes part, out gets 36 floats.
__device__ void select_best(const float *state, const float *cost, const float *res,
                            const float *mind, int B, float *out, Key *sk)
{
    Key best{2, FLT_MAX, 0x7fffffff};
    for (int l = threadIdx.x; l < B; l += blockDim.x) {
        float c = cost[l];
        Key k{mind[l] < 0.99f ? 1 : 0, isfinite(c) ? c : FLT_MAX, l};
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

__global__ void argmin_kernel(const float *state, const float *cost, const float *res,
                              const float *mind, int B, float *out)
{
    __shared__ Key sk[1024];
    select_best(state, cost, res, mind, B, out, sk);
}

__global__ void group_argmin_kernel(const FusedProblem *probs, const int *list, float *out)
{
    __shared__ Key sk[1024];
    const FusedProblem &p = probs[list[blockIdx.x]];
    select_best(p.state, p.cost, p.res, p.mind, p.B, out + 36 * blockIdx.x, sk);
}

}  // namespace

int launch_init_state(float *state, const float *init, const float *warm, int B, void *stream,
                      int *launches)
{
    const int n = B * STATE;
    init_state_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(state, init,
                                                                                      warm, B);
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

int launch_argmin(const float *state, const float *cost, const float *res, const float *mind,
                  int B, float *best_out, void *stream, int *launches)
{
    argmin_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(state, cost, res, mind, B,
                                                                     best_out);
    if (launches) ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam
