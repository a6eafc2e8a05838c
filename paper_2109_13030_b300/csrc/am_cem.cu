// Cross-entropy method (CEM) planner: the sampling-based comparator the paper
// measures its optimizer against (Sec. IV, Table IV: CEM with 8k samples).
//
// The paper gives CEM's sample count only; this form is the textbook one.
// The search space is the interior control points 3..7 of c_x, c_y and c_psi,
// 15 numbers z (the boundary points come from the problem's boundary
// conditions, as in the AM solve).  Every iteration draws N samples
// z ~ N(mu, Sigma), scores each with
//     J = sum_t (x''^2 + y''^2 + psi''^2)                       (Eq. acc_cost)
//       + w_coll  sum_{t,i,j} max(0, 1 - d_ij(t))^2              (penetration)
//       + w_bound sum_t (max(0, |v| - v_max)^2 + max(0, |a| - a_max)^2),
// with d_ij the ellipse distance sqrt(xt^2/a^2 + yt^2/b^2) of circle i to
// obstacle j (inflated semi-axes), keeps the K lowest (ties to the lower
// sample index), and refits mu, Sigma to them with smoothing alpha:
//     mu <- alpha mean + (1 - alpha) mu,  Sigma <- alpha cov + (1 - alpha) Sigma + reg I
// (cov normalised by K).  The lowest J seen over all iterations is the result.
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>

#include "am_internal.h"
#include "am_rng.cuh"

namespace trajam {
namespace {

constexpr int kCemWarps = 8;   // samples in flight per block of the scoring kernel
constexpr int kCemObsSmem = 48 * 1024;  // obstacle tracks staged in shared memory up to this size
constexpr int kZ = 15;         // interior control points searched
constexpr int kParts = 4;      // partial sums per statistic in the refit (225 x 4 <= 1024 threads)

__device__ __forceinline__ float dot11(const float *a, const float *b)
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NV; ++k) s = fmaf(a[k], b[k], s);
    return s;
}

// Bytes of the obstacle sections (tracks and per-obstacle constants) of the constant block.
__host__ __device__ inline int cem_obs_floats(const ConstLayout &L) { return L.off_obt - L.off_obs; }

// Score samples: one warp per sample, the lanes over the time steps.  With
// `given`, the samples are full coefficient vectors (count x 33: c_x, c_y,
// c_psi) instead of draws.  The basis rows, and the obstacle sections when
// they fit, are staged in shared memory once per block.
__global__ void __launch_bounds__(32 * kCemWarps, 4) cem_score_kernel(CemArgs a)
{
    extern __shared__ __align__(16) float cem_sm[];
    const ConstLayout &L = a.L;
    float *rows = cem_sm;                            // [3][q][12] basis rows P, Pd, Pdd
    const int nrow = 3 * L.q * 12;
    for (int i = threadIdx.x; i < nrow; i += blockDim.x) rows[i] = a.cblob[L.off_prow + i];
    float *coef = cem_sm + nrow + 36 * (threadIdx.x >> 5);   // this warp's 33 coefficients
    const int nobs = cem_obs_floats(L);
    const bool staged = nobs * 4 <= kCemObsSmem;
    float *os = cem_sm + nrow + 36 * kCemWarps;      // 16-byte aligned: nrow and 36 k are multiples of 4
    if (staged)
        for (int i = threadIdx.x; i < nobs; i += blockDim.x) os[i] = a.cblob[L.off_obs + i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const float *ends = a.cblob + L.off_ends;
    const float *ob = staged ? os : a.cblob + L.off_obs;
    const float2 *obs = reinterpret_cast<const float2 *>(ob);
    const float4 *obc = reinterpret_cast<const float4 *>(ob + (L.off_obc - L.off_obs));
    for (int s = blockIdx.x * kCemWarps + (threadIdx.x >> 5); s < a.N; s += gridDim.x * kCemWarps) {
        if (a.given) {
            // 33 coefficients over 32 lanes: lane 0 also takes the last one
            coef[lane] = a.given[(size_t)s * 33 + lane];
            if (lane == 0) coef[32] = a.given[(size_t)s * 33 + 32];
        } else {
            // z = mu + chol eps, eps standard normal from stream (iteration, sample)
            double e0 = 0.0, e1 = 0.0;
            if (lane < 8) normal_pair(a.seed, (unsigned long long)a.iter * 16777216ull + s, lane, e0, e1);
            float z = lane < kZ ? a.mu[lane] : 0.f;
            for (int j = 0; j < kZ; ++j) {
                const float v0 = __shfl_sync(full, float(e0), j >> 1), v1 = __shfl_sync(full, float(e1), j >> 1);
                if (lane < kZ && j <= lane) z = fmaf(a.chol[lane * kZ + j], (j & 1) ? v1 : v0, z);
            }
            if (lane < kZ) a.z[(size_t)s * kZ + lane] = z;
            // coefficient k of block b: boundary points from the problem, 3..7
            // from z (lane l holds coefficient l; coefficient 32, the last
            // heading point, is a boundary point and goes to lane 0 as well)
            const int b = lane / NV, k = lane - NV * b, eb = 2 * b;   // ends blocks: c_x 0, c_y 2, c_psi 4
            const float zk = __shfl_sync(full, z, b * 5 + (k >= 3 && k <= 7 ? k - 3 : 0));
            coef[lane] = k <= 2 ? ends[eb * 8 + k] : k >= 8 ? ends[eb * 8 + k - 5] : zk;
            if (lane == 0) coef[32] = ends[4 * 8 + 5];
        }
        __syncwarp();
        float js = 0.f, pc = 0.f, pb = 0.f, dmin = FLT_MAX;
        for (int t = lane; t < L.q; t += 32) {
            const float *p = rows + t * 12, *pd = rows + (L.q + t) * 12, *pdd = rows + (2 * L.q + t) * 12;
            const float x = dot11(p, coef), xd = dot11(pd, coef), xdd = dot11(pdd, coef);
            const float y = dot11(p, coef + 11), yd = dot11(pd, coef + 11), ydd = dot11(pdd, coef + 11);
            const float psi = dot11(p, coef + 22), psidd = dot11(pdd, coef + 22);
            js += xdd * xdd + ydd * ydd + psidd * psidd;
            const float ev = fmaxf(0.f, sqrtf(xd * xd + yd * yd) - L.v_max);
            const float ea = fmaxf(0.f, sqrtf(xdd * xdd + ydd * ydd) - L.a_max);
            pb += ev * ev + ea * ea;
            float sp, cp;
            sincosf(psi, &sp, &cp);
            for (int j = 0; j < L.n; ++j) {
                const float2 o = obs[j * L.qs + t];   // one load per obstacle and step
                const float4 c = obc[j];
                for (int i = 0; i < L.m; ++i) {
                    const float X = fmaf(L.r[i], cp, x), Y = fmaf(L.r[i], sp, y);
                    const float xh = fmaf(X, c.x, -o.x), yh = fmaf(Y, c.y, -o.y);
                    const float D = fmaf(xh, xh, yh * yh);
                    const float d = D * rsqrtf(D + 1e-30f);   // sqrt(D), within a few ulp
                    const float e = fmaxf(0.f, 1.f - d);
                    pc += e * e;
                    dmin = fminf(dmin, d);
                }
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            js += __shfl_xor_sync(full, js, off);
            pc += __shfl_xor_sync(full, pc, off);
            pb += __shfl_xor_sync(full, pb, off);
            dmin = fminf(dmin, __shfl_xor_sync(full, dmin, off));
        }
        if (lane == 0) {
            const float J = js + a.w_coll * pc + a.w_bound * pb;
            a.cost[s] = isfinite(J) ? J : FLT_MAX;
            a.dmin[s] = dmin;
        }
        __syncwarp();
    }
}

// Refit (one block of 1024 threads): sort the N scores with their indices
// (bitonic, ascending by (score, index)), take the K best, form their mean
// and covariance, smooth into mu and Sigma, factor Sigma, and keep the best
// sample seen so far in best = {z (15), J, d_min, coefficients (33)}.
__global__ void __launch_bounds__(1024) cem_refit_kernel(CemArgs a)
{
    extern __shared__ __align__(16) float cem_sm[];
    const int np = a.NP;
    float *key = cem_sm;
    int *idx = reinterpret_cast<int *>(cem_sm + np);
    float *E = cem_sm + 2 * np;          // [K][15] elite samples
    float *mn = E + a.K * kZ;            // [16] elite mean
    float *S = mn + 16;                  // [225] smoothed covariance
    float *Lf = S + 228;                 // [225] its Cholesky factor
    float *part = Lf + 228;              // [kParts][225] partial sums
    const int tid = threadIdx.x;
    for (int i = tid; i < np; i += blockDim.x) {
        key[i] = i < a.N ? a.cost[i] : FLT_MAX;
        idx[i] = i;
    }
    __syncthreads();
    // Bitonic sort of the (score, index) pairs.  The pairs form one chunk per
    // warp (np / 32 pairs, at least 32 or all of them); a sub-stage whose
    // partners lie within a chunk runs on its warp with warp synchronisation,
    // the others on the whole block.  The compare-exchange network, and so
    // the result, is the same either way.
    auto exchange = [&](int i, int j, int k) {
        const int l = i ^ j;
        if (l > i) {
            const bool up = (i & k) == 0;
            const bool gt = key[i] > key[l] || (key[i] == key[l] && idx[i] > idx[l]);
            if (gt == up) {
                const float tk = key[i];
                key[i] = key[l];
                key[l] = tk;
                const int ti = idx[i];
                idx[i] = idx[l];
                idx[l] = ti;
            }
        }
    };
    const int warp = tid >> 5, lane = tid & 31;
    const int chunk = np <= 32 ? np : (np / 32 > 32 ? np / 32 : 32), nchunks = np / chunk;
    bool warp_local = false;  // the last sub-stage ended with warp synchronisation only
    for (int k = 2; k <= np; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < chunk) {
                if (warp < nchunks)
                    for (int m = lane; m < chunk; m += 32) exchange(warp * chunk + m, j, k);
                __syncwarp();
                warp_local = true;
            } else {
                if (warp_local) __syncthreads();
                for (int i = tid; i < np; i += blockDim.x) exchange(i, j, k);
                __syncthreads();
                warp_local = false;
            }
        }
    __syncthreads();
    for (int e = tid; e < a.K * kZ; e += blockDim.x) E[e] = a.z[(size_t)idx[e / kZ] * kZ + e % kZ];
    __syncthreads();
    // elite mean and covariance: kParts threads per entry over strided elites,
    // then one thread per entry adds the partials in a fixed order
    const int slot = tid / kParts, pp = tid - kParts * slot;   // entry (of 225), part
    if (slot < kZ) {
        float s = 0.f;
        for (int e = pp; e < a.K; e += kParts) s += E[e * kZ + slot];
        part[pp * 225 + slot] = s;
    }
    __syncthreads();
    if (tid < kZ) {
        float s = 0.f;
        for (int k = 0; k < kParts; ++k) s += part[k * 225 + tid];
        mn[tid] = s / float(a.K);
    }
    __syncthreads();
    if (slot < kZ * kZ) {
        const int r = slot / kZ, c = slot - kZ * r;
        const int lo = r < c ? r : c, hi = r < c ? c : r;   // both triangles from the same sums
        float s = 0.f;
        for (int e = pp; e < a.K; e += kParts) s = fmaf(E[e * kZ + hi] - mn[hi], E[e * kZ + lo] - mn[lo], s);
        part[pp * 225 + slot] = s;
    }
    __syncthreads();
    if (tid < kZ * kZ) {
        const int r = tid / kZ, c = tid - kZ * r;
        float s = 0.f;
        for (int k = 0; k < kParts; ++k) s += part[k * 225 + tid];
        const float v = a.alpha * (s / float(a.K)) + (1.f - a.alpha) * a.sig[tid] + (r == c ? a.reg : 0.f);
        S[tid] = v;
        a.sig[tid] = v;
    }
    if (tid < kZ) a.mu[tid] = a.alpha * mn[tid] + (1.f - a.alpha) * a.mu[tid];
    if (tid == 0 && key[0] < a.best[kZ]) {
        const int w = idx[0];
        for (int k = 0; k < kZ; ++k) a.best[k] = a.z[(size_t)w * kZ + k];
        a.best[kZ] = key[0];
        a.best[kZ + 1] = a.dmin[w];
        const float *ends = a.cblob + a.L.off_ends;
        for (int b = 0; b < 3; ++b)
            for (int k = 0; k < NV; ++k)
                a.best[kZ + 2 + 11 * b + k] = k <= 2 ? ends[2 * b * 8 + k]
                                              : k >= 8 ? ends[2 * b * 8 + k - 5]
                                                       : a.z[(size_t)w * kZ + 5 * b + k - 3];
    }
    __syncthreads();
    if (tid < 32) {
        // Cholesky of the smoothed covariance (positive definite: reg > 0) by
        // the first warp, column by column: lane i < 15 owns row i
        const int i = tid;
        for (int j = 0; j < kZ; ++j) {
            float s2 = i < j ? Lf[j * kZ + i] * Lf[j * kZ + i] : 0.f;
            for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            const float d = sqrtf(fmaxf(S[j * kZ + j] - s2, 1e-12f));
            if (i == j) Lf[j * kZ + j] = d;
            if (i > j && i < kZ) {
                float v = S[i * kZ + j];
                for (int k = 0; k < j; ++k) v -= Lf[i * kZ + k] * Lf[j * kZ + k];
                Lf[i * kZ + j] = v / d;
            }
            if (i < j) Lf[i * kZ + j] = 0.f;
            __syncwarp();
        }
    }
    __syncthreads();
    if (tid < kZ * kZ) a.chol[tid] = Lf[tid];
}

}  // namespace

size_t cem_score_smem(const ConstLayout &L)
{
    const int nobs = cem_obs_floats(L);
    return sizeof(float) * (3 * L.q * 12 + 36 * kCemWarps + (nobs * 4 <= kCemObsSmem ? nobs : 0));
}

size_t cem_refit_smem(int NP, int K)
{
    return sizeof(float) * (2 * size_t(NP) + size_t(K) * kZ + 16 + 228 + 228 + kParts * 225);
}

// Largest dynamic shared memory either kernel takes (q <= 256, staged
// obstacles <= kCemObsSmem; N <= 8192, K <= 1024), set once per device.
constexpr int kScoreSmemMax = (3 * 256 * 12 + 36 * kCemWarps) * 4 + kCemObsSmem;
constexpr int kRefitSmemMax = (2 * 8192 + 1024 * kZ + 16 + 228 + 228 + kParts * 225) * 4;

int cem_prepare(int dev, int *sms)
{
    static std::mutex mu;
    static int ready_dev = -1, n_sms = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (ready_dev != dev) {
        if (cudaFuncSetAttribute(cem_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kScoreSmemMax) !=
                cudaSuccess ||
            cudaFuncSetAttribute(cem_refit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kRefitSmemMax) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return -2;
        ready_dev = dev;
    }
    *sms = n_sms;
    return 0;
}

int launch_cem_score(const CemArgs &a, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t smem = cem_score_smem(a.L);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    if (smem > size_t(kScoreSmemMax) || cem_prepare(dev, &sms)) return -2;
    int blocks = (a.N + kCemWarps - 1) / kCemWarps;
    if (blocks > 8 * sms) blocks = 8 * sms;
    cem_score_kernel<<<blocks, 32 * kCemWarps, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_cem_refit(const CemArgs &a, void *stream)
{
    const size_t smem = cem_refit_smem(a.NP, a.K);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (smem > size_t(kRefitSmemMax) || cem_prepare(dev, &sms)) return -2;
    cem_refit_kernel<<<1, 1024, smem, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trajam
