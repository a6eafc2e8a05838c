// Internal declarations shared by the host setup, the kernels and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

struct am_problem;
struct am_group;

namespace trajam {

// NVTX range for the duration of a scope (solves, group solves, server
// rounds); free unless a profiler attaches.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int NV = 11;        // coefficients per polynomial (degree 10)
constexpr int NS = 22;        // unknowns per side: (c_pos, c_slack)
constexpr int NX = 44;        // xi1
constexpr int STATE = 110;    // xi1, xi2, lambda, lambda_psi
constexpr int MAXM = 4;

// ---------------------------------------------------------------- host FP64

struct ProblemParams {
    int q = 0;
    double T = 0;
    int m = 0;
    double r[MAXM] = {0, 0, 0, 0};
    double r_c = 0, v_max = 0, a_max = 0, rho = 1, rho_psi = 1;
    double x_bc[6] = {}, y_bc[6] = {}, psi_bc[6] = {};
    int alpha_mode = 0, psi_dual_sign = 0, cs_boundary = 1, precision = 0;
};

// Everything the device needs that depends only on the problem shape, formed
// in FP64 on the host.
struct HostSetup {
    int q = 0, n = 0;
    std::vector<double> P, Pd, Pdd;          // q x NV, row-major
    double H[NV][NV];                         // Pdd^T Pdd
    double PtP[NV][NV];                       // P^T P
    double FtF[NS][NS];                       // per-side F^T F
    double Minv[NS][NS];                      // K^{-1}[:22, :22] of the position KKT
    double MQ[NS][NS];                        // Minv * blockdiag(H, H)
    double kb[2][NS];                         // K^{-1}[:22, 22:] b_side (x then y side)
    double ends[5][6];                        // boundary control points c_0,c_1,c_2,c_8,c_9,c_10
                                              // of c_x, c_c, c_y, c_s, c_psi
    double Mpsi[NV][NV];                      // K_psi^{-1}[:11, :11]
    double MpsiH[NV][NV];                     // Mpsi * H
    double kbpsi[NV];                         // K_psi^{-1}[:11, 11:] b_psi
    std::vector<double> W;                    // q x NV: W = P Mpsi^T
    double cond_pos = 0, cond_psi = 0;        // inf-norm condition estimates
    std::vector<double> Kp, Kq;               // both KKT inverses (b-independent), kept so a
    int kdim = 0;                             // boundary change only re-folds kb, kbpsi
};

// Bernstein basis and derivatives on t_k = k T / (q - 1).
void bernstein_basis(int q, double T, std::vector<double> &P, std::vector<double> &Pd,
                     std::vector<double> &Pdd);

// Forms every matrix of HostSetup for the given problem and obstacle count.
// Returns 0, or -1 when a KKT matrix is singular.
int build_setup(const ProblemParams &pp, int n, HostSetup &S);

// Recomputes only the boundary-dependent vectors kb, kbpsi.
int rebuild_boundary(const ProblemParams &pp, HostSetup &S);

// Value, first and second time derivative at t (clamped to [0, T]) of a
// degree-10 Bernstein polynomial with control points c on [0, T] (Eq. param).
void bernstein_eval(const float *c, double T, double t, double out[3]);

// Lower Cholesky factor (row-major 5 x 5) of the batch initialisation's
// covariance of control points 3..7: the inverse of D2^T D2 restricted to
// them (D2 the second-difference operator on 11 points), scaled to a largest
// variance of 1.
void init_cov_factor(double Lc[25]);

// ------------------------------------------------------------ device layout

// Offsets (in floats) of the sections of the constant block the kernels stage
// into shared memory.  Every section starts on a 16-byte boundary.
struct ConstLayout {
    int q, qs, m, n;          // qs: padded stride of per-step columns
    int qp;                   // stride (in pairs) of the split per-step columns
    int off_pcol;             // [3][NV][qs]  P, Pd, Pdd columns (FP32, plain loop)
    int off_wcol;             // [NV][qs]     W = P Mpsi^T, columns (FP32, plain loop)
    int off_fused;            // start of the part the fused kernel stages, in two regions:
                              // [off_fused, off_obs) and [off_obt, total)
    int off_prow;             // [3][q][12]   P, Pd, Pdd rows (padded to 12)
    int off_pcol2;            // [3][NV][qp][2] P, Pd, Pdd columns as TF32 (hi, lo) pairs
    int off_mt;               // [NS][24]     Minv^T
    int off_mq;               // [NS][24]     (Minv blockdiag(H, H))^T
    int off_ends;             // [5][8]       boundary control points per block (xi1 blocks, c_psi)
    int off_kb;               // [2][24]      kb (x side, y side)
    int off_mpsi;             // [NV][12]     Mpsi^T
    int off_mpsih;            // [NV][12]     (Mpsi H)^T
    int off_ptp;              // [NV][12]     P^T P
    int off_kbpsi;            // [12]
    int off_obs;              // [n][qs][2]   (x_j(t)/a_j, y_j(t)/b_j) pairs
    int off_obc;              // [n][4]       1/a_j, 1/b_j, a_j, b_j (inflated)
    int off_obt;              // [n]          near threshold (1 + (r_max + margin) max(1/a_j, 1/b_j))^2
    int off_obs2;             // [n][qs/2][4] per pair of steps (t, t + 1), t even: -x_j/a_j at t, t + 1,
                              //              then -y_j/b_j at t, t + 1 (the fused kernel's paired form)
    int off_obc2;             // [n][8]       1/a_j, 1/a_j, 1/b_j, 1/b_j, a_j, a_j, b_j, b_j
    int total;                // floats, multiple of 4
    float rho, rho_psi, v_max, a_max;
    float r[MAXM];
    float psi_sign;           // +1 default reading, -1 printed sign
    int alpha_mode;
    int cs_boundary;          // slack blocks carry boundary rows
    int precision;            // the contraction R: 0 FP32 (three TF32 products), 1 one
                              // TF32 product, 2 one BF16 product, 3 split BF16 (three
                              // BF16 products of K = 16)
    int diag_stall;           // diagnostic: stage without the copy, so the bounded
                              // wait on it runs out (failure-detection tests)
    int select;               // best selection among colliding trajectories:
                              // 0 lowest cost, 1 largest smallest distance
};

ConstLayout make_layout(int q, int m, int n);
// Writes the shape-dependent sections (everything except the obstacles).
void fill_constants(const HostSetup &S, const ProblemParams &pp, const ConstLayout &L,
                    std::vector<float> &blob);

// ------------------------------------------------------------ launchers

struct SolveArgs {
    const float *cblob;       // device constant block (ConstLayout)
    ConstLayout L;
    int B, iters;
    float *state;             // B x STATE, in/out
    float *res, *res_psi, *cost, *mind;  // B each
    float *hist;              // B x iters x 3, or nullptr
    int tile;                 // trajectories per CTA (0 = automatic)
    int *err;                 // device status word; kernels set it on a failed wait
};

// Fused persistent kernel: every iteration of the loop in one launch.
int launch_fused(const SolveArgs &a, void *stream, int *launches);

// Large-batch fused kernel on the fifth-generation tensor cores (tiles of
// 128 trajectories).  large_supported: 1 when the problem's form and shape
// fit it (FP32 precision form, default alpha form, q <= 128, no history,
// shared memory within the limit), else 0; launch_large returns -1 then.
int large_supported(const ConstLayout &L, bool hist);
size_t large_smem_bytes(const ConstLayout &L);
int launch_large(const SolveArgs &a, void *stream, int *launches);

// Warp-pair fused kernel (NW = 2, 3 or 4 warps run every iteration of one
// trajectory, for q <= 128, 192, 256; no block barrier inside the loop).
// warp_supported: 1 when the form and shape fit it (FP32 precision form,
// default alpha form, cs_boundary, q <= 256, shared memory within the
// limit), else 0; launch_warp returns -1 then.
int warp_supported(const ConstLayout &L);
size_t warp_smem_bytes(const ConstLayout &L, int traj_per_cta);
int warp_max_traj(const ConstLayout &L);
int warp_auto_traj(const ConstLayout &L, int B, int sms);
int launch_warp(const SolveArgs &a, void *stream, int *launches);
// The warp-pair group kernels (variants 32..43, one per circle count and
// NW): up to 16 / NW trajectory slots per CTA, one count per launch.
// warp_group_traj: the most slots a problem fits in kGroupSmemLimit (0 when
// not even one fits); warp_smem_bytes(L, slots) is what it needs at a given
// count; warp_group_variant: its variant.
int warp_group_traj(const ConstLayout &L);
int warp_group_variant(const ConstLayout &L);

// Dynamic shared memory of the single-problem kernels; the debug build's
// static flag needs a little of the 227 KB.
#ifdef AM_DEBUG_BOUNDS
constexpr size_t kFusedSmemMax = 227 * 1024 - 512;
#else
constexpr size_t kFusedSmemMax = 227 * 1024;
#endif

// One problem as the fused kernels see it (also the element of the work
// descriptor array of a grouped launch).
struct FusedProblem {
    const float *cblob;
    ConstLayout L;
    int B, iters, T, ntiles;
    float *state, *res, *res_psi, *cost, *mind, *hist;
    int *err;
};

// World-space margin (m) of the near-obstacle test: a warp's list of
// obstacles near its steps stays valid until one of its robot centres has
// moved farther than this since the list was formed.
constexpr float kNearMargin = 0.6f;

// Grouped launch: many problems' tiles in persistent kernels, one kernel per
// variant (circle count, alpha form) present; the variant kernels of one
// solve run concurrently.
// Variants 0..31: the small-tile group kernels, precision (4) x circle count
// (4) x alpha form (2); 32..43: the warp-pair group kernels (FP32, default
// alpha form), 32 + 4 (NW - 2) + m - 1 for NW = 2, 3, 4 warps per
// trajectory and 1..4 circles, for problems whose handle selects the
// warp-pair kernel (AM_KERNEL_WARP or AM_KERNEL_AUTO) and whose shape it takes.
constexpr int kGroupWarpVariant0 = 32;
constexpr int kGroupVariants = 44;
// Dynamic shared memory a warp-pair group kernel may take (its problem
// descriptor and work-item slot are static shared memory).
constexpr size_t kGroupSmemLimit = 227 * 1024 - 1024;
// The closed-form obstacle step in the ellipse-scaled frame (Eq. zeta_2,
// compute_zeta_3): the offset (xh, yh) of a circle centre from the
// obstacle's is projected to (xh, yh) max(1, 1/|.|), a correction of
// (xh, yh) h with h = max(1, 1/sqrt(D)) - 1 and D = xh^2 + yh^2 + kTinyD
// (kTinyD keeps D positive).  The x part is (xh + kCoincideT) h, where
// kCoincideT = sqrt(kTinyD).  A centre exactly at the obstacle's (D =
// kTinyD) then gets the correction (1, 0), the oracle's alpha = atan2(0, 0)
// = 0 with d = 1 (the point (a, 0)).  kCoincideT rounds away unless
// |xh| < 3e-12, and the add runs beside the rsqrt, not after it.
constexpr float kTinyD = 2e-38f;
constexpr float kCoincideT = 1.4142135e-19f;
// Raises a kernel's dynamic shared-memory limit on the current device to at
// least smem and never lowers it, so that a CUDA graph captured with a larger
// launch of the kernel stays launchable after smaller launches (a profiler
// re-launches graph nodes one at a time with the function's current limit).
// Thread-safe.
// Returns 0 (cudaSuccess) or the cudaError_t of the failed call.
int raise_smem_limit(const void *kernel, size_t smem);
struct GroupLaunch {
    const FusedProblem *d_probs;  // device array, one per problem
    const int *d_items;           // device array of (problem, tile) pairs, all variants
    const int *d_head;            // device: item count per variant [kGroupVariants], then list
                                  // offset per variant [kGroupVariants]
    int *d_ctl;                   // device {work counter, status} per variant; the
                                  // variant's counter is zeroed by launch_group
    int variant;                  // precision * 8 + m * 2 + alpha_mode - 2
    int threads;
    size_t smem;
    int grid;
    int slots;                    // warp-pair variants: trajectory slots per CTA
};
int group_variant(const ConstLayout &L);
// Tile size (trajectories per CTA) of a problem in a grouped launch of the
// given block size; 0 when the problem does not fit.
int group_tile(const ConstLayout &L, int threads);
int fused_max_threads();
// Returns 0, -1 (configuration out of range) or -2 (CUDA error, *why says which).
int launch_group(const GroupLaunch &g, void *stream, int *launches, const char **why);
int launch_group_warp(const GroupLaunch &g, void *stream, int *launches, const char **why);
// Best-trajectory selection for several problems in one launch: one block per
// listed problem; writes 36 floats per entry ({index, cost, res, 33 coefficients}).
int launch_group_argmin(const FusedProblem *d_probs, const int *d_list, int count, float *d_out,
                        void *stream, int *launches);
// Unfused comparator: one launch per step, intermediates in global memory.
int launch_plain(const SolveArgs &a, float *scratch, size_t scratch_floats, void *stream,
                 int *launches);
size_t plain_scratch_floats(const ConstLayout &L, int B);
// Best-trajectory selection; writes {index, cost, res, 33 coefficients}.
int launch_argmin(int select, const float *state, const float *cost, const float *res, const float *mind,
                  int B, float *best_out, void *stream, int *launches);
// Converts raw obstacle arrays (device) into the kernel's obstacle sections.
int launch_prep_obstacles(float *cblob, const ConstLayout &L, const float *xo, const float *yo,
                          const float *a, const float *b, float r_c, void *stream, int *launches);
// Builds the initial state from B x 3 x 11 coefficients (+ optional lambdas);
// the slack control points start at cos / sin of the heading control points.
// Batch re-draw around the straight line between the boundary positions
// (am_resample); line = (x0, x1, y0, y1, psi0, psi1).
struct ResampleArgs {
    float Lc[25];
    float line[6];
    float sigma;
    unsigned long long seed;
    int B;
};
int launch_resample(float *state, const ResampleArgs &a, void *stream, int *launches);

// Multipliers (state entries 55..109) of B trajectories times factor.
int launch_scale_multipliers(float *state, int B, float factor, void *stream, int *launches);

// Re-timing of a batch (am_shift): S maps old control points to new, row-major.
struct ShiftArgs {
    float S[121];
    int B;
};
int launch_shift(float *state, const ShiftArgs &a, void *stream, int *launches);

// CEM comparator (am_cem_*): device buffers and settings of one run.
struct CemArgs {
    const float *cblob;
    ConstLayout L;
    float *z, *cost, *dmin;    // N x 15 samples, N scores, N smallest ellipse distances
    float *mu, *sig, *chol;    // 15, 15 x 15, 15 x 15 (lower)
    float *best;               // z (15), J, d_min, coefficients (33)
    const float *given;        // nullable: score these N x 33 coefficient vectors instead
    int N, K, NP;              // samples, elites, N rounded up to a power of two
    int iter;
    unsigned long long seed;
    float w_coll, w_bound, alpha, reg;
};
size_t cem_score_smem(const ConstLayout &L);
size_t cem_refit_smem(int NP, int K);
int launch_cem_score(const CemArgs &a, void *stream);
int launch_cem_refit(const CemArgs &a, void *stream);

// Control points of a degree-10 Bernstein polynomial on [s, s + 1] from those on
// [0, 1] (blossoming): row-major 11 x 11, c' = S c.
void shift_matrix(double s, double S[121]);

// The initial state from B x 33 initial coefficients and optional B x 55 warm
// multipliers (device memory, read when the stream reaches the launch); with
// out and err also clears the 4 B results and the status word.
int launch_init_state(float *state, const float *init, const float *warm, int B, void *stream,
                      int *launches, float *out = nullptr, int *err = nullptr);
// Queues the best selection of a group's last solve on st and copies the
// records (36 floats per active problem) and the kernels' status words into
// pinned host memory, without waiting; group_status reads those status words
// once the stream has passed that point.
int group_best_async(::am_group *g, float *h_out, void *st);
int group_status(const ::am_group *g);
// The same for one problem's status word (into the handle's pinned area).
int problem_status_async(::am_problem *h, void *st);
int problem_status(const ::am_problem *h);
// Handle accessors for entry points outside the C-ABI file.
int handle_constants(const ::am_problem *h, const float **cblob, ConstLayout *L);
// Makes work queued next on stream wait for everything queued so far on the
// handle's own stream (its constant uploads and obstacle preparation): an
// event the handle owns is recorded there and waited on.  Nothing is
// allocated.  Skipped when the streams are the same or stream is capturing.
int handle_order_before(const ::am_problem *h, void *stream);
int report_error(int code, const char *msg);
// Scene accessors for the server.  problem_shape returns -1 when the handle
// has no state yet.
int problem_shape(const ::am_problem *h, int *q, int *m, int *n, int *B, double *T);
void problem_boundary(const ::am_problem *h, double x[6], double y[6], double psi[6]);
// New obstacle centre tracks (host, n x q each), semi-axes unchanged.
int problem_update_tracks(::am_problem *h, const float *xo, const float *yo);
size_t problem_device_bytes(const ::am_problem *h);
// Device bytes a handle holds for a batch of B (no history, fused kernel).
size_t scene_bytes(int q, int m, int n, int B);
// Fused kernel tile selection, exposed for the autotuner.
int fused_auto_tile(const ConstLayout &L, int B, int num_sms);
size_t fused_smem_bytes(const ConstLayout &L, int tile);

}  // namespace trajam
