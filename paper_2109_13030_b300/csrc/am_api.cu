// C ABI of the batched AM solver (include/trajam.h): handle lifetime, argument
// checking, device buffers and the launches of one solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "am_internal.h"
#include "../../include/trajam.h"

using namespace trajam;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(AM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

template <typename T>
int ensure(T *&ptr, size_t &cap, size_t count, const char *what)
{
    if (count <= cap && ptr) return AM_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    size_t n = count ? count : 1;
    CK(cudaMalloc(&ptr, n * sizeof(T)), what);
    cap = n;
    return AM_OK;
}

}  // namespace

struct am_problem {
    ProblemParams pp;
    HostSetup S;
    ConstLayout L;
    std::vector<float> blob;
    float *d_blob = nullptr;
    size_t blob_cap = 0;
    int n = 0;
    float *d_raw = nullptr;  // raw obstacles: xo, yo (n x q each), a, b
    size_t raw_cap = 0;
    int B = 0;
    float *d_state = nullptr, *d_out = nullptr, *d_best = nullptr, *d_in = nullptr;
    size_t state_cap = 0, out_cap = 0, best_cap = 0, in_cap = 0;
    float *d_hist = nullptr;
    size_t hist_cap = 0;
    float *d_scratch = nullptr;
    size_t scratch_cap = 0;
    int *d_err = nullptr;
    size_t err_cap = 0;
    bool hist_on = false;
    int hist_iters = 0;
    int kernel = AM_KERNEL_FUSED;
    int tile = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t order_ev = nullptr;  // orders other streams after this handle's stream
    int launches = 0;
    bool solved = false;
    int diag_stall = 0;
    int select = AM_SELECT_COST;
    float *h_best = nullptr;  // pinned: best record (36 floats), status word at 40
    float *h_out = nullptr;   // pinned: staging of the four result arrays (am_get_results)
    size_t h_out_cap = 0;
    // CEM comparator: samples, scores, distribution and best of the last run
    float *d_cem = nullptr, *d_score = nullptr;
    size_t cem_cap = 0, score_cap = 0;
    int cem_N = 0;
};

namespace {

// Waits (at most 60 s) for the work queued so far on a stream.
int wait_event(cudaEvent_t ev, cudaStream_t st)
{
    CK(cudaEventRecord(ev, st), "cudaEventRecord");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return AM_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "stream wait");
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
            return fail(AM_ERR_TIMEOUT, "stream did not finish within 60 s");
        std::this_thread::yield();
    }
}

// A kernel's status word: bit 0 a bounded wait that gave up, bit 1 an index
// outside its array caught by the debug build's checks.
int status_error(int err)
{
    if (err & 2) return fail(AM_ERR_STATE, "a kernel index was out of bounds (debug build; status %d)", err);
    if (err) return fail(AM_ERR_TIMEOUT, "a kernel gave up a bounded wait (status %d)", err);
    return AM_OK;
}

// Largest result set (floats, four arrays of B) that am_get_results stages
// through the handle's pinned area (16 MiB; larger batches copy per array).
constexpr size_t kStagedResultsMax = size_t(1) << 22;

int wait_stream(am_problem *h)
{
    // the status word rides on the same stream into pinned memory, so one
    // bounded wait covers the work and its status
    int *h_err = reinterpret_cast<int *>(h->h_best + 40);
    CK(cudaMemcpyAsync(h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status read");
    int rc = wait_event(h->ev, h->stream);
    if (rc) return rc;
    return status_error(*h_err);
}

cudaMemcpyKind kind_in(int mem) { return mem == AM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int mem) { return mem == AM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

bool finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// A float is non-finite exactly when its exponent bits are all ones.  The
// test runs over blocks of 1024 without an early exit inside a block, so the
// compiler vectorises it (about 7 us for the 33,000 floats of a 1000-sample
// batch, against about 28 us element by element).
bool finite_floats(const float *v, size_t n)
{
    size_t i = 0;
    while (i < n) {
        const size_t end = n - i < 1024 ? n : i + 1024;
        uint32_t bad = 0;
        for (; i < end; ++i) {
            uint32_t bits;
            std::memcpy(&bits, v + i, sizeof(bits));
            bad |= (bits & 0x7f800000u) == 0x7f800000u;
        }
        if (bad) return false;
    }
    return true;
}

// Uploads the non-obstacle sections of the constant block.
int upload_shape_sections(am_problem *h)
{
    fill_constants(h->S, h->pp, h->L, h->blob);
    return cudaMemcpyAsync(h->d_blob, h->blob.data(), size_t(h->L.off_obs) * sizeof(float),
                           cudaMemcpyHostToDevice, h->stream) == cudaSuccess
               ? AM_OK
               : fail(AM_ERR_CUDA, "constant upload failed");
}

void set_scalars(am_problem *h)
{
    ConstLayout &L = h->L;
    L.diag_stall = h->diag_stall;
    L.select = h->select;
    L.rho = float(h->pp.rho);
    L.rho_psi = float(h->pp.rho_psi);
    L.v_max = float(h->pp.v_max);
    L.a_max = float(h->pp.a_max);
    for (int i = 0; i < MAXM; ++i) L.r[i] = i < h->pp.m ? float(h->pp.r[i]) : 0.f;
    L.psi_sign = h->pp.psi_dual_sign ? -1.f : 1.f;
    L.alpha_mode = h->pp.alpha_mode;
    L.cs_boundary = h->pp.cs_boundary;
    L.precision = h->pp.precision;
}

// (Re)forms the setup for n obstacles: FP64 setup, layout, device block.
int reshape(am_problem *h, int n)
{
    HostSetup S;
    if (build_setup(h->pp, n, S) != 0) return fail(AM_ERR_ARG, "singular KKT matrix");
    h->S = S;
    h->n = n;
    h->L = make_layout(h->pp.q, h->pp.m, n);
    set_scalars(h);
    int rc = ensure(h->d_blob, h->blob_cap, size_t(h->L.total), "constant block");
    if (rc) return rc;
    CK(cudaMemsetAsync(h->d_blob, 0, size_t(h->L.total) * sizeof(float), h->stream), "memset");
    return upload_shape_sections(h);
}

int check_B(am_problem *h, int B)
{
    int rc = ensure(h->d_state, h->state_cap, size_t(B) * STATE, "state");
    if (!rc) rc = ensure(h->d_out, h->out_cap, size_t(B) * 4, "results");
    if (!rc) rc = ensure(h->d_in, h->in_cap, size_t(B) * (33 + 55), "input staging");
    if (!rc) rc = ensure(h->d_best, h->best_cap, size_t(64), "best");
    return rc;
}

}  // namespace

extern "C" {

const char *am_last_error(void) { return g_err.c_str(); }

int am_init_problem(const am_problem_desc *d, am_problem **out)
{
    if (!d || !out) return fail(AM_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->q < 2 || d->q > AM_MAX_Q) return fail(AM_ERR_ARG, "q must be in [2, %d]", AM_MAX_Q);
    if (!(d->T > 0) || !std::isfinite(d->T)) return fail(AM_ERR_ARG, "T must be > 0");
    if (d->degree != 10) return fail(AM_ERR_ARG, "only degree 10 is supported");
    if (d->m < 1 || d->m > AM_MAX_M || !d->r) return fail(AM_ERR_ARG, "m must be in [1, %d]", AM_MAX_M);
    if (!finite_all(d->r, d->m)) return fail(AM_ERR_ARG, "non-finite r");
    if (!(d->r_c >= 0) || !(d->v_max > 0) || !(d->a_max > 0) || !(d->rho > 0) || !(d->rho_psi > 0))
        return fail(AM_ERR_ARG, "r_c >= 0 and v_max, a_max, rho, rho_psi > 0 required");
    if (!finite_all(d->x_bc, 6) || !finite_all(d->y_bc, 6) || !finite_all(d->psi_bc, 6))
        return fail(AM_ERR_ARG, "non-finite boundary condition");
    if (d->precision != AM_FP32 && d->precision != AM_TF32 && d->precision != AM_BF16 &&
        d->precision != AM_SPLIT_BF16)
        return fail(AM_ERR_ARG, "precision %d not available", d->precision);
    if (d->alpha_mode < 0 || d->alpha_mode > 1 || d->psi_dual_sign < 0 || d->psi_dual_sign > 1 ||
        d->cs_boundary < 0 || d->cs_boundary > 1)
        return fail(AM_ERR_ARG, "flag out of range");
    am_problem *h = new (std::nothrow) am_problem;
    if (!h) return fail(AM_ERR_ARG, "out of host memory");
    ProblemParams &pp = h->pp;
    pp.q = d->q;
    pp.T = d->T;
    pp.m = d->m;
    for (int i = 0; i < d->m; ++i) pp.r[i] = d->r[i];
    pp.r_c = d->r_c;
    pp.v_max = d->v_max;
    pp.a_max = d->a_max;
    pp.rho = d->rho;
    pp.rho_psi = d->rho_psi;
    std::memcpy(pp.x_bc, d->x_bc, sizeof(pp.x_bc));
    std::memcpy(pp.y_bc, d->y_bc, sizeof(pp.y_bc));
    std::memcpy(pp.psi_bc, d->psi_bc, sizeof(pp.psi_bc));
    pp.alpha_mode = d->alpha_mode;
    pp.psi_dual_sign = d->psi_dual_sign;
    pp.cs_boundary = d->cs_boundary;
    pp.precision = d->precision;
    int rc = AM_OK;
    cudaError_t e = cudaFree(nullptr);
    if (e != cudaSuccess) rc = cuda_fail(e, "CUDA initialisation");
    if (!rc && cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(AM_ERR_CUDA, "event creation failed");
    if (!rc && cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(AM_ERR_CUDA, "event creation failed");
    if (!rc && cudaMallocHost(&h->h_best, 64 * sizeof(float)) != cudaSuccess)
        rc = fail(AM_ERR_CUDA, "pinned allocation failed");
    if (!rc) rc = ensure(h->d_err, h->err_cap, 1, "status word");
    if (!rc && cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess) rc = fail(AM_ERR_CUDA, "memset");
    if (!rc) rc = reshape(h, 0);
    if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = fail(AM_ERR_CUDA, "sync");
    if (rc) {
        am_destroy(h);
        return rc;
    }
    *out = h;
    return AM_OK;
}

void am_destroy(am_problem *h)
{
    if (!h) return;
    // No wait on h->stream: the caller may have destroyed that stream by now.
    // cudaFree itself waits for the device work in flight.
    cudaFree(h->d_blob);
    cudaFree(h->d_raw);
    cudaFree(h->d_state);
    cudaFree(h->d_out);
    cudaFree(h->d_best);
    cudaFree(h->d_in);
    cudaFree(h->d_hist);
    cudaFree(h->d_scratch);
    cudaFree(h->d_err);
    cudaFree(h->d_cem);
    cudaFree(h->d_score);
    if (h->h_best) cudaFreeHost(h->h_best);
    if (h->h_out) cudaFreeHost(h->h_out);
    if (h->ev) cudaEventDestroy(h->ev);
    if (h->order_ev) cudaEventDestroy(h->order_ev);
    delete h;
}

int am_set_stream(am_problem *h, void *stream)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    h->stream = static_cast<cudaStream_t>(stream);
    return AM_OK;
}

int am_set_obstacles(am_problem *h, int n, const float *xo, const float *yo, const float *a,
                     const float *b, int mem)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (n < 0 || n > AM_MAX_N) return fail(AM_ERR_ARG, "n must be in [0, %d]", AM_MAX_N);
    if (n > 0 && (!xo || !yo || !a || !b)) return fail(AM_ERR_ARG, "null obstacle array");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    const int q = h->pp.q;
    if (mem == AM_HOST) {
        for (int j = 0; j < n; ++j)
            if (!(a[j] > 0) || !(b[j] > 0) || !std::isfinite(a[j]) || !std::isfinite(b[j]))
                return fail(AM_ERR_ARG, "semi-axes must be finite and > 0");
        if (n > 0 && (!finite_floats(xo, size_t(n) * q) || !finite_floats(yo, size_t(n) * q)))
            return fail(AM_ERR_ARG, "non-finite obstacle track");
    }
    int rc;
    if (n != h->n) {
        rc = reshape(h, n);
        if (rc) return rc;
    }
    if (n == 0) return AM_OK;
    rc = ensure(h->d_raw, h->raw_cap, size_t(2 * n * q + 2 * n), "obstacles");
    if (rc) return rc;
    const cudaMemcpyKind k = kind_in(mem);
    CK(cudaMemcpyAsync(h->d_raw, xo, sizeof(float) * n * q, k, h->stream), "obstacle copy");
    CK(cudaMemcpyAsync(h->d_raw + n * q, yo, sizeof(float) * n * q, k, h->stream), "obstacle copy");
    CK(cudaMemcpyAsync(h->d_raw + 2 * n * q, a, sizeof(float) * n, k, h->stream), "obstacle copy");
    CK(cudaMemcpyAsync(h->d_raw + 2 * n * q + n, b, sizeof(float) * n, k, h->stream), "obstacle copy");
    if (launch_prep_obstacles(h->d_blob, h->L, h->d_raw, h->d_raw + n * q, h->d_raw + 2 * n * q,
                              h->d_raw + 2 * n * q + n, float(h->pp.r_c), h->stream, nullptr))
        return fail(AM_ERR_CUDA, "obstacle preparation launch failed");
    return AM_OK;
}

int am_set_boundary(am_problem *h, const double x_bc[6], const double y_bc[6],
                    const double psi_bc[6])
{
    if (!h || !x_bc || !y_bc || !psi_bc) return fail(AM_ERR_ARG, "null argument");
    if (!finite_all(x_bc, 6) || !finite_all(y_bc, 6) || !finite_all(psi_bc, 6))
        return fail(AM_ERR_ARG, "non-finite boundary condition");
    std::memcpy(h->pp.x_bc, x_bc, sizeof(h->pp.x_bc));
    std::memcpy(h->pp.y_bc, y_bc, sizeof(h->pp.y_bc));
    std::memcpy(h->pp.psi_bc, psi_bc, sizeof(h->pp.psi_bc));
    if (rebuild_boundary(h->pp, h->S) != 0) return fail(AM_ERR_ARG, "singular KKT matrix");
    return upload_shape_sections(h);
}

int am_set_option(am_problem *h, int option, int value)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (option == AM_OPT_KERNEL) {
        if (value != AM_KERNEL_FUSED && value != AM_KERNEL_PLAIN && value != AM_KERNEL_LARGE &&
            value != AM_KERNEL_WARP && value != AM_KERNEL_AUTO)
            return fail(AM_ERR_ARG, "bad kernel");
        h->kernel = value;
        return AM_OK;
    }
    if (option == AM_OPT_TILE) {
        if (value < 0 || value > 64) return fail(AM_ERR_ARG, "tile must be in [0, 64]");
        h->tile = value;
        return AM_OK;
    }
    if (option == AM_OPT_SELECT) {
        if (value != AM_SELECT_COST && value != AM_SELECT_CLEARANCE) return fail(AM_ERR_ARG, "bad selection rule");
        h->select = value;
        h->L.select = value;
        return AM_OK;
    }
    if (option == AM_OPT_DIAG_STALL) {
        h->diag_stall = value != 0;
        h->L.diag_stall = h->diag_stall;
        return AM_OK;
    }
    return fail(AM_ERR_ARG, "unknown option %d", option);
}

int am_set_history(am_problem *h, int enable)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    h->hist_on = enable != 0;
    return AM_OK;
}

// The kernel a solve of B trajectories runs: the handle's choice, or for
// AM_KERNEL_AUTO the large-batch kernel from B = 16384 on, else the
// warp-pair kernel, else the small-tile kernel, each where it takes the
// problem's form and shape.
int solve_kernel(const am_problem *h, int B)
{
    if (h->kernel != AM_KERNEL_AUTO) return h->kernel;
    if (B >= 16384 && large_supported(h->L, h->hist_on)) return AM_KERNEL_LARGE;
    if (warp_supported(h->L)) return AM_KERNEL_WARP;
    return AM_KERNEL_FUSED;
}

int am_solve_batch(am_problem *h, int B, const float *init, const float *warm_lambda, int iters,
                   void *stream, int mem)
{
    NvtxRange range("am_solve_batch");
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (B < 1 || B > (1 << 24)) return fail(AM_ERR_ARG, "B must be in [1, 2^24]");
    if (iters < 1 || iters > 100000) return fail(AM_ERR_ARG, "iters must be in [1, 100000]");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    const int kern = solve_kernel(h, B);
    if (!init && (!h->solved || B != h->B))
        return fail(AM_ERR_STATE, "warm start needs a previous solve with the same B");
    if (!init && warm_lambda) return fail(AM_ERR_ARG, "warm_lambda needs init");
    if (kern == AM_KERNEL_PLAIN && h->pp.precision != AM_FP32)
        return fail(AM_ERR_ARG, "reduced precision runs on the fused kernel only");
    if (kern == AM_KERNEL_LARGE && !large_supported(h->L, h->hist_on))
        return fail(AM_ERR_ARG,
                    "the large-batch kernel takes the FP32 form, the default alpha form, q <= 128, no history "
                    "and operands within an SM's shared memory (q=%d, m=%d, n=%d: %zu bytes)",
                    h->pp.q, h->pp.m, h->n, large_smem_bytes(h->L));
    if (kern == AM_KERNEL_WARP && !warp_supported(h->L))
        return fail(AM_ERR_ARG,
                    "the warp-pair kernel takes the FP32 form, the default alpha form, cs_boundary, q <= 256 "
                    "and constants within an SM's shared memory (q=%d, m=%d, n=%d: %zu bytes)",
                    h->pp.q, h->pp.m, h->n, warp_smem_bytes(h->L, 1));
    if (h->kernel == AM_KERNEL_WARP && (h->tile < 0 || h->tile > warp_max_traj(h->L)))
        return fail(AM_ERR_ARG, "the warp-pair kernel runs 1..%d trajectories per CTA at q = %d (tile %d)",
                    warp_max_traj(h->L), h->pp.q, h->tile);
    h->stream = static_cast<cudaStream_t>(stream);
    h->launches = 0;
    const float *src = init, *warm = warm_lambda;
    if (init && mem == AM_HOST) {
        // The copies to the handle's staging buffer are queued first and the
        // inputs checked while they run.  A non-finite input returns before
        // anything reads the staging buffer and before the state is touched
        // (check_B below may reallocate it).
        int rc = ensure(h->d_in, h->in_cap, size_t(B) * (33 + 55), "input staging");
        if (rc) return rc;
        CK(cudaMemcpyAsync(h->d_in, init, sizeof(float) * 33 * B, cudaMemcpyHostToDevice, h->stream), "init copy");
        src = h->d_in;
        if (warm_lambda) {
            CK(cudaMemcpyAsync(h->d_in + 33 * size_t(B), warm_lambda, sizeof(float) * 55 * B,
                               cudaMemcpyHostToDevice, h->stream),
               "warm copy");
            warm = h->d_in + 33 * size_t(B);
        }
        if (!finite_floats(init, size_t(B) * 33)) return fail(AM_ERR_ARG, "non-finite initial coefficients");
        if (warm_lambda && !finite_floats(warm_lambda, size_t(B) * 55))
            return fail(AM_ERR_ARG, "non-finite warm multipliers");
    }
    int rc = check_B(h, B);
    if (rc) return rc;
    if (init) {
        // device inputs are read in place by the initial-state launch (which
        // also resets the status word); host inputs come from the staging
        // buffer
        if (launch_init_state(h->d_state, src, warm, B, h->stream, &h->launches, nullptr, h->d_err))
            return fail(AM_ERR_CUDA, "init launch failed");
    } else {
        CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream), "status reset");
    }
    h->B = B;
    float *hist = nullptr;
    if (h->hist_on) {
        rc = ensure(h->d_hist, h->hist_cap, size_t(B) * iters * 3, "history");
        if (rc) return rc;
        hist = h->d_hist;
        h->hist_iters = iters;
    }
    SolveArgs a;
    a.cblob = h->d_blob;
    a.L = h->L;
    a.B = B;
    a.iters = iters;
    a.state = h->d_state;
    a.res = h->d_out;
    a.res_psi = h->d_out + B;
    a.cost = h->d_out + 2 * size_t(B);
    a.mind = h->d_out + 3 * size_t(B);
    a.hist = hist;
    a.tile = h->kernel == AM_KERNEL_AUTO ? 0 : h->tile;
    a.err = h->d_err;
    if (kern == AM_KERNEL_FUSED) {
        rc = launch_fused(a, h->stream, &h->launches);
    } else if (kern == AM_KERNEL_LARGE) {
        rc = launch_large(a, h->stream, &h->launches);
    } else if (kern == AM_KERNEL_WARP) {
        rc = launch_warp(a, h->stream, &h->launches);
    } else {
        const size_t need = plain_scratch_floats(h->L, B);
        rc = ensure(h->d_scratch, h->scratch_cap, need, "plain scratch");
        if (rc) return rc;
        rc = launch_plain(a, h->d_scratch, h->scratch_cap, h->stream, &h->launches);
    }
    if (rc == -1)
        return fail(AM_ERR_ARG,
                    "problem shape (q=%d, m=%d, n=%d, tile %d) does not fit the fused kernel's shared memory; "
                    "the plain kernel (AM_OPT_KERNEL = AM_KERNEL_PLAIN) runs any shape",
                    h->pp.q, h->pp.m, h->n, h->tile);
    if (rc) return fail(AM_ERR_CUDA, "solve launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    h->solved = true;
    return AM_OK;
}

int am_get_results(am_problem *h, float *res, float *res_psi, float *cost, float *mind, int mem)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (!h->solved) return fail(AM_ERR_STATE, "no solve yet");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    float *dst[4] = {res, res_psi, cost, mind};
    const size_t nb = size_t(h->B);
    if (mem == AM_HOST && res && res_psi && cost && mind && 4 * nb <= kStagedResultsMax) {
        // all four to host memory: one copy of the contiguous result arrays
        // into the handle's pinned staging area, then host copies
        if (h->h_out_cap < 4 * nb) {
            if (h->h_out) cudaFreeHost(h->h_out);  // no copy into it is pending
            h->h_out = nullptr;
            h->h_out_cap = 0;
            CK(cudaMallocHost(&h->h_out, sizeof(float) * 4 * nb), "result staging area");
            h->h_out_cap = 4 * nb;
        }
        CK(cudaMemcpyAsync(h->h_out, h->d_out, sizeof(float) * 4 * nb, cudaMemcpyDeviceToHost, h->stream),
           "result copy");
        const int rc = wait_stream(h);
        if (rc) return rc;
        for (int i = 0; i < 4; ++i) std::memcpy(dst[i], h->h_out + i * nb, sizeof(float) * nb);
        return AM_OK;
    }
    for (int i = 0; i < 4; ++i)
        if (dst[i])
            CK(cudaMemcpyAsync(dst[i], h->d_out + size_t(i) * h->B, sizeof(float) * h->B,
                               kind_out(mem), h->stream),
               "result copy");
    return mem == AM_HOST ? wait_stream(h) : AM_OK;
}

int am_get_best(am_problem *h, float coeffs[33], float *cost, float *residual, int *index)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (!h->solved) return fail(AM_ERR_STATE, "no solve yet");
    if (launch_argmin(h->select, h->d_state, h->d_out + 2 * size_t(h->B), h->d_out, h->d_out + 3 * size_t(h->B),
                      h->B, h->d_best, h->stream, nullptr))
        return fail(AM_ERR_CUDA, "argmin launch failed");
    CK(cudaMemcpyAsync(h->h_best, h->d_best, 36 * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
       "best copy");
    int rc = wait_stream(h);
    if (rc) return rc;
    if (index) *index = int(h->h_best[0]);
    if (cost) *cost = h->h_best[1];
    if (residual) *residual = h->h_best[2];
    if (coeffs) std::memcpy(coeffs, h->h_best + 3, 33 * sizeof(float));
    // non-finite trajectories rank last, so a non-finite best means all are
    if (!std::isfinite(h->h_best[1])) return fail(AM_ERR_NAN, "every trajectory of the batch is non-finite");
    return AM_OK;
}

int am_get_best_async(am_problem *h, float *out, int mem, void *stream)
{
    if (!h || !out) return fail(AM_ERR_ARG, "null argument");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    if (!h->solved) return fail(AM_ERR_STATE, "no solve yet");
    h->stream = static_cast<cudaStream_t>(stream);
    float *dst = mem == AM_DEVICE ? out : h->d_best;
    if (launch_argmin(h->select, h->d_state, h->d_out + 2 * size_t(h->B), h->d_out, h->d_out + 3 * size_t(h->B),
                      h->B, dst, h->stream, nullptr))
        return fail(AM_ERR_CUDA, "argmin launch failed");
    if (mem == AM_HOST)
        CK(cudaMemcpyAsync(out, h->d_best, 36 * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "best copy");
    return AM_OK;
}

int am_get_state(am_problem *h, float *out, int mem)
{
    if (!h || !out) return fail(AM_ERR_ARG, "null argument");
    if (!h->solved) return fail(AM_ERR_STATE, "no state yet");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    CK(cudaMemcpyAsync(out, h->d_state, sizeof(float) * STATE * h->B, kind_out(mem), h->stream),
       "state copy");
    return mem == AM_HOST ? wait_stream(h) : AM_OK;
}

int am_set_state(am_problem *h, int B, const float *in, int mem)
{
    if (!h || !in) return fail(AM_ERR_ARG, "null argument");
    if (B < 1 || B > (1 << 24)) return fail(AM_ERR_ARG, "B must be in [1, 2^24]");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    int rc = check_B(h, B);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->d_state, in, sizeof(float) * STATE * B, kind_in(mem), h->stream),
       "state copy");
    h->B = B;
    h->solved = true;
    return AM_OK;
}

int am_get_history(am_problem *h, float *out, int mem)
{
    if (!h || !out) return fail(AM_ERR_ARG, "null argument");
    if (!h->solved || !h->d_hist || h->hist_iters == 0) return fail(AM_ERR_STATE, "no history");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    CK(cudaMemcpyAsync(out, h->d_hist, sizeof(float) * 3 * h->hist_iters * size_t(h->B),
                       kind_out(mem), h->stream),
       "history copy");
    return mem == AM_HOST ? wait_stream(h) : AM_OK;
}

int am_last_solve_stats(am_problem *h, int *launches)
{
    if (!h || !launches) return fail(AM_ERR_ARG, "null argument");
    *launches = h->launches;
    return AM_OK;
}

}  // extern "C"

namespace trajam {

// Read-only view of a handle's device constants, for entry points defined in
// other translation units.  Records the message and returns the code on error.
int handle_constants(const am_problem *h, const float **cblob, ConstLayout *L)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    *cblob = h->d_blob;
    *L = h->L;
    return AM_OK;
}

int handle_order_before(const am_problem *h, void *stream)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st == h->stream) return AM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs), "stream capture query");
    if (cs != cudaStreamCaptureStatusNone) return AM_OK;  // the caller orders a captured stream
    CK(cudaEventRecord(h->order_ev, h->stream), "order event record");
    CK(cudaStreamWaitEvent(st, h->order_ev, 0), "order event wait");
    return AM_OK;
}

int report_error(int code, const char *msg) { return fail(code, "%s", msg); }

}  // namespace trajam

// ----------------------------------------------------------------- groups

struct am_group {
    std::vector<am_problem *> probs;
    std::vector<int> active;  // problems the next solve advances; empty = all
    int threads = 0;          // block size; 0 = tuned or the kernel maximum
    int warp_slots = 0;       // cap on the warp-pair variants' trajectory slots per CTA; 0 = as many as fit
    bool use_graph = true;
    // One upload region per solve, device and pinned host copies:
    //   [count per variant, list offset per variant] [descriptors]
    //   [work items of every variant] [active list]
    char *d_up = nullptr, *h_up = nullptr;
    size_t up_cap = 0, h_up_cap = 0;
    std::vector<char> last_up;        // what the device region holds
    cudaEvent_t up_ev = nullptr;      // recorded after the last upload
    bool up_pending = false;
    FusedProblem *d_probs = nullptr;  // views into d_up
    int *d_items = nullptr, *d_head = nullptr, *d_list = nullptr;
    int *d_ctl = nullptr;     // {work counter, status} per variant
    size_t ctl_cap = 0;
    int *h_status = nullptr;  // pinned copy of the status words
    cudaEvent_t ev = nullptr;
    float *d_bests = nullptr; // 36 floats per active problem
    size_t bests_cap = 0;
    std::vector<FusedProblem> h_probs;
    std::vector<int> h_items, solved_list;  // work lists; active list of the last solve
    int count[kGroupVariants] = {}, offset[kGroupVariants] = {};
    size_t vsmem[kGroupVariants] = {};      // shared memory per variant kernel
    int vslots[kGroupVariants] = {};        // trajectory slots per CTA of a warp-pair variant
    // concurrent variant kernels: a stream each, fork and join events
    cudaStream_t vst[kGroupVariants] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kGroupVariants] = {};
    struct Captured {
        uint64_t mask;
        int threads;
        cudaStream_t stream;
        const char *up;
        size_t smem[kGroupVariants];
        int slots[kGroupVariants];
        cudaGraphExec_t exec;
    };
    std::vector<Captured> graphs;
    int launches = 0, nitems = 0;
    float *d_save = nullptr;  // state copies while tuning
    size_t save_cap = 0;
};

namespace {

void drop_graph(am_group *g)
{
    for (auto &c : g->graphs) cudaGraphExecDestroy(c.exec);
    g->graphs.clear();
}

std::vector<int> active_list(const am_group *g)
{
    if (!g->active.empty()) return g->active;
    std::vector<int> all(g->probs.size());
    for (size_t i = 0; i < all.size(); ++i) all[i] = int(i);
    return all;
}

// Descriptors of every problem (tile size for this block size; shared memory
// per variant as the largest of its problems, so a captured launch fits
// whatever subset is active) and the work lists of the active ones, per
// variant: the problems with the costliest tiles first (longest-processing-
// time order), the tiles of one problem together so a CTA rarely re-stages
// constants.
// The group variant of a problem: a warp-pair kernel (32 + 4 (NW - 2) + m - 1)
// when its handle selects them and they take its shape, else the small-tile
// variant of its precision form, circle count and alpha form.
int problem_variant(const am_problem *h)
{
    if ((h->kernel == AM_KERNEL_WARP || h->kernel == AM_KERNEL_AUTO) && warp_group_traj(h->L) > 0)
        return warp_group_variant(h->L);
    return group_variant(h->L);
}

int build_work(am_group *g, int threads, int iters, int sms)
{
    const int np = int(g->probs.size());
    g->h_probs.resize(np);
    std::memset(static_cast<void *>(g->h_probs.data()), 0, sizeof(FusedProblem) * np);
    for (int v = 0; v < kGroupVariants; ++v) g->vsmem[v] = 0, g->vslots[v] = 0;
    // a warp-pair variant runs as many trajectory slots per CTA as all its
    // problems fit
    for (int i = 0; i < np; ++i) {
        const int v = problem_variant(g->probs[i]);
        if (v < kGroupWarpVariant0) continue;
        int t = warp_group_traj(g->probs[i]->L);
        if (g->warp_slots > 0 && t > g->warp_slots) t = g->warp_slots;
        if (g->vslots[v] == 0 || t < g->vslots[v]) g->vslots[v] = t;
    }
    for (int i = 0; i < np; ++i) {
        am_problem *h = g->probs[i];
        const int v = problem_variant(h);
        const bool warp = v >= kGroupWarpVariant0;
        const int T = warp ? g->vslots[v] : group_tile(h->L, threads);
        if (T < 1) return fail(AM_ERR_ARG, "problem %d (q=%d, n=%d) does not fit a block of %d", i, h->pp.q, h->n, threads);
        FusedProblem &f = g->h_probs[i];
        f.cblob = h->d_blob;
        f.L = h->L;
        f.B = h->B;
        f.iters = iters;
        f.T = T;
        f.ntiles = (h->B + T - 1) / T;
        f.state = h->d_state;
        f.res = h->d_out;
        f.res_psi = h->d_out + h->B;
        f.cost = h->d_out + 2 * size_t(h->B);
        f.mind = h->d_out + 3 * size_t(h->B);
        f.hist = nullptr;
        f.err = h->d_err;  // a failed wait shows in the problem's own getters
        const size_t sm = warp ? warp_smem_bytes(h->L, T) : fused_smem_bytes(h->L, T);
        if (sm > g->vsmem[v]) g->vsmem[v] = sm;
    }
    // Tiles of the active problems: each problem gets a share of the SMs in
    // proportion to its work and tiles no larger than needed to cover that
    // share, so that a few small problems still spread over the whole GPU
    // (a lone problem gets the tile a single-problem solve would use).
    const std::vector<int> act = active_list(g);
    auto work = [&](int i) {
        const am_problem *h = g->probs[i];
        return double(h->B) * h->pp.q * (12.0 * h->pp.m * h->n + 250.0);
    };
    double total = 0;
    for (int i : act) total += work(i);
    for (int i : act) {
        FusedProblem &f = g->h_probs[i];
        double share = total > 0 ? sms * work(i) / total : 1.0;
        if (share < 1) share = 1;
        const int want = int(std::ceil(f.B / share));
        if (want >= 1 && want < f.T) {
            f.T = want;
            f.ntiles = (f.B + f.T - 1) / f.T;
        }
    }
    std::vector<std::pair<double, int>> order[kGroupVariants];
    for (int i : act) {
        const am_problem *h = g->probs[i];
        const double tile_cost = double(g->h_probs[i].T) * h->pp.q * (12.0 * h->pp.m * h->n + 250.0);
        order[problem_variant(h)].push_back({-tile_cost, i});
    }
    g->h_items.clear();
    for (int v = 0; v < kGroupVariants; ++v) {
        std::sort(order[v].begin(), order[v].end());
        g->offset[v] = int(g->h_items.size() / 2);
        for (auto &o : order[v])
            for (int t = 0; t < g->h_probs[o.second].ntiles; ++t) {
                g->h_items.push_back(o.second);
                g->h_items.push_back(t);
            }
        g->count[v] = int(g->h_items.size() / 2) - g->offset[v];
    }
    g->nitems = int(g->h_items.size() / 2);
    return AM_OK;
}

// Packs the header, descriptors, work lists and active list into the pinned
// staging area and uploads them with one copy, unless the device already
// holds the same bytes.  The staging area is rewritten only after the
// previous upload from it has completed (bounded wait).
int upload_work(am_group *g, cudaStream_t st)
{
    const std::vector<int> act = active_list(g);
    const size_t np = g->h_probs.size();
    // header: item count per variant, then list offset per variant
    const size_t o_probs = (2 * sizeof(int) * kGroupVariants + 63) & ~size_t(63);
    const size_t o_items = o_probs + ((sizeof(FusedProblem) * np + 15) & ~size_t(15));
    const size_t o_list = o_items + sizeof(int) * g->h_items.size();
    const size_t bytes = o_list + sizeof(int) * act.size();
    std::vector<char> buf(bytes, 0);
    std::memcpy(buf.data(), g->count, sizeof(g->count));
    std::memcpy(buf.data() + sizeof(int) * kGroupVariants, g->offset, sizeof(g->offset));
    std::memcpy(buf.data() + o_probs, g->h_probs.data(), sizeof(FusedProblem) * np);
    std::memcpy(buf.data() + o_items, g->h_items.data(), sizeof(int) * g->h_items.size());
    std::memcpy(buf.data() + o_list, act.data(), sizeof(int) * act.size());
    g->solved_list = act;
    if (buf == g->last_up) return AM_OK;
    if (g->up_pending) {
        int rc = wait_event(g->up_ev, st);
        if (rc) return rc;
        g->up_pending = false;
    }
    if (bytes > g->up_cap) {
        cudaFree(g->d_up);  // waits for the device: no kernel still reads it
        g->d_up = nullptr;
        g->up_cap = 0;
        CK(cudaMalloc(&g->d_up, bytes * 2), "group upload region");
        g->up_cap = bytes * 2;
    }
    if (bytes > g->h_up_cap) {
        if (g->h_up) cudaFreeHost(g->h_up);
        g->h_up = nullptr;
        g->h_up_cap = 0;
        CK(cudaMallocHost(&g->h_up, bytes * 2), "group staging area");
        g->h_up_cap = bytes * 2;
    }
    std::memcpy(g->h_up, buf.data(), bytes);
    CK(cudaMemcpyAsync(g->d_up, g->h_up, bytes, cudaMemcpyHostToDevice, st), "group upload");
    CK(cudaEventRecord(g->up_ev, st), "event record");
    g->up_pending = true;
    g->last_up.swap(buf);
    g->d_head = reinterpret_cast<int *>(g->d_up);
    g->d_probs = reinterpret_cast<FusedProblem *>(g->d_up + o_probs);
    g->d_items = reinterpret_cast<int *>(g->d_up + o_items);
    g->d_list = reinterpret_cast<int *>(g->d_up + o_list);
    return AM_OK;
}

// Issues the variant kernels of the mask: on the given stream when there is
// one variant, else forked onto the group's streams and joined back.
int issue_variants(am_group *g, uint64_t mask, int threads, int sms, bool fixed_grid, cudaStream_t st,
                   int *launches)
{
    const int nv = __builtin_popcountll(mask);
    GroupLaunch gl;
    gl.d_probs = g->d_probs;
    gl.d_items = g->d_items;
    gl.d_head = g->d_head;
    gl.d_ctl = g->d_ctl;
    gl.threads = threads;
    if (nv > 1) CK(cudaEventRecord(g->fork_ev, st), "fork");
    for (int v = 0; v < kGroupVariants; ++v) {
        if (!(mask >> v & 1ull)) continue;
        gl.variant = v;
        gl.smem = g->vsmem[v];
        gl.slots = g->vslots[v];
        gl.grid = fixed_grid || g->count[v] > sms ? sms : g->count[v];
        cudaStream_t s = st;
        if (nv > 1) {
            s = g->vst[v];
            CK(cudaStreamWaitEvent(s, g->fork_ev, 0), "fork wait");
        }
        const char *why = nullptr;
        const int rc = launch_group(gl, s, launches, &why);
        if (rc == -1) return fail(AM_ERR_ARG, "group does not fit the kernel");
        if (rc) return fail(AM_ERR_CUDA, "group launch failed (variant %d, %d threads, %zu B shared): %s", v,
                            threads, gl.smem, why ? why : "?");
        if (nv > 1) {
            CK(cudaEventRecord(g->join_ev[v], s), "join");
            CK(cudaStreamWaitEvent(st, g->join_ev[v], 0), "join wait");
        }
    }
    return AM_OK;
}

int group_launch(am_group *g, int iters, cudaStream_t st)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = g->threads > 0 ? g->threads : fused_max_threads();
    int rc = build_work(g, threads, iters, sms);
    if (rc) return rc;
    rc = upload_work(g, st);
    if (rc) return rc;
    uint64_t mask = 0;
    for (int v = 0; v < kGroupVariants; ++v)
        if (g->count[v] > 0) mask |= 1ull << v;
    if (!mask) return AM_OK;
    if (__builtin_popcountll(mask) > 1 && !g->vst[0]) {
        for (int v = 0; v < kGroupVariants; ++v) {
            CK(cudaStreamCreateWithFlags(&g->vst[v], cudaStreamNonBlocking), "stream creation");
            CK(cudaEventCreateWithFlags(&g->join_ev[v], cudaEventDisableTiming), "event creation");
        }
        CK(cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming), "event creation");
    }
    const bool graph = g->use_graph && st != nullptr;
    if (!graph) return issue_variants(g, mask, threads, sms, false, st, &g->launches);
    // A captured launch keeps its grids: one CTA per SM for each variant;
    // CTAs that find their list empty leave at once.
    am_group::Captured *hit = nullptr;
    for (auto &c : g->graphs)
        if (c.mask == mask && c.threads == threads && c.stream == st && c.up == g->d_up &&
            !std::memcmp(c.smem, g->vsmem, sizeof(c.smem)) && !std::memcmp(c.slots, g->vslots, sizeof(c.slots)))
            hit = &c;
    if (!hit) {
        // a server's rounds bring many variant sets: keep up to 64 graphs,
        // dropping the oldest
        if (g->graphs.size() >= 64) {
            cudaGraphExecDestroy(g->graphs.front().exec);
            g->graphs.erase(g->graphs.begin());
        }
        cudaGraph_t graph_obj = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
        rc = issue_variants(g, mask, threads, sms, true, st, nullptr);
        cudaError_t e = cudaStreamEndCapture(st, &graph_obj);
        if (rc || e != cudaSuccess) {
            if (graph_obj) cudaGraphDestroy(graph_obj);
            return rc ? rc : cuda_fail(e, "graph capture of the group launch");
        }
        am_group::Captured c;
        c.mask = mask;
        c.threads = threads;
        c.stream = st;
        c.up = g->d_up;
        std::memcpy(c.smem, g->vsmem, sizeof(c.smem));
        std::memcpy(c.slots, g->vslots, sizeof(c.slots));
        e = cudaGraphInstantiate(&c.exec, graph_obj, 0);
        cudaGraphDestroy(graph_obj);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        g->graphs.push_back(c);
        hit = &g->graphs.back();
    }
    CK(cudaGraphLaunch(hit->exec, st), "graph launch");
    g->launches += __builtin_popcountll(mask);
    return AM_OK;
}

}  // namespace

extern "C" {

int am_init_state(am_problem *h, int B, const float *init, const float *warm_lambda, void *stream,
                  int mem)
{
    if (!h || !init) return fail(AM_ERR_ARG, "null argument");
    if (B < 1 || B > (1 << 24)) return fail(AM_ERR_ARG, "B must be in [1, 2^24]");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    h->stream = static_cast<cudaStream_t>(stream);
    int rc = check_B(h, B);
    if (rc) return rc;
    // device inputs are read in place by the initial-state launch, which also
    // clears the results and the status word; host inputs are staged first
    const float *src = init, *warm = warm_lambda;
    if (mem == AM_HOST) {
        CK(cudaMemcpyAsync(h->d_in, init, sizeof(float) * 33 * B, cudaMemcpyHostToDevice, h->stream),
           "init copy");
        src = h->d_in;
        if (warm_lambda) {
            CK(cudaMemcpyAsync(h->d_in + 33 * size_t(B), warm_lambda, sizeof(float) * 55 * B,
                               cudaMemcpyHostToDevice, h->stream),
               "warm copy");
            warm = h->d_in + 33 * size_t(B);
        }
    }
    if (launch_init_state(h->d_state, src, warm, B, h->stream, nullptr, h->d_out, h->d_err))
        return fail(AM_ERR_CUDA, "init launch failed");
    h->B = B;
    h->solved = true;
    return AM_OK;
}

int am_resample(am_problem *h, unsigned long long seed, float sigma, void *stream)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (!(sigma >= 0.f) || !std::isfinite(sigma)) return fail(AM_ERR_ARG, "sigma must be finite and >= 0");
    if (!h->solved || h->B < 1) return fail(AM_ERR_STATE, "no state yet");
    h->stream = static_cast<cudaStream_t>(stream);
    NvtxRange nvtx("am_resample");
    ResampleArgs a;
    double Lc[25];
    init_cov_factor(Lc);
    for (int i = 0; i < 25; ++i) a.Lc[i] = float(Lc[i]);
    const float line[6] = {float(h->pp.x_bc[0]), float(h->pp.x_bc[3]), float(h->pp.y_bc[0]),
                           float(h->pp.y_bc[3]), float(h->pp.psi_bc[0]), float(h->pp.psi_bc[3])};
    std::memcpy(a.line, line, sizeof(line));
    a.sigma = sigma;
    a.seed = seed;
    a.B = h->B;
    if (launch_resample(h->d_state, a, h->stream, nullptr)) return fail(AM_ERR_CUDA, "resample launch failed");
    return AM_OK;
}

int am_shift(am_problem *h, double dt, void *stream)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (!(dt >= 0.0) || !(dt <= h->pp.T)) return fail(AM_ERR_ARG, "dt must be in [0, T]");
    if (!h->solved || h->B < 1) return fail(AM_ERR_STATE, "no state yet");
    h->stream = static_cast<cudaStream_t>(stream);
    NvtxRange nvtx("am_shift");
    double S[121];
    shift_matrix(dt / h->pp.T, S);
    ShiftArgs a;
    for (int i = 0; i < 121; ++i) a.S[i] = float(S[i]);
    a.B = h->B;
    if (launch_shift(h->d_state, a, h->stream, nullptr)) return fail(AM_ERR_CUDA, "shift launch failed");
    return AM_OK;
}

namespace {

// Float offsets of the CEM buffer for N samples.
struct CemLayout {
    size_t z, cost, dmin, mu, sig, chol, best, total;
};

CemLayout cem_layout(int N)
{
    CemLayout c;
    c.z = 0;
    c.cost = size_t(N) * 15;
    c.dmin = c.cost + N;
    c.mu = (c.dmin + N + 3) & ~size_t(3);
    c.sig = c.mu + 16;
    c.chol = c.sig + 228;
    c.best = c.chol + 228;
    c.total = c.best + 64;
    return c;
}

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

}  // namespace

int am_cem_solve(am_problem *h, const am_cem_desc *d, void *stream)
{
    if (!h || !d) return fail(AM_ERR_ARG, "null argument");
    if (d->samples < 16 || d->samples > 8192) return fail(AM_ERR_ARG, "samples must be in [16, 8192]");
    if (d->elites < 2 || d->elites > d->samples || d->elites > 1024)
        return fail(AM_ERR_ARG, "elites must be in [2, min(samples, 1024)]");
    if (d->iters < 1) return fail(AM_ERR_ARG, "iters must be >= 1");
    if (!finite_nonneg(d->sigma_xy) || !finite_nonneg(d->sigma_psi) || !finite_nonneg(d->w_coll) ||
        !finite_nonneg(d->w_bound))
        return fail(AM_ERR_ARG, "spreads and weights must be finite and >= 0");
    if (!(d->alpha > 0.f && d->alpha <= 1.f)) return fail(AM_ERR_ARG, "alpha must be in (0, 1]");
    if (!(d->reg > 0.f) || !std::isfinite(d->reg)) return fail(AM_ERR_ARG, "reg must be finite and > 0");
    if (d->warm) {
        if (!(d->warm_dt >= 0.0 && d->warm_dt <= h->pp.T)) return fail(AM_ERR_ARG, "warm_dt must be in [0, T]");
        for (int k = 0; k < 33; ++k)
            if (!std::isfinite(d->warm[k])) return fail(AM_ERR_ARG, "non-finite warm plan");
    }
    h->stream = static_cast<cudaStream_t>(stream);
    NvtxRange nvtx("am_cem_solve");
    const int N = d->samples;
    const CemLayout c = cem_layout(N);
    int rc = ensure(h->d_cem, h->cem_cap, c.total, "CEM buffers");
    if (rc) return rc;
    // starting distribution (FP64 on the host)
    double mu0[15];
    if (d->warm) {
        double S[121];
        shift_matrix(d->warm_dt / h->pp.T, S);
        for (int b = 0; b < 3; ++b)
            for (int i = 0; i < 5; ++i) {
                double v = 0.0;
                for (int j = 0; j < NV; ++j) v += S[(3 + i) * NV + j] * d->warm[11 * b + j];
                mu0[5 * b + i] = v;
            }
    } else {
        const double *bc[3] = {h->pp.x_bc, h->pp.y_bc, h->pp.psi_bc};
        for (int b = 0; b < 3; ++b)
            for (int i = 0; i < 5; ++i) mu0[5 * b + i] = bc[b][0] + (bc[b][3] - bc[b][0]) * (i + 1) / 6.0;
    }
    double Lc[25];
    init_cov_factor(Lc);
    std::vector<float> up(c.total - c.mu, 0.f);
    float *mu = up.data(), *sig = mu + (c.sig - c.mu), *chol = mu + (c.chol - c.mu), *best = mu + (c.best - c.mu);
    for (int k = 0; k < 15; ++k) mu[k] = float(mu0[k]);
    for (int b = 0; b < 3; ++b) {
        const double s = b < 2 ? d->sigma_xy : d->sigma_psi;
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double cov = 0.0;
                for (int k = 0; k < 5; ++k) cov += Lc[i * 5 + k] * Lc[j * 5 + k];
                sig[(5 * b + i) * 15 + 5 * b + j] = float(s * s * cov);
                chol[(5 * b + i) * 15 + 5 * b + j] = float(s * Lc[i * 5 + j]);
            }
    }
    best[15] = FLT_MAX;
    CK(cudaMemcpyAsync(h->d_cem + c.mu, up.data(), sizeof(float) * up.size(), cudaMemcpyHostToDevice, h->stream),
       "CEM start copy");
    CemArgs a;
    a.cblob = h->d_blob;
    a.L = h->L;
    a.z = h->d_cem + c.z;
    a.cost = h->d_cem + c.cost;
    a.dmin = h->d_cem + c.dmin;
    a.mu = h->d_cem + c.mu;
    a.sig = h->d_cem + c.sig;
    a.chol = h->d_cem + c.chol;
    a.best = h->d_cem + c.best;
    a.given = nullptr;
    a.N = N;
    a.K = d->elites;
    a.NP = 1;
    while (a.NP < N) a.NP <<= 1;
    a.seed = d->seed;
    a.w_coll = d->w_coll;
    a.w_bound = d->w_bound;
    a.alpha = d->alpha;
    a.reg = d->reg;
    h->cem_N = 0;
    for (int it = 0; it < d->iters; ++it) {
        a.iter = it;
        if (launch_cem_score(a, h->stream) || launch_cem_refit(a, h->stream))
            return fail(AM_ERR_CUDA, "CEM launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    h->cem_N = N;
    return AM_OK;
}

int am_cem_get_best(am_problem *h, float coeffs[33], float *cost, float *min_dist)
{
    if (!h || !coeffs) return fail(AM_ERR_ARG, "null argument");
    if (h->cem_N < 1) return fail(AM_ERR_STATE, "no CEM run yet");
    const CemLayout c = cem_layout(h->cem_N);
    float b[64];
    CK(cudaMemcpyAsync(b, h->d_cem + c.best, sizeof(b), cudaMemcpyDeviceToHost, h->stream), "CEM best copy");
    int rc = wait_stream(h);
    if (rc) return rc;
    std::memcpy(coeffs, b + 17, 33 * sizeof(float));
    if (cost) *cost = b[15];
    if (min_dist) *min_dist = b[16];
    return b[15] < FLT_MAX ? AM_OK : fail(AM_ERR_NAN, "every CEM sample scored non-finite");
}

int am_cem_get_samples(am_problem *h, float *z, float *cost, float *mu, float *sigma)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (h->cem_N < 1) return fail(AM_ERR_STATE, "no CEM run yet");
    const int N = h->cem_N;
    const CemLayout c = cem_layout(N);
    if (z) CK(cudaMemcpyAsync(z, h->d_cem + c.z, sizeof(float) * 15 * N, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (cost) CK(cudaMemcpyAsync(cost, h->d_cem + c.cost, sizeof(float) * N, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (mu) CK(cudaMemcpyAsync(mu, h->d_cem + c.mu, sizeof(float) * 15, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (sigma) CK(cudaMemcpyAsync(sigma, h->d_cem + c.sig, sizeof(float) * 225, cudaMemcpyDeviceToHost, h->stream), "copy");
    return wait_stream(h);
}

int am_cem_score(am_problem *h, int count, const float *coeffs, float w_coll, float w_bound, float *cost,
                 float *min_dist)
{
    if (!h || !coeffs || !cost || !min_dist) return fail(AM_ERR_ARG, "null argument");
    if (count < 1 || count > 8192) return fail(AM_ERR_ARG, "count must be in [1, 8192]");
    if (!finite_nonneg(w_coll) || !finite_nonneg(w_bound)) return fail(AM_ERR_ARG, "weights must be finite and >= 0");
    for (size_t k = 0; k < size_t(count) * 33; ++k)
        if (!std::isfinite(coeffs[k])) return fail(AM_ERR_ARG, "non-finite coefficient");
    int rc = ensure(h->d_score, h->score_cap, size_t(count) * 35, "CEM score buffers");
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->d_score, coeffs, sizeof(float) * 33 * count, cudaMemcpyHostToDevice, h->stream),
       "plan copy");
    CemArgs a{};
    a.cblob = h->d_blob;
    a.L = h->L;
    a.given = h->d_score;
    a.cost = h->d_score + size_t(33) * count;
    a.dmin = a.cost + count;
    a.N = count;
    a.w_coll = w_coll;
    a.w_bound = w_bound;
    if (launch_cem_score(a, h->stream)) return fail(AM_ERR_CUDA, "score launch failed");
    CK(cudaMemcpyAsync(cost, a.cost, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream), "copy");
    CK(cudaMemcpyAsync(min_dist, a.dmin, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream), "copy");
    return wait_stream(h);
}

int am_scale_multipliers(am_problem *h, float factor, void *stream)
{
    if (!h) return fail(AM_ERR_ARG, "null handle");
    if (!(factor >= 0.f) || !std::isfinite(factor)) return fail(AM_ERR_ARG, "factor must be finite and >= 0");
    if (!h->solved || h->B < 1) return fail(AM_ERR_STATE, "no state yet");
    h->stream = static_cast<cudaStream_t>(stream);
    if (factor == 1.f) return AM_OK;
    if (factor == 0.f) {
        // entries 55..109 of every trajectory's state: one strided memset
        CK(cudaMemset2DAsync(h->d_state + 55, STATE * sizeof(float), 0, 55 * sizeof(float), h->B, h->stream),
           "multiplier reset");
        return AM_OK;
    }
    if (launch_scale_multipliers(h->d_state, h->B, factor, h->stream, nullptr))
        return fail(AM_ERR_CUDA, "multiplier scaling launch failed");
    return AM_OK;
}

int am_plan_eval(const float coeffs[33], double T, int count, const double *t, double *out)
{
    if (!coeffs || count < 0 || (count > 0 && (!t || !out))) return fail(AM_ERR_ARG, "null argument");
    if (!(T > 0) || !std::isfinite(T)) return fail(AM_ERR_ARG, "T must be finite and > 0");
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(t[i])) return fail(AM_ERR_ARG, "non-finite time %d", i);
    for (int k = 0; k < 33; ++k)
        if (!std::isfinite(coeffs[k])) return fail(AM_ERR_ARG, "non-finite coefficient %d", k);
    for (int i = 0; i < count; ++i)
        for (int s = 0; s < 3; ++s) bernstein_eval(coeffs + 11 * s, T, t[i], out + 9 * i + 3 * s);
    return AM_OK;
}

int am_group_create(am_problem *const *problems, int count, am_group **out)
{
    if (!problems || !out || count < 1) return fail(AM_ERR_ARG, "need at least one problem");
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!problems[i]) return fail(AM_ERR_ARG, "null problem %d", i);
    }
    am_group *g = new (std::nothrow) am_group;
    if (!g) return fail(AM_ERR_ARG, "out of host memory");
    g->probs.assign(problems, problems + count);
    int rc = ensure(g->d_ctl, g->ctl_cap, 2 * kGroupVariants, "work counters");
    if (!rc && cudaMemset(g->d_ctl, 0, 2 * kGroupVariants * sizeof(int)) != cudaSuccess)
        rc = fail(AM_ERR_CUDA, "memset");
    if (!rc && cudaEventCreateWithFlags(&g->up_ev, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(AM_ERR_CUDA, "event creation failed");
    if (!rc && cudaMallocHost(&g->h_status, 2 * kGroupVariants * sizeof(int)) != cudaSuccess)
        rc = fail(AM_ERR_CUDA, "pinned alloc");
    if (!rc && cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(AM_ERR_CUDA, "event creation failed");
    if (rc) {
        am_group_destroy(g);
        return rc;
    }
    *out = g;
    return AM_OK;
}

void am_group_destroy(am_group *g)
{
    if (!g) return;
    drop_graph(g);
    cudaFree(g->d_up);
    if (g->h_up) cudaFreeHost(g->h_up);
    cudaFree(g->d_ctl);
    if (g->h_status) cudaFreeHost(g->h_status);
    if (g->ev) cudaEventDestroy(g->ev);
    if (g->up_ev) cudaEventDestroy(g->up_ev);
    for (int v = 0; v < kGroupVariants; ++v) {
        if (g->vst[v]) cudaStreamDestroy(g->vst[v]);
        if (g->join_ev[v]) cudaEventDestroy(g->join_ev[v]);
    }
    if (g->fork_ev) cudaEventDestroy(g->fork_ev);
    cudaFree(g->d_bests);
    cudaFree(g->d_save);
    delete g;
}

int am_group_set_option(am_group *g, int option, int value)
{
    if (!g) return fail(AM_ERR_ARG, "null group");
    if (option == AM_GOPT_THREADS) {
        if (value != 0 && (value < 32 || value > fused_max_threads() || value % 32))
            return fail(AM_ERR_ARG, "threads must be 0 or a multiple of 32 up to %d", fused_max_threads());
        g->threads = value;
        return AM_OK;
    }
    if (option == AM_GOPT_GRAPH) {
        g->use_graph = value != 0;
        if (!g->use_graph) drop_graph(g);
        return AM_OK;
    }
    if (option == AM_GOPT_WARP_SLOTS) {
        if (value < 0 || value > AM_GROUP_MAX_WARP_SLOTS)
            return fail(AM_ERR_ARG, "warp slots must be in [0, %d]", AM_GROUP_MAX_WARP_SLOTS);
        g->warp_slots = value;
        return AM_OK;
    }
    return fail(AM_ERR_ARG, "unknown group option %d", option);
}

int am_group_get_option(am_group *g, int option, int *value)
{
    if (!g || !value) return fail(AM_ERR_ARG, "null argument");
    if (option == AM_GOPT_THREADS) *value = g->threads;
    else if (option == AM_GOPT_GRAPH) *value = g->use_graph ? 1 : 0;
    else if (option == AM_GOPT_WARP_SLOTS) *value = g->warp_slots;
    else return fail(AM_ERR_ARG, "unknown group option %d", option);
    return AM_OK;
}

int am_group_set_active(am_group *g, const int *idx, int count)
{
    if (!g) return fail(AM_ERR_ARG, "null group");
    if (count < 0 || (count > 0 && !idx)) return fail(AM_ERR_ARG, "bad active list");
    std::vector<char> seen(g->probs.size(), 0);
    for (int k = 0; k < count; ++k) {
        if (idx[k] < 0 || idx[k] >= int(g->probs.size())) return fail(AM_ERR_ARG, "problem index %d out of range", idx[k]);
        if (seen[idx[k]]) return fail(AM_ERR_ARG, "problem %d listed twice", idx[k]);
        seen[idx[k]] = 1;
    }
    g->active.assign(idx, idx + count);
    return AM_OK;
}

int am_group_solve(am_group *g, int iters, void *stream)
{
    NvtxRange range("am_group_solve");
    if (!g) return fail(AM_ERR_ARG, "null group");
    if (iters < 1 || iters > 100000) return fail(AM_ERR_ARG, "iters must be in [1, 100000]");
    const std::vector<int> act = active_list(g);
    for (int i : act)
        if (!g->probs[i]->solved) return fail(AM_ERR_STATE, "problem %d has no state (am_init_state)", i);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int before = g->launches;
    int rc = group_launch(g, iters, st);
    if (rc) return rc;
    for (int i : act) {
        g->probs[i]->stream = st;
        g->probs[i]->launches = g->launches - before;
    }
    return AM_OK;
}

int am_group_get_best(am_group *g, float *out, int mem, void *stream)
{
    if (!g || !out) return fail(AM_ERR_ARG, "null argument");
    if (mem != AM_HOST && mem != AM_DEVICE) return fail(AM_ERR_ARG, "bad mem flag");
    const std::vector<int> act = active_list(g);
    for (int i : act)
        if (!g->probs[i]->solved) return fail(AM_ERR_STATE, "problem %d has no state", i);
    if (!g->d_up) return fail(AM_ERR_STATE, "no group solve yet");
    if (act != g->solved_list) return fail(AM_ERR_STATE, "the active list changed since the last solve");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure(g->d_bests, g->bests_cap, 36 * act.size(), "best records");
    if (rc) return rc;
    if (launch_group_argmin(g->d_probs, g->d_list, int(act.size()), g->d_bests, st, &g->launches))
        return fail(AM_ERR_CUDA, "best selection launch failed");
    CK(cudaMemcpyAsync(out, g->d_bests, sizeof(float) * 36 * act.size(), kind_out(mem), st), "best copy");
    if (mem == AM_DEVICE) return AM_OK;
    CK(cudaMemcpyAsync(g->h_status, g->d_ctl, 2 * kGroupVariants * sizeof(int), cudaMemcpyDeviceToHost, st),
       "status copy");
    rc = wait_event(g->ev, st);
    if (rc) return rc;
    for (int v = 0; v < kGroupVariants; ++v)
        if (g->h_status[2 * v + 1]) return fail(AM_ERR_TIMEOUT, "a kernel of the group gave up a bounded wait");
    return AM_OK;
}

}  // extern "C"

namespace trajam {

int group_best_async(::am_group *g, float *h_out, void *stream)
{
    const std::vector<int> act = active_list(g);
    if (!g->d_up || act != g->solved_list) return fail(AM_ERR_STATE, "no group solve of this active list");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure(g->d_bests, g->bests_cap, 36 * act.size(), "best records");
    if (rc) return rc;
    if (launch_group_argmin(g->d_probs, g->d_list, int(act.size()), g->d_bests, st, &g->launches))
        return fail(AM_ERR_CUDA, "best selection launch failed");
    CK(cudaMemcpyAsync(h_out, g->d_bests, sizeof(float) * 36 * act.size(), cudaMemcpyDeviceToHost, st), "best copy");
    CK(cudaMemcpyAsync(g->h_status, g->d_ctl, 2 * kGroupVariants * sizeof(int), cudaMemcpyDeviceToHost, st),
       "status copy");
    return AM_OK;
}

int group_status(const ::am_group *g)
{
    for (int v = 0; v < kGroupVariants; ++v)
        if (g->h_status[2 * v + 1]) return fail(AM_ERR_TIMEOUT, "a kernel of the group gave up a bounded wait");
    return AM_OK;
}

int problem_status_async(::am_problem *h, void *stream)
{
    int *h_err = reinterpret_cast<int *>(h->h_best + 40);
    CK(cudaMemcpyAsync(h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)),
       "status read");
    return AM_OK;
}

int problem_status(const ::am_problem *h)
{
    return status_error(reinterpret_cast<const int *>(h->h_best + 40)[0]);
}

}  // namespace trajam

extern "C" {

int am_group_autotune(am_group *g, int iters, void *stream, int *threads_out, float *ms_out)
{
    if (!g) return fail(AM_ERR_ARG, "null group");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Solves advance the states: keep copies and put them back afterwards.
    size_t total = 0;
    for (am_problem *h : g->probs) total += size_t(h->B) * STATE;
    int rc = ensure(g->d_save, g->save_cap, total, "tuning copies");
    if (rc) return rc;
    size_t o = 0;
    for (am_problem *h : g->probs) {
        CK(cudaMemcpyAsync(g->d_save + o, h->d_state, sizeof(float) * STATE * h->B,
                           cudaMemcpyDeviceToDevice, st), "save state");
        o += size_t(h->B) * STATE;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved = g->threads, saved_slots = g->warp_slots;
    bool has_small = false, has_warp = false;
    for (const am_problem *h : g->probs) (problem_variant(h) >= kGroupWarpVariant0 ? has_warp : has_small) = true;
    // average time of three solves in the current settings (a warm-up, which
    // also captures the graph, first); < 0 when they do not run
    auto time_solves = [&]() -> float {
        if (build_work(g, g->threads > 0 ? g->threads : fused_max_threads(), iters, sms) != AM_OK) return -1.f;
        if (am_group_solve(g, iters, stream) != AM_OK) return -1.f;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) am_group_solve(g, iters, stream);
        cudaEventRecord(e1, st);
        if (wait_event(g->ev, st) != AM_OK) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 3.f;
    };
    // the small-tile variants' block size (the warp-pair variants' block is
    // their slot count times 32 NW and does not depend on it)
    int best = 0;
    float best_ms = 1e30f;
    for (int threads = 128; threads <= fused_max_threads(); threads += 64) {
        if (!has_small && threads != fused_max_threads()) continue;
        g->threads = threads;
        const float ms = time_solves();
        if (ms >= 0.f && ms < best_ms) {
            best_ms = ms;
            best = threads;
        }
    }
    g->threads = best ? best : saved;
    // then the warp-pair variants' trajectory slots per CTA: as many as fit
    // (0), or at most 7 .. 3
    int best_slots = saved_slots;
    if (has_warp && best) {
        float slots_ms = 1e30f;
        for (int cap : {0, 7, 6, 5, 4, 3}) {
            g->warp_slots = cap;
            const float ms = time_solves();
            if (ms >= 0.f && ms < slots_ms) {
                slots_ms = ms;
                best_slots = cap;
            }
        }
        if (slots_ms < 1e30f) best_ms = slots_ms;
    }
    g->warp_slots = best_slots;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    o = 0;
    for (am_problem *h : g->probs) {
        CK(cudaMemcpyAsync(h->d_state, g->d_save + o, sizeof(float) * STATE * h->B,
                           cudaMemcpyDeviceToDevice, st), "restore state");
        o += size_t(h->B) * STATE;
    }
    rc = wait_event(g->ev, st);
    if (rc) return rc;
    if (!best) return fail(AM_ERR_ARG, "no block size fits every problem of the group");
    if (threads_out) *threads_out = best;
    if (ms_out) *ms_out = best_ms;
    return AM_OK;
}

int am_group_stats(am_group *g, int *launches, int *items)
{
    if (!g) return fail(AM_ERR_ARG, "null group");
    if (launches) *launches = g->launches;
    if (items) *items = g->nitems;
    return AM_OK;
}

}  // extern "C"

namespace trajam {

int problem_shape(const ::am_problem *h, int *q, int *m, int *n, int *B, double *T)
{
    *q = h->pp.q;
    *m = h->pp.m;
    *n = h->n;
    *B = h->B;
    *T = h->pp.T;
    return h->solved ? 0 : -1;
}

void problem_boundary(const ::am_problem *h, double x[6], double y[6], double psi[6])
{
    std::memcpy(x, h->pp.x_bc, sizeof(h->pp.x_bc));
    std::memcpy(y, h->pp.y_bc, sizeof(h->pp.y_bc));
    std::memcpy(psi, h->pp.psi_bc, sizeof(h->pp.psi_bc));
}

int problem_update_tracks(::am_problem *h, const float *xo, const float *yo)
{
    const int n = h->n, q = h->pp.q;
    if (n == 0) return AM_OK;
    if (!h->d_raw) return fail(AM_ERR_STATE, "no obstacles set");
    CK(cudaMemcpyAsync(h->d_raw, xo, sizeof(float) * n * q, cudaMemcpyHostToDevice, h->stream), "track copy");
    CK(cudaMemcpyAsync(h->d_raw + n * q, yo, sizeof(float) * n * q, cudaMemcpyHostToDevice, h->stream),
       "track copy");
    if (launch_prep_obstacles(h->d_blob, h->L, h->d_raw, h->d_raw + n * q, h->d_raw + 2 * n * q,
                              h->d_raw + 2 * n * q + n, float(h->pp.r_c), h->stream, nullptr))
        return fail(AM_ERR_CUDA, "obstacle preparation launch failed");
    return AM_OK;
}

size_t problem_device_bytes(const ::am_problem *h)
{
    return sizeof(float) * (h->blob_cap + h->raw_cap + h->state_cap + h->out_cap + h->best_cap +
                            h->in_cap + h->hist_cap + h->scratch_cap) +
           sizeof(int) * h->err_cap;
}

size_t scene_bytes(int q, int m, int n, int B)
{
    const ConstLayout L = make_layout(q, m, n);
    const size_t floats = size_t(L.total) + size_t(2 * n * q + 2 * n) + size_t(B) * (STATE + 4 + 33 + 55) + 64;
    return floats * sizeof(float) + sizeof(int);
}

}  // namespace trajam
