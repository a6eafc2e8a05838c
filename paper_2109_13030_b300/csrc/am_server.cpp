// Re-planning server (include/trajam.h, "serving"): resident warm-started
// scenes, HBM-budget admission, and a worker thread that keeps up to `lanes`
// rounds of continuous batching in flight, each a grouped launch (or a
// scene's own kernel) on its own stream, admitting new requests while
// earlier rounds run.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "am_internal.h"
#include "../../include/trajam.h"

using namespace trajam;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    long long ticket;
    am_request r;
    std::vector<float> xo, yo;
    double t_submit;
};

struct Scene {
    am_problem *h;
    int q, m, n, B;
    double T;
    size_t bytes;
    bool has_best = false;
    float best[33];
};

// One round in flight: its stream, group (a grouped launch touches the
// group's own device buffers, so each lane has one), pinned best records and
// completion event.
struct Lane {
    cudaStream_t st = nullptr;
    am_group *g = nullptr;
    float *h_bests = nullptr;  // 36 floats per request of the round
    cudaEvent_t ev = nullptr;
    std::vector<Request> batch;
    bool busy = false, grouped = false;
    bool dead = false;  // its round ran out of time: the stream may still write, never reused
    int rc = AM_OK;
    double t_start = 0;
};

constexpr int kMaxLanes = 8;
// A round still running after this long completes with AM_ERR_TIMEOUT.
constexpr double kRoundLimitS = 60.0;

}  // namespace

struct am_server {
    am_server_desc d;
    int device = 0;
    cudaStream_t st = nullptr;   // scene admission (cold starts) and autotuning
    std::vector<Scene> scenes;
    size_t used = 0;
    std::vector<Lane> lanes;
    std::vector<char> in_flight;  // per scene
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::unordered_map<long long, am_result> done;
    std::unordered_set<long long> outstanding;
    long long next_ticket = 1, rounds = 0, completed = 0;
    bool stop = false, started = false;
};

namespace {

// New boundary conditions of a request: the start state from the scene's
// last best plan at t = advance, and/or the goal state given with it.
int update_boundary(Scene &sc, const am_request &r)
{
    const bool adv = r.advance > 0 && sc.has_best, goal = (r.flags & AM_REQ_GOAL) != 0;
    if (!adv && !goal) return AM_OK;
    double x[6], y[6], psi[6];
    problem_boundary(sc.h, x, y, psi);
    if (adv) {
        bernstein_eval(sc.best, sc.T, r.advance, x);
        bernstein_eval(sc.best + 11, sc.T, r.advance, y);
        bernstein_eval(sc.best + 22, sc.T, r.advance, psi);
    }
    if (goal) {
        std::memcpy(x + 3, r.goal, 3 * sizeof(double));
        std::memcpy(y + 3, r.goal + 3, 3 * sizeof(double));
        std::memcpy(psi + 3, r.goal + 6, 3 * sizeof(double));
    }
    return am_set_boundary(sc.h, x, y, psi);
}

// Queues one round on the lane's stream: each request's updates, the solve
// (one grouped launch for several scenes, a scene's own kernel for one, one
// solve per request in the sequential mode), the best selection and the
// copy of the best records and status words to pinned memory, then the
// lane's event.  Nothing here waits for the device.
void issue_round(am_server *s, Lane &ln)
{
    int rc = AM_OK;
    ln.t_start = now_s();
    for (auto &q : ln.batch) {
        Scene &sc = s->scenes[q.r.scene];
        rc = am_set_stream(sc.h, ln.st);
        if (!rc && !q.xo.empty()) rc = problem_update_tracks(sc.h, q.xo.data(), q.yo.data());
        if (!rc) rc = update_boundary(sc, q.r);
        if (!rc && (q.r.flags & AM_REQ_RESAMPLE)) rc = am_resample(sc.h, q.r.seed, q.r.sigma, ln.st);
        else if (!rc && (q.r.flags & AM_REQ_SHIFT) && q.r.advance > 0 && sc.has_best)
            rc = am_shift(sc.h, q.r.advance, ln.st);  // re-timed together with the start state
        if (!rc && (q.r.flags & AM_REQ_SCALE_LAMBDA)) rc = am_scale_multipliers(sc.h, q.r.lambda_scale, ln.st);
        if (rc) break;
    }
    ln.grouped = !rc && s->d.mode == AM_SRV_BATCHED && ln.batch.size() > 1;
    if (ln.grouped) {
        std::vector<int> act;
        for (auto &q : ln.batch) act.push_back(q.r.scene);
        rc = am_group_set_active(ln.g, act.data(), int(act.size()));
        if (!rc) rc = am_group_solve(ln.g, s->d.iters, ln.st);
        if (!rc) rc = group_best_async(ln.g, ln.h_bests, ln.st);
    } else {
        for (size_t k = 0; k < ln.batch.size() && !rc; ++k) {
            Scene &sc = s->scenes[ln.batch[k].r.scene];
            rc = am_solve_batch(sc.h, sc.B, nullptr, nullptr, s->d.iters, ln.st, AM_DEVICE);
            if (!rc) rc = am_get_best_async(sc.h, ln.h_bests + 36 * k, AM_HOST, ln.st);
            if (!rc) rc = problem_status_async(sc.h, ln.st);
        }
    }
    if (cudaEventRecord(ln.ev, ln.st) != cudaSuccess && !rc) rc = AM_ERR_CUDA;
    ln.rc = rc;
    ln.busy = true;
}

// Completes a finished round (its event passed, or it failed): results,
// the scenes' last best plans, and the scenes leave the in-flight set.
void complete_round(am_server *s, Lane &ln, int rc)
{
    if (!rc && ln.grouped) rc = group_status(ln.g);
    if (!rc && !ln.grouped)
        for (auto &q : ln.batch)
            if (!rc) rc = problem_status(s->scenes[q.r.scene].h);
    const double t_done = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t k = 0; k < ln.batch.size(); ++k) {
        Request &q = ln.batch[k];
        am_result r;
        std::memset(&r, 0, sizeof(r));
        r.status = rc;
        r.t_submit = q.t_submit;
        r.t_start = ln.t_start;
        r.t_done = t_done;
        r.round = s->rounds;
        r.batch = int(ln.batch.size());
        if (!rc) {
            const float *o = ln.h_bests + 36 * k;
            r.index = int(o[0]);
            r.cost = o[1];
            r.residual = o[2];
            std::memcpy(r.coeffs, o + 3, sizeof(r.coeffs));
            if (!std::isfinite(r.cost)) {
                r.status = AM_ERR_NAN;  // every trajectory of the scene is non-finite
            } else {
                Scene &sc = s->scenes[q.r.scene];
                std::memcpy(sc.best, r.coeffs, sizeof(sc.best));
                sc.has_best = true;
            }
        }
        s->in_flight[q.r.scene] = 0;
        s->done[q.ticket] = r;
        ++s->completed;
    }
    ++s->rounds;
    ln.batch.clear();
    ln.busy = false;
    s->cv_done.notify_all();
}

// A round groups several scenes only when at least this many requests are
// admissible.  Measured on the serving mix (30 iterations, device time per
// round): two scenes cost the same grouped as one launch each (0.69 ms both
// on the small-tile kernels, 0.41 against 0.38 ms on the warp-pair ones),
// and the grouped round adds host work; from four scenes on grouping is
// cheaper (1.09 against 1.22 ms, 0.75 against 0.78 ms).  Below the threshold
// a round takes one request, and the next request goes to the next free
// lane, where it runs beside the first and completes on its own.
constexpr size_t kGroupMinRequests = 3;

// Takes the next round's requests: at most one per scene, oldest first,
// scenes in flight skipped; one request unless at least kGroupMinRequests
// are admissible.  Called with the lock held.
void take_batch(am_server *s, std::vector<Request> &batch, std::vector<char> &taken)
{
    const size_t nsc = s->scenes.size();
    size_t limit = s->d.mode == AM_SRV_SEQUENTIAL ? 1 : nsc;
    if (s->d.max_batch > 0 && size_t(s->d.max_batch) < limit) limit = size_t(s->d.max_batch);
    std::fill(taken.begin(), taken.end(), 0);
    if (limit > 1) {
        size_t admissible = 0;
        for (const Request &q : s->pending)
            if (!taken[q.r.scene] && !s->in_flight[q.r.scene]) {
                taken[q.r.scene] = 1;
                if (++admissible >= kGroupMinRequests) break;
            }
        if (admissible < kGroupMinRequests) limit = 1;
        std::fill(taken.begin(), taken.end(), 0);
    }
    for (auto it = s->pending.begin(); it != s->pending.end() && batch.size() < limit;) {
        const int sc = it->r.scene;
        if (!taken[sc] && !s->in_flight[sc]) {
            taken[sc] = 1;
            s->in_flight[sc] = 1;
            batch.push_back(std::move(*it));
            it = s->pending.erase(it);
        } else {
            ++it;
        }
    }
}

bool admissible(const am_server *s)
{
    for (const Request &q : s->pending)
        if (!s->in_flight[q.r.scene]) return true;
    return false;
}

void worker_main(am_server *s)
{
    cudaSetDevice(s->device);
    std::vector<char> taken(s->scenes.size());
    bool stopping = false;
    for (;;) {
        bool busy = false, progressed = false;
        // rounds that finished (or ran out of time) complete first
        for (Lane &ln : s->lanes) {
            if (!ln.busy) continue;
            const cudaError_t e = cudaEventQuery(ln.ev);
            if (e == cudaErrorNotReady) {
                if (now_s() - ln.t_start > kRoundLimitS) {
                    complete_round(s, ln, AM_ERR_TIMEOUT);
                    ln.dead = true;
                    progressed = true;
                } else {
                    busy = true;
                }
                continue;
            }
            complete_round(s, ln, e == cudaSuccess ? ln.rc : AM_ERR_CUDA);
            progressed = true;
        }
        // then every free lane takes a round of what is admissible
        if (!stopping) {
            for (Lane &ln : s->lanes) {
                if (ln.busy || ln.dead) continue;
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    if (s->stop) {
                        stopping = true;
                        break;
                    }
                    take_batch(s, ln.batch, taken);
                }
                if (ln.batch.empty()) break;
                issue_round(s, ln);
                busy = progressed = true;
            }
        }
        if (stopping && !busy) break;
        if (progressed) continue;
        bool live = false;
        for (const Lane &ln : s->lanes) live = live || !ln.dead;
        if (!live) break;  // every lane ran out of time: what is queued fails below
        if (busy) {
            // rounds in flight: poll their events (a request arriving now
            // waits for a free lane, at most one round)
            std::this_thread::yield();
            continue;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_work.wait(lk, [&] { return s->stop || admissible(s); });
        if (s->stop) stopping = true;
    }
    // Stopped: what is still queued completes with AM_ERR_STATE.
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &q : s->pending) {
        am_result r;
        std::memset(&r, 0, sizeof(r));
        r.status = AM_ERR_STATE;
        r.t_submit = q.t_submit;
        s->done[q.ticket] = r;
    }
    s->pending.clear();
    s->cv_done.notify_all();
}

void free_lanes(am_server *s)
{
    for (Lane &ln : s->lanes) {
        if (ln.g) am_group_destroy(ln.g);
        if (ln.h_bests) cudaFreeHost(ln.h_bests);
        if (ln.ev) cudaEventDestroy(ln.ev);
        if (ln.st) cudaStreamDestroy(ln.st);
    }
    s->lanes.clear();
}

}  // namespace

extern "C" {

size_t am_scene_bytes(int q, int m, int n, int B)
{
    if (q < 2 || q > AM_MAX_Q || m < 1 || m > AM_MAX_M || n < 0 || n > AM_MAX_N || B < 1) return 0;
    return scene_bytes(q, m, n, B);
}

int am_server_create(const am_server_desc *d, am_server **out)
{
    if (!d || !out) return report_error(AM_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->iters < 1 || d->iters > 100000) return report_error(AM_ERR_ARG, "iters must be in [1, 100000]");
    if (d->mode != AM_SRV_BATCHED && d->mode != AM_SRV_SEQUENTIAL) return report_error(AM_ERR_ARG, "bad mode");
    if (d->max_batch < 0 || d->max_pending < 0 || d->lanes < 0) return report_error(AM_ERR_ARG, "negative limit");
    if (d->lanes > kMaxLanes) return report_error(AM_ERR_ARG, "at most 8 lanes");
    am_server *s = new (std::nothrow) am_server;
    if (!s) return report_error(AM_ERR_ARG, "out of host memory");
    s->d = *d;
    if (s->d.max_pending == 0) s->d.max_pending = 65536;
    if (s->d.mode == AM_SRV_SEQUENTIAL) s->d.lanes = 1;
    else if (s->d.lanes == 0) s->d.lanes = 2;
    cudaGetDevice(&s->device);
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return report_error(AM_ERR_CUDA, "stream creation failed");
    }
    *out = s;
    return AM_OK;
}

int am_server_add_scene(am_server *s, am_problem *h, int B, const float *init, int mem, int *scene)
{
    if (!s || !h || !init || !scene) return report_error(AM_ERR_ARG, "null argument");
    if (s->started) return report_error(AM_ERR_STATE, "scenes are added before am_server_start");
    Scene sc;
    sc.h = h;
    int b0;
    problem_shape(h, &sc.q, &sc.m, &sc.n, &b0, &sc.T);
    if (B < 1 || B > (1 << 24)) return report_error(AM_ERR_ARG, "B must be in [1, 2^24]");
    for (const Scene &o : s->scenes)
        if (o.h == h) return report_error(AM_ERR_ARG, "handle already added");
    sc.B = B;
    sc.bytes = scene_bytes(sc.q, sc.m, sc.n, B);
    if (s->used + sc.bytes > s->d.budget_bytes) {
        char msg[160];
        snprintf(msg, sizeof(msg), "scene needs %zu bytes, %zu of the %zu-byte budget are in use", sc.bytes,
                 s->used, s->d.budget_bytes);
        return report_error(AM_ERR_BUDGET, msg);
    }
    int rc = am_init_state(h, B, init, nullptr, s->st, mem);
    if (rc) return rc;
    s->used += sc.bytes;
    s->scenes.push_back(sc);
    *scene = int(s->scenes.size()) - 1;
    return AM_OK;
}

int am_server_start(am_server *s)
{
    if (!s) return report_error(AM_ERR_ARG, "null server");
    if (s->started) return report_error(AM_ERR_STATE, "already started");
    if (s->scenes.empty()) return report_error(AM_ERR_STATE, "no scenes");
    std::vector<am_problem *> hs;
    for (auto &sc : s->scenes) hs.push_back(sc.h);
    int threads = 0;
    s->lanes.resize(size_t(s->d.lanes));
    for (size_t k = 0; k < s->lanes.size(); ++k) {
        Lane &ln = s->lanes[k];
        int rc = AM_OK;
        if (cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&ln.h_bests, sizeof(float) * 36 * s->scenes.size()) != cudaSuccess)
            rc = report_error(AM_ERR_CUDA, "lane set-up failed");
        if (!rc && s->d.mode == AM_SRV_BATCHED) {
            rc = am_group_create(hs.data(), int(hs.size()), &ln.g);
            // the block size is tuned once (on the admission stream) and shared
            float ms = 0;
            if (!rc && k == 0) rc = am_group_autotune(ln.g, s->d.iters, s->st, &threads, &ms);
            else if (!rc) rc = am_group_set_option(ln.g, AM_GOPT_THREADS, threads);
        }
        if (rc) {
            free_lanes(s);
            return rc;
        }
    }
    s->in_flight.assign(s->scenes.size(), 0);
    s->started = true;
    s->worker = std::thread(worker_main, s);
    return AM_OK;
}

int am_server_submit(am_server *s, const am_request *req, long long *ticket)
{
    if (!s || !req || !ticket) return report_error(AM_ERR_ARG, "null argument");
    if (req->scene < 0 || req->scene >= int(s->scenes.size())) return report_error(AM_ERR_ARG, "unknown scene");
    if (!(req->advance >= 0) || !std::isfinite(req->advance)) return report_error(AM_ERR_ARG, "bad advance");
    if ((req->xo == nullptr) != (req->yo == nullptr)) return report_error(AM_ERR_ARG, "xo and yo go together");
    if (req->flags & ~(AM_REQ_GOAL | AM_REQ_RESAMPLE | AM_REQ_SHIFT | AM_REQ_SCALE_LAMBDA))
        return report_error(AM_ERR_ARG, "unknown request flags");
    if ((req->flags & AM_REQ_SHIFT) && !(req->advance <= s->scenes[req->scene].T))
        return report_error(AM_ERR_ARG, "a shifted advance must be <= T");
    if (req->flags & AM_REQ_GOAL)
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(req->goal[k])) return report_error(AM_ERR_ARG, "non-finite goal");
    if ((req->flags & AM_REQ_RESAMPLE) && !(req->sigma >= 0.f && std::isfinite(req->sigma)))
        return report_error(AM_ERR_ARG, "sigma must be finite and >= 0");
    if ((req->flags & AM_REQ_SCALE_LAMBDA) && !(req->lambda_scale >= 0.f && std::isfinite(req->lambda_scale)))
        return report_error(AM_ERR_ARG, "lambda_scale must be finite and >= 0");
    const Scene &sc = s->scenes[req->scene];
    Request q;
    q.r = *req;
    if (req->xo) {
        q.xo.assign(req->xo, req->xo + size_t(sc.n) * sc.q);
        q.yo.assign(req->yo, req->yo + size_t(sc.n) * sc.q);
    }
    q.r.xo = q.r.yo = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return report_error(AM_ERR_STATE, "server stopping");
    if (int(s->pending.size()) >= s->d.max_pending) return report_error(AM_ERR_BUDGET, "request queue full");
    q.t_submit = now_s();
    q.ticket = s->next_ticket++;
    *ticket = q.ticket;
    s->outstanding.insert(q.ticket);
    s->pending.push_back(std::move(q));
    s->cv_work.notify_one();
    return AM_OK;
}

int am_server_poll(am_server *s, long long ticket, am_result *out, int timeout_ms)
{
    if (!s || !out) return report_error(AM_ERR_ARG, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->outstanding.count(ticket)) return report_error(AM_ERR_ARG, "unknown ticket");
    const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (!s->done.count(ticket))
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && !s->done.count(ticket))
            return AM_PENDING;
    *out = s->done[ticket];
    s->done.erase(ticket);
    s->outstanding.erase(ticket);
    return AM_OK;
}

int am_server_stats(am_server *s, long long *rounds, long long *completed, size_t *device_bytes)
{
    if (!s) return report_error(AM_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (rounds) *rounds = s->rounds;
    if (completed) *completed = s->completed;
    if (device_bytes) *device_bytes = s->used;
    return AM_OK;
}

void am_server_destroy(am_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    // Let the server's stream drain (bounded), then hand the scenes back to
    // the default stream: their handles must not keep the stream destroyed
    // below.
    if (s->st) {
        const auto t0 = std::chrono::steady_clock::now();
        while (cudaStreamQuery(s->st) == cudaErrorNotReady &&
               std::chrono::steady_clock::now() - t0 < std::chrono::seconds(60))
            std::this_thread::yield();
    }
    for (Scene &sc : s->scenes) am_set_stream(sc.h, nullptr);
    free_lanes(s);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

}  // extern "C"
