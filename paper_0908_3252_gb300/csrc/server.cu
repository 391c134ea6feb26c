// server.cu -- request loop for many reconstructions on one GPU (continuous
// batching), and the batched solve.
//
// A server owns `max_slots` worker threads.  Each worker keeps one plan (its
// own CUDA stream, trajectory tables, iterate and scratch resident on the
// device) and reuses it while requests keep the same (N, L).  Requests wait
// in a FIFO queue; the head is admitted when a worker is idle and its device
// footprint fits the HBM budget next to the plans already resident (a worker
// whose plan does not fit the next request releases it first).  When the
// head fits only once plans held by other idle workers go, the admitting
// worker asks those workers to release them (they are idle, so their plans
// are not in use), instead of waiting for a completion that may never come.
// Admitted requests run concurrently on their workers' streams, so a request
// that arrives while others are on the GPU starts as soon as a slot and
// memory free up, and its kernels overlap theirs.
//
// Co-residency: a solve on the persistent CG loop is one cooperative launch
// whose blocks wait on each other at every grid synchronisation, so all of
// them must be resident at once.  Concurrent loops of several workers must
// therefore fit the device together: before a solve, a worker reserves its
// loop's blocks against the device's capacity for that loop (one block per
// SM) and waits while the running loops hold too many; the reservation ends
// when the solve returns.  Other kernels never wait on each other, so they
// can only delay a loop's blocks, not hold them off for good.
//
// Results are identical alone and in a mix: every kernel's launch shape and
// summation order depend only on the request's own sizes.
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace spirec {
namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t ticket;
    spirec_request req;  // pointers below point into the owned vectors
    std::vector<double> kx, ky;
    std::vector<float> s;
    std::vector<float> x;
    Clock::time_point t_submit, t_start, t_end;
    double J = 0.0;
    int status = SPIREC_OK;
    bool done = false;
    char err[256] = "";
};

}  // namespace
}  // namespace spirec

namespace spirec {
namespace {
// A worker's state as the admission sees it (guarded by the server's mutex).
struct Slot {
    bool idle = false;   // waiting for work, its plan unused
    bool evict = false;  // asked to release its plan
    size_t bytes = 0;    // footprint of its resident plan
};
}  // namespace
}  // namespace spirec

struct spirec_server_s {
    int device;
    int precision;
    size_t budget;
    size_t in_use = 0;  // device bytes of resident plans
    int loop_blocks = 0;  // persistent-loop blocks of the running solves
    std::vector<spirec::Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<spirec::Job>> queue;
    std::map<uint64_t, std::shared_ptr<spirec::Job>> jobs;
    std::vector<std::thread> workers;
    std::vector<double> latencies;  // seconds, completed requests
    uint64_t next_ticket = 1;
    int64_t completed = 0, failed = 0;
    bool stop = false;
};

namespace spirec {
namespace {

// Device bytes a plan of this shape holds (mirrors spirec_plan_create).
size_t plan_bytes(int N, int64_t L, int M, int precision)
{
    const size_t NN = (size_t)N * N;
    size_t b = 0;
    b += 2 * ((size_t)L + 32) * 8;              // fixed-point trajectory
    if (precision != SPIREC_FP32) b += ((size_t)L + 32) * 8;  // the paired contractions' weights
    b += 2 * (size_t)L * 8;                      // staging
    b += (size_t)N * (2 * N - 1) * 8;            // G
    b += (size_t)M * M * 4 + (size_t)M * M * 8;  // spectrum + work
    b += (size_t)N * M * 8;                      // rows
    b += 3 * ((size_t)L + 32) * 8;               // data, its staging, the host upload buffer
    b += 10 * NN * 8;                            // iterates, directions, gradients, D, scratch
    b += (size_t)M * 8 + (size_t)P_NSLOTS * kMaxParts * 8 + 4096;
    b += fsplit_bytes_tc(N, precision);  // split image of the tensor-core forward
    size_t a = 8 * (size_t)N * (2 * N - 1) * 2, c = 4 * (size_t)L * 2, t = kpart_floats_tc(N, L, precision);
    b += std::max(std::max(a, c), t) * 4;        // split-K partials
    return b;
}

int choose_M(int N)
{
    // the plan's own default (smallest 2,3,5-smooth >= 2N-1), or the next
    // power of two when it costs at most 40% more and enables the persistent loop
    auto smooth = [](int m) {
        for (int f : {2, 3, 5})
            while (m % f == 0) m /= f;
        return m == 1;
    };
    int m = 2 * N - 1;
    while (!smooth(m)) ++m;
    int p2 = 1;
    while (p2 < 2 * N - 1) p2 <<= 1;
    return (double)p2 <= 1.4 * m && loop_supported(p2) ? p2 : m;
}

void worker_main(spirec_server srv, int me)
{
    cudaSetDevice(srv->device);
    // the worker's own stream: plans joined to the legacy default stream would
    // serialise the workers against each other
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    spirec_plan plan = nullptr;
    int pN = 0, pM = 0;
    int64_t pL = 0;
    Slot& slot = srv->slots[me];
    auto release_plan = [&](std::unique_lock<std::mutex>& lk) {
        // the plan is idle: drop it outside the lock, then return its bytes
        spirec_plan old = plan;
        plan = nullptr;
        pN = 0;
        lk.unlock();
        if (old) spirec_plan_destroy(old);
        lk.lock();
        srv->in_use -= slot.bytes;
        slot.bytes = 0;
        slot.evict = false;
        srv->cv_work.notify_all();
    };
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            slot.idle = true;
            for (;;) {
                if (srv->stop) break;
                if (slot.evict) {
                    release_plan(lk);
                    continue;
                }
                if (!srv->queue.empty()) {
                    const spirec_request& r = srv->queue.front()->req;
                    const int M = choose_M(r.N);
                    const bool reuse = plan && pN == r.N && pL == r.L && pM == M;
                    const size_t need = reuse ? 0 : plan_bytes(r.N, r.L, M, srv->precision);
                    const size_t freed = reuse ? 0 : slot.bytes;
                    if (srv->in_use - freed + need <= srv->budget || srv->in_use == slot.bytes) {
                        job = srv->queue.front();
                        srv->queue.pop_front();
                        if (!reuse) {
                            srv->in_use = srv->in_use - freed + need;
                            slot.bytes = need;
                        }
                        break;
                    }
                    // would the plans of the other idle workers, released,
                    // make room?  Then ask them (largest first) to release
                    std::vector<int> idle;
                    size_t avail = srv->budget - std::min(srv->budget, srv->in_use - freed);
                    for (int i = 0; i < (int)srv->slots.size(); ++i)
                        if (i != me && srv->slots[i].idle && srv->slots[i].bytes > 0 && !srv->slots[i].evict)
                            idle.push_back(i);
                    std::sort(idle.begin(), idle.end(),
                              [&](int a, int b) { return srv->slots[a].bytes > srv->slots[b].bytes; });
                    size_t pending = 0;
                    for (auto& o : srv->slots)
                        if (o.evict) pending += o.bytes;
                    size_t gain = pending;
                    std::vector<int> pick;
                    for (int i : idle) {
                        if (avail + gain >= need) break;
                        gain += srv->slots[i].bytes;
                        pick.push_back(i);
                    }
                    if (avail + gain >= need && !pick.empty()) {
                        for (int i : pick) srv->slots[i].evict = true;
                        srv->cv_work.notify_all();
                    }
                }
                srv->cv_work.wait(lk);
            }
            slot.idle = false;
            if (!job) break;
        }
        job->t_start = Clock::now();
        const spirec_request& r = job->req;
        const int M = choose_M(r.N);
        int rc = SPIREC_OK;
        if (!(plan && pN == r.N && pL == r.L && pM == M)) {
            if (plan) spirec_plan_destroy(plan);
            plan = nullptr;
            rc = spirec_plan_create(&plan, r.N, r.L, M, srv->precision, st, nullptr, nullptr);
            if (rc == SPIREC_OK) {
                pN = r.N;
                pL = r.L;
                pM = M;
            } else {
                plan = nullptr;
                pN = 0;
            }
        }
        if (rc == SPIREC_OK) rc = spirec_set_trajectory(plan, r.kx, r.ky);
        if (rc == SPIREC_OK) rc = spirec_set_data(plan, r.s);
        if (rc == SPIREC_OK) rc = spirec_set_reg(plan, r.lambda1, r.alpha1, r.lambda0, r.alpha0, r.phi);
        std::vector<double> Jh((size_t)std::max(r.iters, 0) + 1);
        int blocks = 0, capacity = 0;
        if (rc == SPIREC_OK && r.iters > 0) solve_loop_demand(plan, &blocks, &capacity);
        if (blocks > 0) {
            // the loop's blocks must be resident together with those of
            // the other running loops (a loop alone always fits)
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->loop_blocks == 0 || srv->loop_blocks + blocks <= capacity; });
            srv->loop_blocks += blocks;
        }
        if (rc == SPIREC_OK) rc = spirec_solve(plan, nullptr, r.iters, job->x.data(), Jh.data());
        job->t_end = Clock::now();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->loop_blocks -= blocks;
            job->status = rc;
            if (rc != SPIREC_OK) {
                snprintf(job->err, sizeof(job->err), "%s", spirec_last_error());
                ++srv->failed;
                if (!plan) {
                    srv->in_use -= slot.bytes;
                    slot.bytes = 0;
                }
            } else {
                job->J = Jh[(size_t)r.iters];
                ++srv->completed;
                srv->latencies.push_back(std::chrono::duration<double>(job->t_end - job->t_submit).count());
            }
            job->done = true;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    if (plan) spirec_plan_destroy(plan);
    if (st) cudaStreamDestroy(st);
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->in_use -= slot.bytes;
    slot.bytes = 0;
}

}  // namespace

size_t server_plan_bytes(int N, int64_t L, int precision, int* M)
{
    *M = choose_M(N);
    return plan_bytes(N, L, *M, precision);
}

namespace {

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace spirec

using namespace spirec;

extern "C" {

int spirec_server_create(spirec_server* out, size_t hbm_budget_bytes, int32_t max_slots, int32_t precision)
{
    if (!out || max_slots < 1 || max_slots > 64 || precision < SPIREC_FP32 || precision > SPIREC_MIXED_BF16X3) {
        set_error("bad server arguments");
        return SPIREC_EINVAL;
    }
    spirec_server srv = new (std::nothrow) spirec_server_s();
    if (!srv) {
        set_error("host allocation failed");
        return SPIREC_ENOMEM;
    }
    cudaError_t e = cudaGetDevice(&srv->device);
    if (e != cudaSuccess) {
        delete srv;
        return cuda_fail(e, "cudaGetDevice");
    }
    srv->precision = precision;
    srv->budget = hbm_budget_bytes;
    srv->slots.resize((size_t)max_slots);
    for (int i = 0; i < max_slots; ++i) srv->workers.emplace_back(worker_main, srv, i);
    *out = srv;
    return SPIREC_OK;
}

int spirec_server_plan_bytes(int32_t N, int64_t L, int32_t precision, size_t* bytes, int32_t* M)
{
    if (!bytes || N < 2 || N > 2048 || L < 1 || precision < SPIREC_FP32 || precision > SPIREC_MIXED_BF16X3) {
        set_error("bad arguments");
        return SPIREC_EINVAL;
    }
    int m = 0;
    *bytes = server_plan_bytes(N, L, precision, &m);
    if (M) *M = m;
    return SPIREC_OK;
}

int spirec_server_submit(spirec_server srv, const spirec_request* req, uint64_t* ticket)
{
    if (!srv || !req || !ticket || !req->kx || !req->ky || !req->s || req->N < 2 || req->L < 1 ||
        req->iters < 0) {
        set_error("bad request");
        return SPIREC_EINVAL;
    }
    const int M = choose_M(req->N);
    if (plan_bytes(req->N, req->L, M, srv->precision) > srv->budget) {
        set_error("request footprint exceeds the server's HBM budget");
        return SPIREC_EBUSY;
    }
    auto job = std::make_shared<Job>();
    job->kx.assign(req->kx, req->kx + req->L);
    job->ky.assign(req->ky, req->ky + req->L);
    job->s.assign(req->s, req->s + 2 * req->L);
    job->x.assign((size_t)2 * req->N * req->N, 0.f);
    job->req = *req;
    job->req.kx = job->kx.data();
    job->req.ky = job->ky.data();
    job->req.s = job->s.data();
    job->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        job->ticket = srv->next_ticket++;
        srv->jobs[job->ticket] = job;
        srv->queue.push_back(job);
    }
    srv->cv_work.notify_all();
    *ticket = job->ticket;
    return SPIREC_OK;
}

int spirec_server_wait(spirec_server srv, uint64_t ticket, int32_t timeout_ms, float* x_out, double* J,
                       double* latency_s)
{
    if (!srv) {
        set_error("null server");
        return SPIREC_EINVAL;
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return SPIREC_EINVAL;
    }
    std::shared_ptr<Job> job = it->second;
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                          [&] { return job->done; });
    if (!ok) {
        set_error("request %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
        return SPIREC_ETIMEOUT;
    }
    srv->jobs.erase(it);
    if (job->status != SPIREC_OK) {
        set_error("%s", job->err);
        return job->status;
    }
    if (x_out) std::copy(job->x.begin(), job->x.end(), x_out);
    if (J) *J = job->J;
    if (latency_s) *latency_s = std::chrono::duration<double>(job->t_end - job->t_submit).count();
    return SPIREC_OK;
}

int spirec_server_stats(spirec_server srv, double* p50_s, double* p99_s, int64_t* completed, int64_t* failed,
                        int64_t* queued)
{
    if (!srv) {
        set_error("null server");
        return SPIREC_EINVAL;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (p50_s) *p50_s = percentile(srv->latencies, 0.50);
    if (p99_s) *p99_s = percentile(srv->latencies, 0.99);
    if (completed) *completed = srv->completed;
    if (failed) *failed = srv->failed;
    if (queued) *queued = (int64_t)srv->queue.size();
    return SPIREC_OK;
}

int spirec_server_destroy(spirec_server srv)
{
    if (!srv) return SPIREC_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers) t.join();
    delete srv;
    return SPIREC_OK;
}

int spirec_batch_solve(const spirec_plan* plans, int32_t n, const float* const* x0, int32_t iters,
                       float* const* x_out, double* const* J_hist)
{
    if (!plans || n < 0 || !x_out) {
        set_error("bad batch arguments");
        return SPIREC_EINVAL;
    }
    // enqueue every solve on its own plan's stream, then wait for all
    for (int i = 0; i < n; ++i) {
        const int rc = spirec_solve_dev(plans[i], x0 ? x0[i] : nullptr, iters, x_out[i], J_hist ? J_hist[i] : nullptr);
        if (rc != SPIREC_OK) return rc;
    }
    int first = SPIREC_OK;
    for (int i = 0; i < n; ++i) {
        const int rc = spirec_sync(plans[i]);
        if (rc != SPIREC_OK && first == SPIREC_OK) first = rc;
    }
    return first;
}

}  // extern "C"
