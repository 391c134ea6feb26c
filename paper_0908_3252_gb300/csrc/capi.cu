// capi.cu -- the C ABI of libspirec.so (declared in include/spirec.h): plan
// lifetime, argument checks, stream joins, the solve driver and its CUDA
// graph.  Every compute step runs in the kernels of the other .cu files.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <new>
#include <vector>

#include "internal.cuh"

// the per-interleave kernel cache (spirec_kcache_*)
struct spirec_kcache_s {
    int N = 0, M = 0, precision = 0, n = 0, device = 0;
    std::vector<int64_t> off;  // n + 1 sample offsets
    int64_t* kxq = nullptr;    // all samples, fixed point (device)
    int64_t* kyq = nullptr;
    float* spec = nullptr;     // n x M x M kernel spectra
    float2* G = nullptr;       // n x N x (2N-1) halves of G
};

namespace spirec {

static thread_local char g_err[512] = "";

// 2 s: far beyond any wait of a working launch, short enough that a stuck
// one gives its SMs back soon
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;
static std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};

unsigned long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

static std::atomic<int> g_stall{0};

bool injected_stall(int kind) { return (g_stall.load(std::memory_order_relaxed) & kind) != 0; }

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    if (e == cudaErrorMemoryAllocation) return SPIREC_ENOMEM;
    return SPIREC_ECUDA;
}

namespace {

// k * 2^64 mod 2^64 as a signed 64-bit integer; flags |k| > 0.5 or non-finite.
__global__ void k_traj_fixed(const double* __restrict__ kx, const double* __restrict__ ky,
                             int64_t L, int64_t* __restrict__ kxq, int64_t* __restrict__ kyq,
                             int* flag)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
         l += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const double k = c == 0 ? kx[l] : ky[l];
            int64_t q = 0;
            if (!(fabs(k) <= 0.5)) {  // also catches NaN
                atomicOr(flag, 1);
            } else {
                double t = k * 18446744073709551616.0;  // exact: power-of-two scaling
                if (t >= 9223372036854775808.0) t -= 18446744073709551616.0;
                q = __double2ll_rn(t);
            }
            if (c == 0) kxq[l] = q;
            else kyq[l] = q;
        }
    }
}

// out[ky*M + kx] = Chat[kx*M + ky]
__global__ void k_transpose_real(const float* __restrict__ in, int M, float* __restrict__ out)
{
    const int64_t MM = (int64_t)M * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MM;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ky = e / M, kx = e % M;
        out[e] = in[kx * M + ky];
    }
}

bool smooth235(int m)
{
    if (m < 1) return false;
    for (int f : {2, 3, 5})
        while (m % f == 0) m /= f;
    return m == 1;
}

constexpr int kCacheMaxTerms = 64;
struct CacheTerms {
    int n;
    int idx[kCacheMaxTerms];
};

// dst[e] = sum_j src[idx[j] * stride + e], j in the listed order.
__global__ void k_sum_cached(const float* __restrict__ src, int64_t stride, CacheTerms t, float* __restrict__ dst)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < stride;
         e += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int j = 0; j < t.n; ++j) acc += __ldg(src + t.idx[j] * stride + e);
        dst[e] = acc;
    }
}

struct Join {
    // Orders the plan's stream after the caller's stream on entry, and the
    // caller's stream after the plan's stream on exit.
    spirec_plan p;
    explicit Join(spirec_plan pp) : p(pp)
    {
        cudaEventRecord(p->ev_join, p->user_stream);
        cudaStreamWaitEvent(p->stream, p->ev_join, 0);
    }
    ~Join()
    {
        cudaEventRecord(p->ev_join, p->stream);
        cudaStreamWaitEvent(p->user_stream, p->ev_join, 0);
    }
};

// Plan buffers come from the device's stream-ordered pool (cudaMallocAsync on
// the plan's stream, cudaFreeAsync when the plan goes): a plan's creation and
// destruction then neither synchronise the device nor stall the streams of
// other plans, which matters to a server that re-plans per request shape.
// The pool keeps freed memory for reuse instead of returning it to the driver
// (a release threshold of the whole address range; a property of this
// process's allocator, set once per device).
void keep_pool(int dev)
{
    static std::atomic<bool> done[64];
    if (dev < 0 || dev >= 64 || done[dev].load(std::memory_order_acquire)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev].store(true, std::memory_order_release);
}

// Injected allocation failure (spirec_inject_alloc_failure): the number of
// plan allocations that still succeed, or < 0 when nothing is injected.
std::atomic<int64_t> g_allocs_left{-1};

// One allocation against the injected budget: false once it is spent.
bool alloc_allowed()
{
    int64_t cur = g_allocs_left.load(std::memory_order_relaxed);
    while (cur >= 0) {
        if (cur == 0) return false;
        if (g_allocs_left.compare_exchange_weak(cur, cur - 1, std::memory_order_relaxed)) return true;
    }
    return true;
}

template <typename T>
int dalloc(spirec_plan p, T** ptr, size_t count)
{
    *ptr = nullptr;
    if (count == 0) count = 1;
    const size_t bytes = count * sizeof(T);
    if (!alloc_allowed()) {
        set_error("injected allocation failure (spirec_inject_alloc_failure)");
        return SPIREC_ENOMEM;
    }
    keep_pool(p->device);
    cudaError_t e = cudaMallocAsync((void**)ptr, bytes, p->stream);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        set_error("cudaMallocAsync of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return SPIREC_ENOMEM;
    }
    p->device_bytes += bytes;
    return SPIREC_OK;
}

void free_plan(spirec_plan p)
{
    if (!p) return;
    void* bufs[] = {p->kxq, p->kyq, p->dflag, p->G, p->Chat, p->cwork, p->X, p->D, p->s, p->fsplit, p->ydir,
                    p->f[0], p->f[1], p->dbuf[0], p->dbuf[1], p->g, p->res, p->Td, p->tmp, p->twiddle,
                    p->part, p->scal, p->counters, p->Jdev, p->kpart, p->kstage, p->ystage, p->hqw,
                    p->wpair, p->s_in};
    for (void* b : bufs)
        if (b) {
            if (p->stream) cudaFreeAsync(b, p->stream);
            else cudaFree(b);
        }
    if (p->graph) cudaGraphExecDestroy(p->graph);
    for (int i = 0; i < (int)(sizeof(p->tev) / sizeof(p->tev[0])); ++i)
        if (p->tev_made[i]) cudaEventDestroy(p->tev[i]);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->ev_s_ready) cudaEventDestroy(p->ev_s_ready);
    if (p->ev_sin_free) cudaEventDestroy(p->ev_sin_free);
    if (p->ev_traj_in) cudaEventDestroy(p->ev_traj_in);
    if (p->hpin) cudaFreeHost(p->hpin);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

int check_plan(spirec_plan p)
{
    if (!p) {
        set_error("null plan");
        return SPIREC_EINVAL;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) {
        set_error("plan belongs to device %d, current device is %d", p->device, dev);
        return SPIREC_EINVAL;
    }
    return SPIREC_OK;
}

// --- timing: event pairs per stage on the plan's stream
int tstart(spirec_plan p, int stage, cudaEvent_t* out)
{
    *out = nullptr;
    if (!p->timing) return SPIREC_OK;
    if (p->tev_used + 2 > (int)(sizeof(p->tev) / sizeof(p->tev[0]))) {
        // fold finished pairs into the totals
        SPIREC_CK(cudaStreamSynchronize(p->stream));
        for (int i = 0; i < p->tev_used; i += 2) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->tev[i], p->tev[i + 1]);
            p->t_ms[p->tev_stage[i / 2]] += ms;
            p->t_cnt[p->tev_stage[i / 2]] += 1;
        }
        p->tev_used = 0;
    }
    cudaEvent_t* e = &p->tev[p->tev_used];
    if (!p->tev_made[p->tev_used]) {
        SPIREC_CK(cudaEventCreate(&e[0]));
        SPIREC_CK(cudaEventCreate(&e[1]));
        p->tev_made[p->tev_used] = p->tev_made[p->tev_used + 1] = true;
    }
    p->tev_stage[p->tev_used / 2] = stage;
    SPIREC_CK(cudaEventRecord(e[0], p->stream));
    *out = e[1];
    p->tev_used += 2;
    return SPIREC_OK;
}

int tstop(spirec_plan p, cudaEvent_t e)
{
    if (e) SPIREC_CK(cudaEventRecord(e, p->stream));
    return SPIREC_OK;
}

// The plan's pinned host words (made on first use) and the copy of the device
// error word into the second, enqueued on the plan's stream; read with
// pinned_flags after a synchronisation.
int enqueue_flags(spirec_plan p)
{
    if (!p->hpin) SPIREC_CK(cudaMallocHost(reinterpret_cast<void**>(&p->hpin), 2 * sizeof(double)));
    SPIREC_CK(cudaMemcpyAsync(reinterpret_cast<int*>(p->hpin + 1), p->dflag, sizeof(int), cudaMemcpyDeviceToHost,
                              p->stream));
    return SPIREC_OK;
}

int pinned_flags(spirec_plan p) { return *reinterpret_cast<const int*>(p->hpin + 1); }

int read_device_flags(spirec_plan p, int* flags)
{
    int rc = enqueue_flags(p);
    if (rc != SPIREC_OK) return rc;
    SPIREC_CK(cudaStreamSynchronize(p->stream));
    *flags = pinned_flags(p);
    return SPIREC_OK;
}

int flags_status(int flags)
{
    if (flags & E_TRAJ) {
        set_error("trajectory has a value outside [-0.5, 0.5] or not finite");
        return SPIREC_EINVAL;
    }
    if (flags & E_TIMEOUT) {
        set_error("a tensor-core pipeline wait ran out of time");
        return SPIREC_ETIMEOUT;
    }
    return SPIREC_OK;
}

// Fixed-point trajectory, G and the kernel spectrum.  With check_now the host
// waits for the conversion (not for G) and reports a bad trajectory at once;
// otherwise (the _dev entry point, which must not block) the device error
// word is reported at the next host synchronisation of the plan
// (spirec_solve, spirec_sync), as is a timeout of the contraction either way.
int build_trajectory(spirec_plan p, const double* kx_dev, const double* ky_dev, bool check_now)
{
    p->have_traj = false;
    p->have_data = false;
    SPIREC_CK(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
    int blocks = (int)((p->L + 255) / 256);
    if (blocks > 8 * 152) blocks = 8 * 152;
    k_traj_fixed<<<blocks, 256, 0, p->stream>>>(kx_dev, ky_dev, p->L, p->kxq, p->kyq, p->dflag);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    int rc;
    if (check_now) {
        int flags = 0;
        if ((rc = read_device_flags(p, &flags)) != SPIREC_OK) return rc;
        if ((rc = flags_status(flags)) != SPIREC_OK) return rc;
    }
    cudaEvent_t e;
    if ((rc = tstart(p, 0, &e)) != SPIREC_OK) return rc;
    if ((rc = launch_gram(p)) != SPIREC_OK) return rc;
    if ((rc = tstop(p, e)) != SPIREC_OK) return rc;
    if ((rc = tstart(p, 1, &e)) != SPIREC_OK) return rc;
    if ((rc = launch_spectrum(p)) != SPIREC_OK) return rc;
    if ((rc = tstop(p, e)) != SPIREC_OK) return rc;
    p->have_traj = true;
    return SPIREC_OK;
}

int build_data(spirec_plan p)
{
    int rc;
    if ((rc = launch_data_norm(p)) != SPIREC_OK) return rc;
    cudaEvent_t e;
    if ((rc = tstart(p, 2, &e)) != SPIREC_OK) return rc;
    if ((rc = launch_adjoint(p, p->s, p->D)) != SPIREC_OK) return rc;
    if ((rc = tstop(p, e)) != SPIREC_OK) return rc;
    p->have_data = true;
    return SPIREC_OK;
}

int ensure_J(spirec_plan p, int iters)
{
    if (p->Jcap >= iters + 1) return SPIREC_OK;
    if (p->Jdev) {
        cudaFreeAsync(p->Jdev, p->stream);  // after the stream's earlier users
        p->Jdev = nullptr;
    }
    int cap = iters + 1 < 64 ? 64 : iters + 1;
    int rc = dalloc(p, &p->Jdev, (size_t)cap);
    if (rc != SPIREC_OK) {
        p->Jcap = 0;
        return rc;
    }
    p->Jcap = cap;
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    return SPIREC_OK;
}

// Iteration loop, replayed from a CUDA graph captured once per (plan, iters).
int run_iterations(spirec_plan p, int iters)
{
    if (iters == 0) return SPIREC_OK;
    // re-capture when the tuning table changed: the graph holds launch shapes
    if (!p->graph || p->graph_iters != iters || p->graph_tune_gen != tune_generation()) {
        if (p->graph) {
            cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        SPIREC_CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = p->launches;
        int rc = SPIREC_OK;
        const int mn = p->minimiser;
        for (int k = 0; k < iters && rc == SPIREC_OK; ++k)
            rc = mn == SPIREC_MIN_HALF_QUADRATIC ? hq_outer_step(p, k, p->Jdev)
                 : mn == SPIREC_MIN_NEWTON       ? nt_outer_step(p, k, p->Jdev)
                                                 : cg_iteration(p, k, p->Jdev);
        if (mn != SPIREC_MIN_PRCG && rc == SPIREC_OK) rc = launch_hq_objective(p, p->Jdev + iters);  // last J
        cudaError_t e = cudaStreamEndCapture(p->stream, &g);
        p->graph_kernels = p->launches - l0;  // captured, not yet run
        p->launches = l0;
        if (rc != SPIREC_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&p->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->graph = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        p->graph_iters = iters;
        p->graph_tune_gen = tune_generation();
    }
    SPIREC_CK(cudaGraphLaunch(p->graph, p->stream));
    p->launches += p->graph_kernels;
    return SPIREC_OK;
}

bool solve_uses_loop(spirec_plan p)
{
    return p->mode != SPIREC_MODE_DIRECT && p->minimiser == SPIREC_MIN_PRCG && loop_supported(p->M) &&
           !getenv("SPIREC_NO_LOOP");
}

int solve_core(spirec_plan p, const float* x0, bool x0_dev, int iters)
{
    if (!p->have_traj || !p->have_data) {
        set_error("solve needs a trajectory and data (spirec_set_trajectory, spirec_set_data)");
        return SPIREC_ESTATE;
    }
    if (!p->have_reg) {
        set_error("solve needs spirec_set_reg first");
        return SPIREC_ESTATE;
    }
    if (iters < 0) {
        set_error("iters must be >= 0");
        return SPIREC_EINVAL;
    }
    int rc;
    if ((rc = ensure_J(p, iters)) != SPIREC_OK) return rc;
    const size_t img = (size_t)p->N * p->N * sizeof(float2);
    cudaEvent_t e;
    if ((rc = tstart(p, 3, &e)) != SPIREC_OK) return rc;
    const bool direct = p->mode == SPIREC_MODE_DIRECT;
    if (x0) {
        SPIREC_CK(cudaMemcpyAsync(p->f[0], x0, img,
                                  x0_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
        if ((rc = direct ? launch_normal_direct(p, p->f[0], p->res, false) : launch_toeplitz(p, p->f[0], p->res, -1)) !=
            SPIREC_OK)
            return rc;
    } else {
        SPIREC_CK(cudaMemsetAsync(p->f[0], 0, img, p->stream));
    }
    // the iteration carries res = T f - D (the data term's gradient is 2 res)
    if ((rc = launch_res_init(p, p->res, x0 != nullptr)) != SPIREC_OK) return rc;
    if (p->minimiser != SPIREC_MIN_PRCG) {
        // outer steps in a captured graph; the iterate stays in f[0]
        p->result_slot = 0;
        rc = iters == 0 ? launch_hq_objective(p, p->Jdev) : run_iterations(p, iters);
        if (rc != SPIREC_OK) return rc;
        return tstop(p, e);
    }
    rc = SPIREC_EUNSUPPORTED;
    if (solve_uses_loop(p)) {
        // first gradient and every iteration in one persistent kernel
        rc = launch_cg_loop(p, iters);
        if (rc != SPIREC_OK && rc != SPIREC_EUNSUPPORTED) return rc;
        p->result_slot = 0;
    }
    if (rc == SPIREC_EUNSUPPORTED) {
        p->result_slot = iters & 1;
        // gradient at x0, J(x0), beta = 0 (the first direction is -g)
        if ((rc = launch_update(p, p->f[0], p->f[0], p->dbuf[1], p->res, nullptr, p->g, 1, p->Jdev)) !=
            SPIREC_OK)
            return rc;
        if ((rc = run_iterations(p, iters)) != SPIREC_OK) return rc;
    }
    return tstop(p, e);
}

}  // namespace

int solve_loop_demand(spirec_plan p, int* blocks, int* capacity)
{
    *blocks = 0;
    *capacity = 0;
    if (!solve_uses_loop(p)) return 0;
    return loop_demand(p, blocks, capacity);
}

namespace {

// ------------------------------------------------------------ autotuning

// CUDA events that are destroyed on every path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Median milliseconds of three runs of fn after one warm-up, timed with
// events on the plan's stream.
template <class F>
int time_median(spirec_plan p, F fn, double* ms)
{
    EventPair ev;
    SPIREC_CK(cudaEventCreate(&ev.a));
    SPIREC_CK(cudaEventCreate(&ev.b));
    int rc = fn();
    if (rc != SPIREC_OK) return rc;
    float t[3];
    for (int r = 0; r < 3; ++r) {
        SPIREC_CK(cudaEventRecord(ev.a, p->stream));
        if ((rc = fn()) != SPIREC_OK) return rc;
        SPIREC_CK(cudaEventRecord(ev.b, p->stream));
        SPIREC_CK(cudaEventSynchronize(ev.b));
        SPIREC_CK(cudaEventElapsedTime(&t[r], ev.a, ev.b));
    }
    if (t[0] > t[1]) std::swap(t[0], t[1]);
    if (t[1] > t[2]) std::swap(t[1], t[2]);
    if (t[0] > t[1]) std::swap(t[0], t[1]);
    *ms = t[1];
    return SPIREC_OK;
}

// Candidates of a contraction split around the heuristic's value v0: for the
// tensor-core schedule fractions of the CTA count down to 1/32 (few CTAs
// leave the other SMs to concurrent solves), for the FP32 one halvings and
// doublings of the slice count.  The heuristic's value comes first.
std::vector<int> split_candidates(int precision, int v0)
{
    std::vector<int> c;
    auto add = [&](int v) {
        if (v < 1) v = 1;
        for (int x : c)
            if (x == v) return;
        c.push_back(v);
    };
    add(v0);
    if (precision != SPIREC_FP32) {
        for (int num : {24, 16, 12, 8, 4, 2, 1}) add(v0 * num / 32);
    } else {
        for (int f : {2, 4}) add(v0 / f);
        for (int f : {2, 4}) add(v0 * f);
    }
    return c;
}

int tune_contraction(spirec_plan p, int knob, int objective, int sms, int* chosen, double* best_ms)
{
    int rc;
    if ((rc = tune_store(knob, p, sms, 0)) != SPIREC_OK) return rc;
    int v0 = 0, used0 = 0;
    if ((rc = contraction_split(p, knob, &v0, &used0)) != SPIREC_OK) return rc;
    std::vector<int> seen;
    double best_score = 0.0;
    int best = 0;
    for (int c : split_candidates(p->precision, v0)) {
        if ((rc = tune_store(knob, p, sms, c)) != SPIREC_OK) return rc;
        int v = 0, used = 0;
        if ((rc = contraction_split(p, knob, &v, &used)) != SPIREC_OK) return rc;
        bool dup = false;
        for (int x : seen) dup = dup || x == v;  // clipped onto a value already timed
        if (dup) continue;
        seen.push_back(v);
        double ms = 0.0;
        if (knob == SPIREC_KNOB_GRAM_SPLIT)
            rc = time_median(p, [&] { return launch_gram(p); }, &ms);
        else
            rc = time_median(p, [&] { return launch_adjoint(p, p->s, p->D); }, &ms);
        if (rc != SPIREC_OK) return rc;
        const double score = objective == SPIREC_TUNE_THROUGHPUT ? ms * used : ms;
        if (best == 0 || score < best_score) {
            best = v;
            best_score = score;
            *best_ms = ms;
        }
    }
    *chosen = best;
    return tune_store(knob, p, sms, best);
}

// The tile shape of a contraction (tensor-core paths): both shapes timed at
// the heuristic split, the better one stored; the split is tuned after it.
int tune_tile(spirec_plan p, int split_knob, int objective, int sms, int* chosen, double* best_ms)
{
    const int tile_knob = split_knob == SPIREC_KNOB_GRAM_SPLIT ? SPIREC_KNOB_GRAM_TILE : SPIREC_KNOB_ADJOINT_TILE;
    *chosen = 0;
    *best_ms = 0.0;
    int rc;
    if (p->precision == SPIREC_FP32) return tune_store(tile_knob, p, sms, 0);
    if ((rc = tune_store(split_knob, p, sms, 0)) != SPIREC_OK) return rc;
    double best_score = 0.0;
    int best = 0;
    for (int t : {2, 1}) {
        if ((rc = tune_store(tile_knob, p, sms, t)) != SPIREC_OK) return rc;
        int v = 0, used = 0;
        if ((rc = contraction_split(p, split_knob, &v, &used)) != SPIREC_OK) return rc;
        double ms = 0.0;
        if (split_knob == SPIREC_KNOB_GRAM_SPLIT)
            rc = time_median(p, [&] { return launch_gram(p); }, &ms);
        else
            rc = time_median(p, [&] { return launch_adjoint(p, p->s, p->D); }, &ms);
        if (rc != SPIREC_OK) return rc;
        const double score = objective == SPIREC_TUNE_THROUGHPUT ? ms * used : ms;
        if (best == 0 || score < best_score) {
            best = t;
            best_score = score;
            *best_ms = ms;
        }
    }
    *chosen = best;
    return tune_store(tile_knob, p, sms, best);
}

int tune_loop(spirec_plan p, int objective, int iters, int sms, int* chosen, double* best_ms)
{
    *chosen = 0;
    if (p->mode == SPIREC_MODE_DIRECT || p->minimiser != SPIREC_MIN_PRCG || !loop_supported(p->M) ||
        getenv("SPIREC_NO_LOOP"))
        return SPIREC_OK;
    int rc;
    if ((rc = ensure_J(p, iters)) != SPIREC_OK) return rc;
    if ((rc = tune_store(SPIREC_KNOB_LOOP_ROWS, p, sms, 0)) != SPIREC_OK) return rc;
    int RB[8], grid[8];
    const int n = loop_candidates(p, RB, grid, 8);
    const size_t img = (size_t)p->N * p->N * sizeof(float2);
    double best_score = 0.0;
    int best = 0;
    for (int i = 0; i < n; ++i) {
        if ((rc = tune_store(SPIREC_KNOB_LOOP_ROWS, p, sms, RB[i])) != SPIREC_OK) return rc;
        double ms = 0.0;
        rc = time_median(
            p,
            [&]() -> int {
                SPIREC_CK(cudaMemsetAsync(p->f[0], 0, img, p->stream));
                const int rc1 = launch_res_init(p, p->res, false);
                if (rc1 != SPIREC_OK) return rc1;
                return launch_cg_loop(p, iters);
            },
            &ms);
        if (rc != SPIREC_OK) return rc;
        int flags = 0;
        if ((rc = read_device_flags(p, &flags)) != SPIREC_OK) return rc;
        if ((rc = flags_status(flags)) != SPIREC_OK) return rc;
        const double score = objective == SPIREC_TUNE_THROUGHPUT ? ms * (grid[i] < sms ? grid[i] : sms) : ms;
        if (best == 0 || score < best_score) {
            best = RB[i];
            best_score = score;
            *best_ms = ms;
        }
    }
    p->result_slot = 0;
    *chosen = best;
    return tune_store(SPIREC_KNOB_LOOP_ROWS, p, sms, best);
}

}  // namespace
}  // namespace spirec

using namespace spirec;

extern "C" {

const char* spirec_last_error(void) { return g_err; }

const char* spirec_version(void) { return "spirec 0.1 (sm_103a)"; }

int spirec_plan_create(spirec_plan* out, int32_t N, int64_t L, int32_t M, int32_t precision,
                       void* stream, const double* kx, const double* ky)
{
    g_err[0] = 0;
    if (!out) {
        set_error("out is NULL");
        return SPIREC_EINVAL;
    }
    *out = nullptr;
    if (N < 2 || N > 2048 || L < 1 || L > (int64_t)1 << 31) {
        set_error("unsupported sizes N=%d L=%lld", N, (long long)L);
        return SPIREC_EINVAL;
    }
    if (precision < SPIREC_FP32 || precision > SPIREC_MIXED_BF16X3) {
        set_error("unknown precision %d", precision);
        return SPIREC_EINVAL;
    }
    if (M == 0) {
        M = 2 * N - 1;
        while (!smooth235(M)) ++M;
    }
    if (M < 2 * N - 1 || !smooth235(M) || M > 4096) {
        set_error("M=%d must be >= 2N-1 = %d, <= 4096 and factor into 2, 3, 5", M, 2 * N - 1);
        return SPIREC_EINVAL;
    }
    spirec_plan p = new (std::nothrow) spirec_plan_s();
    if (!p) {
        set_error("host allocation failed");
        return SPIREC_ENOMEM;
    }
    memset((void*)p, 0, sizeof(*p));
    p->N = N;
    p->L = L;
    p->M = M;
    p->precision = precision;
    p->user_stream = (cudaStream_t)stream;
    int rc = SPIREC_OK;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    make_fft_plan(M, &p->fft);
#define TRY(x)                       \
    do {                             \
        if ((rc = (x)) != SPIREC_OK) { \
            free_plan(p);            \
            return rc;               \
        }                            \
    } while (0)
#define TRYCUDA(x)                         \
    do {                                   \
        cudaError_t e2 = (x);              \
        if (e2 != cudaSuccess) {           \
            rc = cuda_fail(e2, #x);        \
            free_plan(p);                  \
            return rc;                     \
        }                                  \
    } while (0)
    TRYCUDA(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
    TRYCUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    TRYCUDA(cudaEventCreateWithFlags(&p->ev_traj_in, cudaEventDisableTiming));
    const size_t NN = (size_t)N * N;
    // sample arrays carry 32 elements of padding: the tensor-core kernel reads
    // whole 16-byte multiples of a 32-sample chunk by TMA bulk copy
    TRY(dalloc(p, &p->kxq, (size_t)L + 32));
    TRY(dalloc(p, &p->kyq, (size_t)L + 32));
    if (precision != SPIREC_FP32) {
        TRY(dalloc(p, &p->wpair, (size_t)L + 32));
    }
    TRY(dalloc(p, &p->kstage, 2 * (size_t)L));
    TRY(dalloc(p, &p->dflag, 1));
    TRY(dalloc(p, &p->G, (size_t)N * (2 * N - 1)));
    TRY(dalloc(p, &p->Chat, (size_t)M * M));
    TRY(dalloc(p, &p->cwork, (size_t)M * M));
    TRY(dalloc(p, &p->X, (size_t)N * M));
    if ((p->fsplit_bytes = fsplit_bytes_tc(N, precision)) > 0) TRY(dalloc(p, &p->fsplit, p->fsplit_bytes));
    TRY(dalloc(p, &p->D, NN));
    TRY(dalloc(p, &p->s, (size_t)L + 32));
    TRY(dalloc(p, &p->ystage, (size_t)L + 32));
    TRY(dalloc(p, &p->f[0], NN));
    TRY(dalloc(p, &p->f[1], NN));
    TRY(dalloc(p, &p->dbuf[0], NN));
    TRY(dalloc(p, &p->dbuf[1], NN));
    TRY(dalloc(p, &p->g, NN));
    TRY(dalloc(p, &p->res, NN));
    TRY(dalloc(p, &p->Td, NN));
    TRY(dalloc(p, &p->tmp, NN));
    TRY(dalloc(p, &p->twiddle, (size_t)M));
    TRY(dalloc(p, &p->part, (size_t)P_NSLOTS * kMaxParts));
    TRY(dalloc(p, &p->scal, (size_t)S_NSCAL));
    TRY(dalloc(p, &p->counters, (size_t)C_N));
    {
        size_t a = 8 * (size_t)N * (2 * N - 1) * 2;  // floats: 8 splits of G
        size_t b = 4 * (size_t)L * 2;                 // forward row-block partials
        size_t c = kpart_floats_tc(N, L, precision);
        size_t n = a > b ? a : b;
        if (c > n) n = c;
        TRY(dalloc(p, &p->kpart, n));
        p->kpart_bytes = n * sizeof(float);
    }
    TRYCUDA(cudaMemsetAsync(p->counters, 0, C_N * sizeof(unsigned), p->stream));
    // the sample arrays are written over [0, L) only: their padding stays
    // zero, so a contraction chunk that runs past L gets zero weights
    TRYCUDA(cudaMemsetAsync(p->s, 0, sizeof(float2) * ((size_t)L + 32), p->stream));
    TRYCUDA(cudaMemsetAsync(p->ystage, 0, sizeof(float2) * ((size_t)L + 32), p->stream));
    if (p->wpair) TRYCUDA(cudaMemsetAsync(p->wpair, 0, sizeof(float2) * ((size_t)L + 32), p->stream));
    TRYCUDA(cudaMemsetAsync(p->scal, 0, S_NSCAL * sizeof(double), p->stream));
    TRYCUDA(cudaMemsetAsync(p->dbuf[0], 0, NN * sizeof(float2), p->stream));
    TRYCUDA(cudaMemsetAsync(p->dbuf[1], 0, NN * sizeof(float2), p->stream));
    TRYCUDA(cudaMemsetAsync(p->g, 0, NN * sizeof(float2), p->stream));
    {
        float2* tw = (float2*)malloc(sizeof(float2) * M);
        if (!tw) {
            free_plan(p);
            set_error("host allocation failed");
            return SPIREC_ENOMEM;
        }
        for (int k = 0; k < M; ++k) {
            const double a = -2.0 * M_PI * (double)k / (double)M;
            tw[k] = make_float2((float)cos(a), (float)sin(a));
        }
        e = cudaMemcpyAsync(p->twiddle, tw, sizeof(float2) * M, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        free(tw);
        TRYCUDA(e);
    }
    {
        // kernel attributes (shared-memory limits) are per device context:
        // set once, not per plan
        static std::atomic<bool> attrs_set[64];
        const bool once = p->device >= 0 && p->device < 64;
        if (!once || !attrs_set[p->device].load(std::memory_order_acquire)) {
            TRY(fft_setup_attributes(M));
            TRY(tc_setup_attributes());
            if (once) attrs_set[p->device].store(true, std::memory_order_release);
        }
    }
    if (kx || ky) {
        if (!kx || !ky) {
            free_plan(p);
            set_error("kx and ky must both be given or both be NULL");
            return SPIREC_EINVAL;
        }
        TRY(spirec_set_trajectory(p, kx, ky));
    }
#undef TRY
#undef TRYCUDA
    *out = p;
    return SPIREC_OK;
}

int spirec_plan_destroy(spirec_plan plan)
{
    if (!plan) return SPIREC_OK;
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
    return SPIREC_OK;
}

static void free_kcache(spirec_kcache c)
{
    if (!c) return;
    void* bufs[] = {c->kxq, c->kyq, c->spec, c->G};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete c;
}

int spirec_kcache_create(spirec_kcache* out, int32_t N, int32_t M, int32_t precision, int32_t n,
                         const int64_t* offsets, const double* kx, const double* ky, void* stream)
{
    if (!out || !offsets || !kx || !ky || n < 1) {
        set_error("kcache_create: null argument or n < 1");
        return SPIREC_EINVAL;
    }
    *out = nullptr;
    if (offsets[0] != 0) {
        set_error("offsets[0] must be 0");
        return SPIREC_EINVAL;
    }
    for (int i = 0; i < n; ++i)
        if (offsets[i + 1] <= offsets[i]) {
            set_error("offsets must increase (interleave %d is empty)", i);
            return SPIREC_EINVAL;
        }
    spirec_kcache c = new (std::nothrow) spirec_kcache_s;
    if (!c) {
        set_error("host allocation failed");
        return SPIREC_ENOMEM;
    }
    c->n = n;
    c->off.assign(offsets, offsets + n + 1);
    const int64_t Ltot = offsets[n];
    // one helper plan per distinct interleave length builds G and the spectrum
    std::map<int64_t, spirec_plan> helpers;
    int rc = SPIREC_OK;
    auto fail = [&](int code) {
        for (auto& h : helpers) spirec_plan_destroy(h.second);
        free_kcache(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGetDevice"));
    for (int i = 0; i < n; ++i) {
        const int64_t Li = offsets[i + 1] - offsets[i];
        spirec_plan h = nullptr;
        auto it = helpers.find(Li);
        if (it == helpers.end()) {
            if ((rc = spirec_plan_create(&h, N, Li, M, precision, stream, nullptr, nullptr)) != SPIREC_OK)
                return fail(rc);
            helpers[Li] = h;
            if (i == 0) {
                c->N = h->N;
                c->M = h->M;
                c->precision = h->precision;
                const size_t MM = (size_t)c->M * c->M, NG = (size_t)c->N * (2 * c->N - 1);
                if ((e = cudaMalloc((void**)&c->kxq, sizeof(int64_t) * (size_t)(Ltot + 32))) != cudaSuccess ||
                    (e = cudaMalloc((void**)&c->kyq, sizeof(int64_t) * (size_t)(Ltot + 32))) != cudaSuccess ||
                    (e = cudaMalloc((void**)&c->spec, sizeof(float) * MM * n)) != cudaSuccess ||
                    (e = cudaMalloc((void**)&c->G, sizeof(float2) * NG * n)) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(cuda_fail(e, "cudaMalloc (kernel cache)"));
                }
            }
        } else {
            h = it->second;
        }
        if ((rc = spirec_set_trajectory(h, kx + offsets[i], ky + offsets[i])) != SPIREC_OK) return fail(rc);
        const size_t MM = (size_t)c->M * c->M, NG = (size_t)c->N * (2 * c->N - 1);
        const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
        if ((e = cudaMemcpyAsync(c->kxq + offsets[i], h->kxq, sizeof(int64_t) * Li, d2d, h->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(c->kyq + offsets[i], h->kyq, sizeof(int64_t) * Li, d2d, h->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(c->spec + MM * i, h->Chat, sizeof(float) * MM, d2d, h->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(c->G + NG * i, h->G, sizeof(float2) * NG, d2d, h->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
            return fail(cuda_fail(e, "kernel cache copy"));
    }
    for (auto& h : helpers) spirec_plan_destroy(h.second);
    *out = c;
    return SPIREC_OK;
}

int spirec_kcache_destroy(spirec_kcache c)
{
    if (!c) return SPIREC_OK;
    cudaDeviceSynchronize();
    free_kcache(c);
    return SPIREC_OK;
}

int spirec_set_trajectory_cached(spirec_plan p, spirec_kcache c, const int32_t* which, int32_t count)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!c || !which || count < 1 || count > kCacheMaxTerms) {
        set_error("set_trajectory_cached: null cache or list, or count not in [1, %d]", kCacheMaxTerms);
        return SPIREC_EINVAL;
    }
    if (c->N != p->N || c->M != p->M || c->device != p->device) {
        set_error("cache is for N=%d, M=%d on device %d; plan N=%d, M=%d on device %d", c->N, c->M, c->device, p->N,
                  p->M, p->device);
        return SPIREC_EINVAL;
    }
    CacheTerms t{};
    t.n = count;
    int64_t total = 0;
    for (int j = 0; j < count; ++j) {
        if (which[j] < 0 || which[j] >= c->n) {
            set_error("interleave %d not in the cache (n = %d)", which[j], c->n);
            return SPIREC_EINVAL;
        }
        t.idx[j] = which[j];
        total += c->off[which[j] + 1] - c->off[which[j]];
    }
    if (total != p->L) {
        set_error("the listed interleaves hold %lld samples, the plan %lld", (long long)total, (long long)p->L);
        return SPIREC_EINVAL;
    }
    Join j(p);
    p->have_traj = false;
    p->have_data = false;
    SPIREC_CK(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
    int64_t pos = 0;
    for (int k = 0; k < count; ++k) {
        const int64_t o = c->off[which[k]], Li = c->off[which[k] + 1] - o;
        SPIREC_CK(cudaMemcpyAsync(p->kxq + pos, c->kxq + o, sizeof(int64_t) * Li, cudaMemcpyDeviceToDevice, p->stream));
        SPIREC_CK(cudaMemcpyAsync(p->kyq + pos, c->kyq + o, sizeof(int64_t) * Li, cudaMemcpyDeviceToDevice, p->stream));
        pos += Li;
    }
    const int64_t MM = (int64_t)p->M * p->M, NG2 = 2 * (int64_t)p->N * (2 * p->N - 1);
    int blocks = (int)((MM + 255) / 256);
    if (blocks > 8 * 152) blocks = 8 * 152;
    k_sum_cached<<<blocks, 256, 0, p->stream>>>(c->spec, MM, t, p->Chat);
    SPIREC_CK(cudaGetLastError());
    blocks = (int)((NG2 + 255) / 256);
    if (blocks > 8 * 152) blocks = 8 * 152;
    k_sum_cached<<<blocks, 256, 0, p->stream>>>(reinterpret_cast<const float*>(c->G), NG2, t,
                                                reinterpret_cast<float*>(p->G));
    SPIREC_CK(cudaGetLastError());
    p->launches += 2;
    p->have_traj = true;
    return SPIREC_OK;
}

int spirec_set_trajectory(spirec_plan p, const double* kx, const double* ky)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!kx || !ky) {
        set_error("kx, ky must not be NULL");
        return SPIREC_EINVAL;
    }
    Join j(p);
    SPIREC_CK(cudaMemcpyAsync(p->kstage, kx, sizeof(double) * p->L, cudaMemcpyHostToDevice, p->stream));
    SPIREC_CK(cudaMemcpyAsync(p->kstage + p->L, ky, sizeof(double) * p->L, cudaMemcpyHostToDevice, p->stream));
    SPIREC_CK(cudaEventRecord(p->ev_traj_in, p->stream));
    rc = build_trajectory(p, p->kstage, p->kstage + p->L, false);
    // the device conversion's range test, on the host while the GPU builds G
    bool bad = false;
    for (int64_t l = 0; l < p->L; ++l) bad |= !(fabs(kx[l]) <= 0.5) | !(fabs(ky[l]) <= 0.5);
    SPIREC_CK(cudaEventSynchronize(p->ev_traj_in));  // the caller's arrays are copied
    if (rc != SPIREC_OK) return rc;
    if (bad) {
        p->have_traj = false;
        set_error("trajectory has a value outside [-0.5, 0.5] or not finite");
        return SPIREC_EINVAL;
    }
    return SPIREC_OK;
}

int spirec_set_trajectory_dev(spirec_plan p, const double* kx, const double* ky)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!kx || !ky) {
        set_error("kx, ky must not be NULL");
        return SPIREC_EINVAL;
    }
    Join j(p);
    return build_trajectory(p, kx, ky, false);
}

int spirec_set_data(spirec_plan p, const float* s)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!s) {
        set_error("s must not be NULL");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("set_data needs a trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    // The caller's buffer is copied on a side stream and the call returns
    // once that copy is done, not after the trajectory work queued before it
    // on the plan's stream; the plan's stream then moves it into place.
    const size_t bytes = sizeof(float2) * p->L;
    if (!p->s_in) {
        SPIREC_CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        SPIREC_CK(cudaEventCreateWithFlags(&p->ev_s_ready, cudaEventDisableTiming));
        SPIREC_CK(cudaEventCreateWithFlags(&p->ev_sin_free, cudaEventDisableTiming));
        if ((rc = dalloc(p, &p->s_in, (size_t)p->L + 32)) != SPIREC_OK) return rc;
        SPIREC_CK(cudaEventRecord(p->ev_sin_free, p->stream));  // the copy stream follows the allocation
    }
    SPIREC_CK(cudaStreamWaitEvent(p->copy_stream, p->ev_sin_free, 0));  // no-op before its first record
    SPIREC_CK(cudaMemcpyAsync(p->s_in, s, bytes, cudaMemcpyHostToDevice, p->copy_stream));
    SPIREC_CK(cudaEventRecord(p->ev_s_ready, p->copy_stream));
    SPIREC_CK(cudaStreamWaitEvent(p->stream, p->ev_s_ready, 0));
    SPIREC_CK(cudaMemcpyAsync(p->s, p->s_in, bytes, cudaMemcpyDeviceToDevice, p->stream));
    SPIREC_CK(cudaEventRecord(p->ev_sin_free, p->stream));
    rc = build_data(p);
    if (rc == SPIREC_OK) SPIREC_CK(cudaEventSynchronize(p->ev_s_ready));
    return rc;
}

int spirec_set_data_dev(spirec_plan p, const float* s)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!s) {
        set_error("s must not be NULL");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("set_data needs a trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    SPIREC_CK(cudaMemcpyAsync(p->s, s, sizeof(float2) * p->L, cudaMemcpyDeviceToDevice, p->stream));
    return build_data(p);
}

int spirec_set_reg(spirec_plan p, double lambda1, double alpha1, double lambda0, double alpha0,
                   int32_t phi)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!(lambda1 >= 0.0) || !(lambda0 >= 0.0) || !isfinite(lambda1) || !isfinite(lambda0)) {
        set_error("lambdas must be finite and >= 0");
        return SPIREC_EINVAL;
    }
    if (phi < SPIREC_PHI_HUBER || phi > SPIREC_PHI_QUADRATIC) {
        set_error("unknown phi %d", phi);
        return SPIREC_EINVAL;
    }
    if (phi != SPIREC_PHI_QUADRATIC &&
        (!(alpha1 > 0.0) || !(alpha0 > 0.0) || !isfinite(alpha1) || !isfinite(alpha0))) {
        set_error("alphas must be finite and > 0");
        return SPIREC_EINVAL;
    }
    p->reg.lambda1 = (float)lambda1;
    p->reg.alpha1 = (float)alpha1;
    p->reg.lambda0 = (float)lambda0;
    p->reg.alpha0 = (float)alpha0;
    p->reg.kind = phi;
    p->have_reg = true;
    if (p->graph) {  // the graph holds the penalty by value
        cudaStreamSynchronize(p->stream);
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    return SPIREC_OK;
}

int spirec_set_mode(spirec_plan p, int32_t mode)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (mode != SPIREC_MODE_TOEPLITZ && mode != SPIREC_MODE_DIRECT) {
        set_error("mode must be SPIREC_MODE_TOEPLITZ or SPIREC_MODE_DIRECT, not %d", mode);
        return SPIREC_EINVAL;
    }
    if (mode == SPIREC_MODE_DIRECT && !p->ydir) {
        if ((rc = dalloc(p, &p->ydir, (size_t)p->L + 32)) != SPIREC_OK) return rc;
    }
    if (p->mode != mode && p->graph) {  // the captured iteration is mode-specific
        cudaStreamSynchronize(p->stream);
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    p->mode = mode;
    return SPIREC_OK;
}

int spirec_set_minimiser(spirec_plan p, int32_t kind, int32_t inner_iters)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (kind != SPIREC_MIN_PRCG && kind != SPIREC_MIN_HALF_QUADRATIC && kind != SPIREC_MIN_NEWTON) {
        set_error("minimiser must be SPIREC_MIN_PRCG, SPIREC_MIN_HALF_QUADRATIC or SPIREC_MIN_NEWTON, not %d", kind);
        return SPIREC_EINVAL;
    }
    if (kind != SPIREC_MIN_PRCG && (inner_iters < 1 || inner_iters > 1000)) {
        set_error("inner_iters must be in [1, 1000], not %d", inner_iters);
        return SPIREC_EINVAL;
    }
    if (kind != SPIREC_MIN_PRCG && !p->hqw) {
        if ((rc = dalloc(p, &p->hqw, (size_t)6 * p->N * p->N)) != SPIREC_OK) return rc;
    }
    const int inner = kind != SPIREC_MIN_PRCG ? inner_iters : 0;
    if ((p->minimiser != kind || p->hq_inner != inner) && p->graph) {  // the captured loop is minimiser-specific
        cudaStreamSynchronize(p->stream);
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    p->minimiser = kind;
    p->hq_inner = inner;
    return SPIREC_OK;
}

int spirec_solve(spirec_plan p, const float* x0, int32_t iters, float* x_out, double* J_hist)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x_out) {
        set_error("x_out must not be NULL");
        return SPIREC_EINVAL;
    }
    Join j(p);
    if ((rc = solve_core(p, x0, false, iters)) != SPIREC_OK) return rc;
    // every copy enqueued (the last J and the error word into the pinned
    // words), then one synchronisation
    const size_t img = (size_t)p->N * p->N * sizeof(float2);
    SPIREC_CK(cudaMemcpyAsync(x_out, p->f[p->result_slot], img, cudaMemcpyDeviceToHost, p->stream));
    if (J_hist)
        SPIREC_CK(cudaMemcpyAsync(J_hist, p->Jdev, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost,
                                  p->stream));
    if ((rc = enqueue_flags(p)) != SPIREC_OK) return rc;
    SPIREC_CK(cudaMemcpyAsync(p->hpin, p->Jdev + iters, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    SPIREC_CK(cudaStreamSynchronize(p->stream));
    if ((rc = flags_status(pinned_flags(p))) != SPIREC_OK) return rc;
    const double Jlast = p->hpin[0];
    if (!isfinite(Jlast)) {
        set_error("criterion is not finite after %d iterations", iters);
        return SPIREC_ENUMERIC;
    }
    return SPIREC_OK;
}

int spirec_solve_dev(spirec_plan p, const float* x0, int32_t iters, float* x_out, double* J_hist)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x_out) {
        set_error("x_out must not be NULL");
        return SPIREC_EINVAL;
    }
    Join j(p);
    if ((rc = solve_core(p, x0, true, iters)) != SPIREC_OK) return rc;
    const size_t img = (size_t)p->N * p->N * sizeof(float2);
    SPIREC_CK(cudaMemcpyAsync(x_out, p->f[p->result_slot], img, cudaMemcpyDeviceToDevice, p->stream));
    if (J_hist)
        SPIREC_CK(cudaMemcpyAsync(J_hist, p->Jdev, sizeof(double) * (iters + 1), cudaMemcpyDeviceToDevice,
                                  p->stream));
    return SPIREC_OK;
}

int spirec_forward_dev(spirec_plan p, const float* x, float* y)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !y) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("forward needs a trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    return launch_forward(p, (const float2*)x, (float2*)y);
}

int spirec_adjoint_dev(spirec_plan p, const float* y, float* x)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !y) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("adjoint needs a trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    return launch_adjoint(p, (const float2*)y, (float2*)x);
}

int spirec_gram_dev(spirec_plan p, float* G)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!G) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("no trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    SPIREC_CK(cudaMemcpyAsync(G, p->G, sizeof(float2) * (size_t)p->N * (2 * p->N - 1),
                              cudaMemcpyDeviceToDevice, p->stream));
    return SPIREC_OK;
}

int spirec_kernel_spectrum_dev(spirec_plan p, float* C)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!C) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("no trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    k_transpose_real<<<4 * 152, 256, 0, p->stream>>>(p->Chat, p->M, C);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int spirec_data_adjoint_dev(spirec_plan p, float* D)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!D) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_data) {
        set_error("no data");
        return SPIREC_ESTATE;
    }
    Join j(p);
    SPIREC_CK(cudaMemcpyAsync(D, p->D, sizeof(float2) * (size_t)p->N * p->N, cudaMemcpyDeviceToDevice,
                              p->stream));
    return SPIREC_OK;
}

int spirec_toeplitz_dev(spirec_plan p, const float* x, float* Tx)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !Tx) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("no trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    return launch_toeplitz(p, (const float2*)x, (float2*)Tx, -1);
}

int spirec_objective_grad_dev(spirec_plan p, const float* x, double* J_host, float* g)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !g) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_data || !p->have_reg) {
        set_error("objective needs data and a penalty");
        return SPIREC_ESTATE;
    }
    Join j(p);
    if ((rc = launch_toeplitz(p, (const float2*)x, p->tmp, -1)) != SPIREC_OK) return rc;
    if ((rc = launch_res_init(p, p->tmp, true)) != SPIREC_OK) return rc;  // T x - D
    if ((rc = launch_update(p, (const float2*)x, (float2*)x, p->dbuf[0], p->tmp, nullptr, (float2*)g, 1,
                            nullptr)) != SPIREC_OK)
        return rc;
    if (J_host) {
        SPIREC_CK(cudaMemcpyAsync(J_host, p->scal + S_J, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        SPIREC_CK(cudaStreamSynchronize(p->stream));
    }
    return SPIREC_OK;
}

// ---- host-pointer operator calls: the input goes to a plan buffer, the
// operator runs on the plan's stream, the result comes back; each returns
// after its copy-out (and reports device-side errors like spirec_solve).

namespace spirec {
namespace {
int finish_host_call(spirec_plan p)
{
    int flags = 0, rc;
    if ((rc = read_device_flags(p, &flags)) != SPIREC_OK) return rc;  // one synchronisation
    return flags_status(flags);
}
}  // namespace
}  // namespace spirec

int spirec_forward(spirec_plan p, const float* x, float* y)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !y) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("forward needs a trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    SPIREC_CK(cudaMemcpyAsync(p->tmp, x, sizeof(float2) * (size_t)p->N * p->N, cudaMemcpyHostToDevice, p->stream));
    if ((rc = launch_forward(p, p->tmp, p->ystage)) != SPIREC_OK) return rc;
    SPIREC_CK(cudaMemcpyAsync(y, p->ystage, sizeof(float2) * (size_t)p->L, cudaMemcpyDeviceToHost, p->stream));
    return finish_host_call(p);
}

int spirec_adjoint(spirec_plan p, const float* y, float* x)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !y) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("adjoint needs a trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    // ystage is the plan's padded sample buffer the contractions read
    SPIREC_CK(cudaMemcpyAsync(p->ystage, y, sizeof(float2) * (size_t)p->L, cudaMemcpyHostToDevice, p->stream));
    if ((rc = launch_adjoint(p, p->ystage, p->tmp)) != SPIREC_OK) return rc;
    SPIREC_CK(cudaMemcpyAsync(x, p->tmp, sizeof(float2) * (size_t)p->N * p->N, cudaMemcpyDeviceToHost, p->stream));
    return finish_host_call(p);
}

int spirec_gram_apply(spirec_plan p, const float* x, float* Tx)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !Tx) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj) {
        set_error("no trajectory");
        return SPIREC_ESTATE;
    }
    Join j(p);
    const size_t img = sizeof(float2) * (size_t)p->N * p->N;
    SPIREC_CK(cudaMemcpyAsync(p->tmp, x, img, cudaMemcpyHostToDevice, p->stream));
    if ((rc = launch_toeplitz(p, p->tmp, p->Td, -1)) != SPIREC_OK) return rc;
    SPIREC_CK(cudaMemcpyAsync(Tx, p->Td, img, cudaMemcpyDeviceToHost, p->stream));
    return finish_host_call(p);
}

int spirec_objective_grad(spirec_plan p, const float* x, double* J, float* g)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!x || !g) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (!p->have_data || !p->have_reg) {
        set_error("objective needs data and a penalty");
        return SPIREC_ESTATE;
    }
    Join j(p);
    const size_t img = sizeof(float2) * (size_t)p->N * p->N;
    SPIREC_CK(cudaMemcpyAsync(p->Td, x, img, cudaMemcpyHostToDevice, p->stream));
    if ((rc = launch_toeplitz(p, p->Td, p->tmp, -1)) != SPIREC_OK) return rc;
    if ((rc = launch_res_init(p, p->tmp, true)) != SPIREC_OK) return rc;  // T x - D
    if ((rc = launch_update(p, p->Td, p->Td, p->dbuf[0], p->tmp, nullptr, p->g, 1, nullptr)) != SPIREC_OK)
        return rc;
    SPIREC_CK(cudaMemcpyAsync(g, p->g, img, cudaMemcpyDeviceToHost, p->stream));
    double Jv = 0.0;
    SPIREC_CK(cudaMemcpyAsync(&Jv, p->scal + S_J, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    if ((rc = finish_host_call(p)) != SPIREC_OK) return rc;
    if (J) *J = Jv;
    if (!isfinite(Jv)) {
        set_error("criterion is not finite");
        return SPIREC_ENUMERIC;
    }
    return SPIREC_OK;
}

int spirec_autotune(spirec_plan p, int32_t objective, int32_t loop_iters, int32_t* chosen, double* best_ms)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!chosen) {
        set_error("chosen must not be NULL");
        return SPIREC_EINVAL;
    }
    if (objective != SPIREC_TUNE_LATENCY && objective != SPIREC_TUNE_THROUGHPUT) {
        set_error("objective must be SPIREC_TUNE_LATENCY or SPIREC_TUNE_THROUGHPUT, not %d", objective);
        return SPIREC_EINVAL;
    }
    if (loop_iters < 1) {
        set_error("loop_iters must be >= 1");
        return SPIREC_EINVAL;
    }
    if (!p->have_traj || !p->have_data || !p->have_reg) {
        set_error("autotune needs the plan's trajectory, data and regularisation");
        return SPIREC_ESTATE;
    }
    int sms = 0;
    if ((rc = device_sms(&sms)) != SPIREC_OK) return rc;
    int got[SPIREC_NUM_KNOBS] = {};
    double ms[SPIREC_NUM_KNOBS] = {};
    SPIREC_CK(cudaStreamSynchronize(p->stream));
    if ((rc = tune_tile(p, SPIREC_KNOB_GRAM_SPLIT, objective, sms, &got[SPIREC_KNOB_GRAM_TILE],
                        &ms[SPIREC_KNOB_GRAM_TILE])) != SPIREC_OK)
        return rc;
    if ((rc = tune_contraction(p, SPIREC_KNOB_GRAM_SPLIT, objective, sms, &got[0], &ms[0])) != SPIREC_OK) return rc;
    if ((rc = tune_tile(p, SPIREC_KNOB_ADJOINT_SPLIT, objective, sms, &got[SPIREC_KNOB_ADJOINT_TILE],
                        &ms[SPIREC_KNOB_ADJOINT_TILE])) != SPIREC_OK)
        return rc;
    if ((rc = tune_contraction(p, SPIREC_KNOB_ADJOINT_SPLIT, objective, sms, &got[1], &ms[1])) != SPIREC_OK)
        return rc;
    // G, the spectrum and D as a new plan of this shape computes them
    if ((rc = launch_gram(p)) != SPIREC_OK) return rc;
    if ((rc = launch_spectrum(p)) != SPIREC_OK) return rc;
    if ((rc = launch_adjoint(p, p->s, p->D)) != SPIREC_OK) return rc;
    if ((rc = tune_loop(p, objective, loop_iters, sms, &got[2], &ms[2])) != SPIREC_OK) return rc;
    int flags = 0;
    if ((rc = read_device_flags(p, &flags)) != SPIREC_OK) return rc;
    if ((rc = flags_status(flags)) != SPIREC_OK) return rc;
    for (int k = 0; k < SPIREC_NUM_KNOBS; ++k) {
        chosen[k] = got[k];
        if (best_ms) best_ms[k] = ms[k];
    }
    return SPIREC_OK;
}

int spirec_inject_alloc_failure(int64_t n)
{
    g_allocs_left.store(n < 0 ? -1 : n, std::memory_order_relaxed);
    return SPIREC_OK;
}

int spirec_inject_wait_stall(int32_t kernels)
{
    if (kernels & ~(kStallLoop | kStallContraction)) {
        set_error("unknown kernel bits %d", kernels);
        return SPIREC_EINVAL;
    }
    g_stall.store(kernels, std::memory_order_relaxed);
    return SPIREC_OK;
}

int spirec_set_wait_limit_ns(uint64_t ns)
{
    g_wait_ns.store(ns == 0 ? kDefaultWaitNs : (unsigned long long)ns, std::memory_order_relaxed);
    return SPIREC_OK;
}

int spirec_sync(spirec_plan p)
{
    int rc = check_plan(p);
    if (rc) return rc;
    int flags = 0;
    if ((rc = read_device_flags(p, &flags)) != SPIREC_OK) return rc;
    return flags_status(flags);
}

int spirec_plan_info(spirec_plan p, int32_t* N, int64_t* L, int32_t* M, int32_t* precision,
                     size_t* device_bytes)
{
    if (!p) {
        set_error("null plan");
        return SPIREC_EINVAL;
    }
    if (N) *N = p->N;
    if (L) *L = p->L;
    if (M) *M = p->M;
    if (precision) *precision = p->precision;
    if (device_bytes) *device_bytes = p->device_bytes;
    return SPIREC_OK;
}

int spirec_plan_scalars(spirec_plan p, double* out, int32_t n)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (!out || n < 0) {
        set_error("bad output");
        return SPIREC_EINVAL;
    }
    if (n > S_NSCAL) n = S_NSCAL;
    SPIREC_CK(cudaMemcpyAsync(out, p->scal, sizeof(double) * n, cudaMemcpyDeviceToHost, p->stream));
    SPIREC_CK(cudaStreamSynchronize(p->stream));
    return SPIREC_OK;
}

int spirec_launch_count(spirec_plan p, int64_t* count)
{
    if (!p || !count) {
        set_error("null argument");
        return SPIREC_EINVAL;
    }
    *count = p->launches;
    return SPIREC_OK;
}

int spirec_timing(spirec_plan p, int32_t enable)
{
    int rc = check_plan(p);
    if (rc) return rc;
    SPIREC_CK(cudaStreamSynchronize(p->stream));
    p->timing = enable != 0;
    p->tev_used = 0;
    for (int i = 0; i < SPIREC_NUM_STAGES; ++i) {
        p->t_ms[i] = 0.0;
        p->t_cnt[i] = 0;
    }
    return SPIREC_OK;
}

int spirec_timing_read(spirec_plan p, double* out_ms, int64_t* out_count)
{
    int rc = check_plan(p);
    if (rc) return rc;
    SPIREC_CK(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < p->tev_used; i += 2) {
        float ms = 0.f;
        SPIREC_CK(cudaEventElapsedTime(&ms, p->tev[i], p->tev[i + 1]));
        p->t_ms[p->tev_stage[i / 2]] += ms;
        p->t_cnt[p->tev_stage[i / 2]] += 1;
    }
    p->tev_used = 0;
    for (int i = 0; i < SPIREC_NUM_STAGES; ++i) {
        if (out_ms) out_ms[i] = p->t_ms[i];
        if (out_count) out_count[i] = p->t_cnt[i];
    }
    return SPIREC_OK;
}

}  // extern "C"
