// Job server: whole slots (factorise + select paths + precode) admitted as
// they arrive onto a set of CUDA streams ("lanes"), each job's per-channel
// state carved from one device pool. Admission is first come, first served,
// gated by an idle lane and a first-fit piece of the pool; progress (retiring
// finished jobs, admitting waiting ones) happens inside the calls.
//
// A server made by vp_server_create_fake runs the same admission, pool and
// reporting logic on a host clock instead of the GPU (a job "runs" for its
// channel count in microseconds), so that the scheduling can be tested, and
// studied, without a device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vp_internal.cuh"

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxLanes = 32;
constexpr int kFakeRanks = 6;   // priority ranks a fake server models under the age policy

size_t round_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Pool {
public:
    explicit Pool(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            if (used_ > high_) high_ = used_;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t high() const { return high_; }

private:
    size_t size_, used_ = 0, high_ = 0;
    std::map<size_t, size_t> free_;
};

struct Job {
    vp_job_desc desc;
    vp_plan plan;          // parameters; d points into the pool once admitted
    size_t bytes = 0, off = 0;
    int lane = -1;
    int rank = 0;          // priority rank of its stream (age policy), 0 = highest
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int status = VP_OK;
    double fake_t0 = 0.0, fake_t1 = 0.0;   // host-clock run of a fake server's job (ms)
};

bool finite_nonneg(float v) { return v >= 0.f && std::isfinite(v); }

// The limits of vp_plan_create, the plan setters and vp_precode_noalloc.
bool job_ok(const vp_job_desc& j)
{
    if (j.K < 1 || j.K > VP_MAX_K || j.M < 1 || j.M > VP_MAX_M) return false;
    if (!(j.qam == 4 || j.qam == 16 || j.qam == 64 || j.qam == 256)) return false;
    long long p9 = 1;
    for (int i = 0; i < j.K && p9 <= VP_MAX_PATHS; ++i) p9 *= 9;
    if (j.n_paths < 1 || j.n_paths > VP_MAX_PATHS || (long long)j.n_paths > p9) return false;
    if (!finite_nonneg(j.tau) || !finite_nonneg(j.lambda) || !finite_nonneg(j.fp64_threshold)) return false;
    if (j.K > j.M && !(j.lambda > 0.f)) return false;
    if (j.demap != VP_DEMAP_EXACT && j.demap != VP_DEMAP_LUT) return false;
    if (j.frac_bits < 0 || j.frac_bits > 15 || (j.frac_bits > 0 && j.demap != VP_DEMAP_EXACT)) return false;
    if (j.C < 1 || j.S < 0 || (long long)j.C * j.S > 0x7fffffffLL) return false;
    if (!j.H) return false;
    if (j.S > 0 && (!j.sym_idx || !j.x || !j.l || !j.gamma)) return false;
    return true;
}

vp_plan plan_of(const vp_job_desc& j)
{
    vp_plan p;
    p.K = j.K;
    p.M = j.M;
    p.qam = j.qam;
    p.n_paths = j.n_paths;
    p.tau = (j.tau == 0.f) ? 2.0f * std::sqrt((float)j.qam) : j.tau;
    p.kappa_thr = (j.fp64_threshold == 0.f) ? 1e4f : j.fp64_threshold;
    p.lambda = j.lambda;
    p.demap = j.demap;
    p.frac_bits = j.frac_bits;
    return p;
}

}  // namespace

struct vp_server {
    std::mutex mu;
    bool fake = false;                    // host-clock executor, no device work
    int nlanes = 0;
    std::chrono::steady_clock::time_point t_ref;
    int device = 0;
    size_t pool_bytes = 0;
    unsigned char* pool_base = nullptr;
    Pool* pool = nullptr;
    std::vector<cudaStream_t> lanes;
    std::vector<int64_t> lane_job;        // job on each lane, 0 = idle
    int policy = VP_SERVE_FCFS;
    int nranks = 1;                       // priority ranks in use by the age policy
    std::vector<std::vector<cudaStream_t>> ranked;   // age policy: [rank][lane], rank 0 highest priority
    std::vector<cudaEvent_t> spare_events;
    cudaEvent_t ref = nullptr;
    std::unordered_map<int64_t, Job> jobs;
    std::deque<int64_t> waiting;
    std::vector<int64_t> running;
    std::deque<vp_job_done> finished;
    int64_t next_id = 1, submitted = 0, completed = 0;
    int max_in_flight = 0;
};

namespace {

double host_ms(const vp_server* s)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s->t_ref).count();
}

cudaError_t take_event(vp_server* s, cudaEvent_t* e)
{
    if (!s->spare_events.empty()) {
        *e = s->spare_events.back();
        s->spare_events.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// Ends a job: frees its state and lane, keeps its events for reuse, queues
// its record for vp_server_poll.
void finish(vp_server* s, int64_t id, Job& j, float t0, float t1)
{
    if (j.lane >= 0) s->lane_job[j.lane] = 0;
    if (j.bytes) s->pool->release(j.off, j.bytes);
    if (j.ev0) s->spare_events.push_back(j.ev0);
    if (j.ev1) s->spare_events.push_back(j.ev1);
    s->finished.push_back(vp_job_done{id, j.status, t0, t1, j.rank});
    s->jobs.erase(id);
    ++s->completed;
}

// Retire the running jobs whose last event has completed.
void retire(vp_server* s)
{
    for (size_t i = 0; i < s->running.size();) {
        const int64_t id = s->running[i];
        Job& j = s->jobs[id];
        if (s->fake) {
            if (host_ms(s) < j.fake_t1) {
                ++i;
                continue;
            }
            finish(s, id, j, (float)j.fake_t0, (float)j.fake_t1);
            s->running[i] = s->running.back();
            s->running.pop_back();
            continue;
        }
        const cudaError_t q = cudaEventQuery(j.ev1);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        float t0 = 0.f, t1 = 0.f;
        if (q != cudaSuccess || cudaEventElapsedTime(&t0, s->ref, j.ev0) != cudaSuccess ||
            cudaEventElapsedTime(&t1, s->ref, j.ev1) != cudaSuccess) {
            cudaGetLastError();
            if (q != cudaSuccess) j.status = VP_ERR_CUDA;
        }
        finish(s, id, j, t0, t1);
        s->running[i] = s->running.back();
        s->running.pop_back();
    }
}

// Priority rank for a job admitted now under the age policy: one below the
// youngest running job's (so every running job outranks it), 0 when nothing
// runs, and the lowest rank once the ranks run out (ties then share).
int age_rank(const vp_server* s)
{
    const int lowest = s->nranks - 1;
    int r = -1;
    for (int64_t id : s->running) r = std::max(r, s->jobs.at(id).rank);
    return std::min(lowest, r + 1);
}

// Admit waiting jobs, oldest first, while a lane is idle and the oldest fits.
void admit(vp_server* s)
{
    while (!s->waiting.empty()) {
        int lane = -1;
        for (int k = 0; k < s->nlanes; ++k)
            if (s->lane_job[k] == 0) { lane = k; break; }
        if (lane < 0) return;
        const int64_t id = s->waiting.front();
        Job& j = s->jobs[id];
        size_t off = 0;
        if (!s->pool->alloc(j.bytes, &off)) return;
        s->waiting.pop_front();
        j.off = off;
        j.lane = lane;
        s->lane_job[lane] = id;
        if (s->fake) {
            j.rank = age_rank(s);
            j.fake_t0 = host_ms(s);
            j.fake_t1 = j.fake_t0 + 1e-3 * j.desc.C;
            s->running.push_back(id);
            if ((int)s->running.size() > s->max_in_flight) s->max_in_flight = (int)s->running.size();
            continue;
        }
        vp::carve_state(s->pool_base + off, j.desc.C, j.plan.K, vp::p_rows(&j.plan), j.plan.n_paths, &j.plan.d);
        j.plan.cap = j.desc.C;
        j.plan.cap_mp = vp::p_rows(&j.plan);
        j.plan.C = j.desc.C;
        cudaStream_t st = s->lanes[lane];
        if (s->policy == VP_SERVE_AGE_PRIORITY) {
            j.rank = age_rank(s);
            st = s->ranked[j.rank][lane];
        }
        cudaError_t e = take_event(s, &j.ev0);
        if (e == cudaSuccess) e = take_event(s, &j.ev1);
        if (e == cudaSuccess && j.desc.ready_event)
            e = cudaStreamWaitEvent(st, static_cast<cudaEvent_t>(j.desc.ready_event), 0);
        if (e == cudaSuccess) e = cudaEventRecord(j.ev0, st);
        if (e == cudaSuccess)
            e = vp::enqueue_slot(&j.plan, static_cast<const float2*>(j.desc.H), j.desc.C, j.desc.sym_idx, j.desc.S,
                                 static_cast<float2*>(j.desc.x), j.desc.l, j.desc.gamma, j.desc.status, st);
        if (e == cudaSuccess) e = cudaEventRecord(j.ev1, st);
        if (e != cudaSuccess) {
            // the lane may still run what was enqueued: wait for it before
            // the state goes back to the pool
            cudaGetLastError();
            cudaStreamSynchronize(st);
            cudaGetLastError();
            j.status = VP_ERR_CUDA;
            finish(s, id, j, 0.f, 0.f);
            continue;
        }
        s->running.push_back(id);
        if ((int)s->running.size() > s->max_in_flight) s->max_in_flight = (int)s->running.size();
    }
}

void progress(vp_server* s)
{
    retire(s);
    admit(s);
}

// Clock zero: an event on lane 0 that the host waits for; the host clock is
// set when the wait returns, so host times read at most the wait's latency
// behind device times (caller holds the lock).
vp_status reset_ref(vp_server* s)
{
    if (!s->fake) {
        if (cudaEventRecord(s->ref, s->lanes[0]) != cudaSuccess || cudaEventSynchronize(s->ref) != cudaSuccess) {
            cudaGetLastError();
            return VP_ERR_CUDA;
        }
    }
    s->t_ref = std::chrono::steady_clock::now();
    return VP_OK;
}

// Validation and state size of a job (no lock needed).
vp_status prepare(const vp_server* s, const vp_job_desc& job, Job* j)
{
    if (!job_ok(job)) return VP_ERR_INVALID_ARG;
    j->desc = job;
    j->plan = plan_of(job);
    vp::DeviceState probe;
    j->bytes = vp::carve_state(nullptr, job.C, j->plan.K, vp::p_rows(&j->plan), j->plan.n_paths, &probe);
    if (round_up(j->bytes) > s->pool_bytes) return VP_ERR_CAPACITY;
    return VP_OK;
}

int64_t enqueue_job(vp_server* s, const Job& j)
{
    const int64_t k = s->next_id++;
    s->jobs.emplace(k, j);
    s->waiting.push_back(k);
    ++s->submitted;
    progress(s);
    return k;
}

void destroy_streams(std::vector<cudaStream_t>& v)
{
    for (cudaStream_t st : v) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    v.clear();
}

}  // namespace

extern "C" {

vp_status vp_server_create(size_t pool_bytes, int lanes, vp_server** out)
{
    if (!out) return VP_ERR_INVALID_ARG;
    *out = nullptr;
    if (pool_bytes < (size_t(1) << 20) || lanes < 1 || lanes > kMaxLanes) return VP_ERR_INVALID_ARG;
    vp_server* s = new (std::nothrow) vp_server();
    if (!s) return VP_ERR_OOM;
    s->pool = new (std::nothrow) Pool(pool_bytes);
    if (!s->pool) {
        delete s;
        return VP_ERR_OOM;
    }
    s->pool_bytes = pool_bytes;
    bool ok = cudaGetDevice(&s->device) == cudaSuccess;
    if (ok && cudaMalloc(reinterpret_cast<void**>(&s->pool_base), pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        vp_server_destroy(s);
        return VP_ERR_OOM;
    }
    for (int k = 0; ok && k < lanes; ++k) {
        cudaStream_t st = nullptr;
        ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) s->lanes.push_back(st);
    }
    s->nlanes = (int)s->lanes.size();
    s->lane_job.assign(s->lanes.size(), 0);
    ok = ok && cudaEventCreate(&s->ref) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        vp_server_destroy(s);
        return VP_ERR_CUDA;
    }
    if (vp_server_reset_clock(s) != VP_OK) {
        vp_server_destroy(s);
        return VP_ERR_CUDA;
    }
    *out = s;
    return VP_OK;
}

vp_status vp_server_create_fake(size_t pool_bytes, int lanes, vp_server** out)
{
    if (!out) return VP_ERR_INVALID_ARG;
    *out = nullptr;
    if (pool_bytes < (size_t(1) << 20) || lanes < 1 || lanes > kMaxLanes) return VP_ERR_INVALID_ARG;
    vp_server* s = new (std::nothrow) vp_server();
    if (!s) return VP_ERR_OOM;
    s->pool = new (std::nothrow) Pool(pool_bytes);
    if (!s->pool) {
        delete s;
        return VP_ERR_OOM;
    }
    s->fake = true;
    s->pool_bytes = pool_bytes;
    s->nlanes = lanes;
    s->lane_job.assign((size_t)lanes, 0);
    s->t_ref = std::chrono::steady_clock::now();
    *out = s;
    return VP_OK;
}

vp_status vp_server_submit(vp_server* s, const vp_job_desc* job, int64_t* id)
{
    if (!s || !job || !id) return VP_ERR_INVALID_ARG;
    Job j;
    const vp_status st = prepare(s, *job, &j);
    if (st != VP_OK) return st;
    std::lock_guard<std::mutex> lock(s->mu);
    *id = enqueue_job(s, j);
    return VP_OK;
}

vp_status vp_server_set_policy(vp_server* s, int policy)
{
    if (!s || (policy != VP_SERVE_FCFS && policy != VP_SERVE_AGE_PRIORITY)) return VP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->running.empty() || !s->waiting.empty()) return VP_ERR_INVALID_ARG;
    if (policy == s->policy) return VP_OK;
    if (s->fake) {
        s->nranks = policy == VP_SERVE_AGE_PRIORITY ? kFakeRanks : 1;
        s->policy = policy;
        return VP_OK;
    }
    for (auto& v : s->ranked) destroy_streams(v);
    s->ranked.clear();
    s->nranks = 1;
    s->policy = VP_SERVE_FCFS;
    if (policy == VP_SERVE_FCFS) return VP_OK;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return VP_ERR_CUDA;
    }
    // CUDA priorities: lower numbers run first; rank 0 takes `greatest`
    const int nr = std::max(1, least - greatest + 1);
    s->ranked.resize((size_t)nr);
    bool ok = true;
    for (int r = 0; ok && r < nr; ++r)
        for (int k = 0; ok && k < s->nlanes; ++k) {
            cudaStream_t st = nullptr;
            ok = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest + r) == cudaSuccess;
            if (ok) s->ranked[(size_t)r].push_back(st);
        }
    if (!ok) {
        cudaGetLastError();
        for (auto& v : s->ranked) destroy_streams(v);
        s->ranked.clear();
        return VP_ERR_CUDA;
    }
    s->nranks = nr;
    s->policy = policy;
    return VP_OK;
}

vp_status vp_server_replay(vp_server* s, const vp_job_desc* jobs, const double* arrival_ms, int n,
                           double timeout_s, vp_job_done* done, double* submit_ms)
{
    if (!s || n < 0 || (n > 0 && (!jobs || !arrival_ms || !done)) || !(timeout_s >= 0.0)) return VP_ERR_INVALID_ARG;
    std::vector<Job> js((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!(arrival_ms[i] >= 0.0) || !std::isfinite(arrival_ms[i]) || (i > 0 && arrival_ms[i] < arrival_ms[i - 1]))
            return VP_ERR_INVALID_ARG;
        const vp_status st = prepare(s, jobs[i], &js[(size_t)i]);
        if (st != VP_OK) return st;
    }
    int64_t first = 0;
    int got = 0;
    // moves this replay's finished records to `done` (caller holds the lock)
    auto collect = [&]() {
        for (auto it = s->finished.begin(); it != s->finished.end();) {
            const int64_t i = it->id - first;
            if (i < 0 || i >= n) {
                ++it;
                continue;
            }
            done[i] = *it;
            ++got;
            it = s->finished.erase(it);
        }
    };
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (!s->running.empty() || !s->waiting.empty()) return VP_ERR_INVALID_ARG;
        const vp_status st = reset_ref(s);
        if (st != VP_OK) return st;
        first = s->next_id;
    }
    for (int i = 0; i < n; ++i) {
        for (;;) {
            std::lock_guard<std::mutex> lock(s->mu);
            const double now = host_ms(s);
            if (now >= arrival_ms[i]) {
                if (submit_ms) submit_ms[i] = now;
                enqueue_job(s, js[(size_t)i]);
                collect();
                break;
            }
            progress(s);
            collect();
        }
    }
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            progress(s);
            collect();
            if (got == n) break;
        }
        if (std::chrono::steady_clock::now() >= t_end) return VP_ERR_TIMEOUT;
        std::this_thread::yield();
    }
    return VP_OK;
}

vp_status vp_server_poll(vp_server* s, vp_job_done* done, int max_done, int* n_done)
{
    if (!s || max_done < 0 || (max_done > 0 && !done)) return VP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    progress(s);
    int n = 0;
    while (n < max_done && !s->finished.empty()) {
        done[n++] = s->finished.front();
        s->finished.pop_front();
    }
    if (n_done) *n_done = n;
    return VP_OK;
}

vp_status vp_server_drain(vp_server* s, double timeout_s)
{
    if (!s || !(timeout_s >= 0.0)) return VP_ERR_INVALID_ARG;
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            progress(s);
            if (s->running.empty() && s->waiting.empty()) return VP_OK;
        }
        if (std::chrono::steady_clock::now() >= t_end) return VP_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

vp_status vp_server_reset_clock(vp_server* s)
{
    if (!s || s->nlanes < 1) return VP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fake) {
        s->t_ref = std::chrono::steady_clock::now();
        return VP_OK;
    }
    return reset_ref(s);
}

vp_status vp_server_get_stats(vp_server* s, vp_server_stats* out)
{
    if (!s || !out) return VP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    out->lanes = s->nlanes;
    out->queued = (int)s->waiting.size();
    out->in_flight = (int)s->running.size();
    out->max_in_flight = s->max_in_flight;
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->pool_bytes = s->pool_bytes;
    out->pool_used = s->pool->used();
    out->pool_high_water = s->pool->high();
    return VP_OK;
}

vp_status vp_server_destroy(vp_server* s)
{
    if (!s) return VP_OK;
    if (s->fake) {
        delete s->pool;
        delete s;
        return VP_OK;
    }
    for (cudaStream_t st : s->lanes) cudaStreamSynchronize(st);
    for (auto& v : s->ranked) destroy_streams(v);
    for (auto& kv : s->jobs) {
        if (kv.second.ev0) cudaEventDestroy(kv.second.ev0);
        if (kv.second.ev1) cudaEventDestroy(kv.second.ev1);
    }
    for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
    if (s->ref) cudaEventDestroy(s->ref);
    for (cudaStream_t st : s->lanes) cudaStreamDestroy(st);
    cudaFree(s->pool_base);
    cudaGetLastError();
    delete s->pool;
    delete s;
    return VP_OK;
}

}  // extern "C"
