// Request server: continuous batching of force solves on one GPU.
//
// Requests (a plan plus caller-owned device buffers) are queued by sg_submit.
// A worker thread admits them in arrival order while a slot (stream) is free
// and the device bytes of their per-request workspace fit in the server's
// budget; each admitted request gets its own workspace (stream-ordered
// allocation from the server's memory pool) and runs on its slot's stream, so
// requests that arrive while others run are started as soon as a slot and
// memory free up and overlap with them on the device. A host function enqueued
// after the solve marks completion; the worker then returns the workspace and
// the slot. Plans (kernel spectra, geometry tables) stay resident and are shared
// by all requests that use them; the work split of a solve depends only on its
// plan, so a result is bit-for-bit the same alone and in any mix.
//
// Requests of single in-plane patches with equal padded lengths, precision and
// slope handling that are queued together are admitted together as a group
// (up to the server's group limit, 16 by default) on one slot: each keeps its
// own workspace, and each pass of the convolution is one launch over all of
// them (group.cuh, the batches' grouped launches), with the same arithmetic
// per member, so a result is still bit-for-bit that of the request alone. The
// head of the queue is always admitted first; queued requests of its group
// join it out of arrival order.
//
// Nothing on the device waits for anything: completion is observed on the host.
#include "common.cuh"
#include "group.cuh"

#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_GPU_DONE = 2, RQ_FINISHED = 3 };

constexpr int GROUP_MAX = 16;   // members of one grouped admission (upper bound of the limit)
constexpr int GROUP_SCAN = 256; // queued requests looked at for the head's group

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct sg_group_run;

struct sg_request {
    uint64_t ticket = 0;
    sg_plan *plan = nullptr;
    const void *sigma = nullptr, *dx = nullptr, *dy = nullptr;
    void *fx = nullptr, *fy = nullptr;
    int64_t bytes = 0;
    int slot = -1;
    sg_workspace ws;
    std::atomic<int> state{RQ_QUEUED};
    sg_status result = SG_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    struct sg_server *server = nullptr;
    sg_group_run *group = nullptr;  // the grouped admission it runs in (NULL: alone)
};

// Requests admitted together on one slot; the slot and the device argument
// arrays are released when the last member has finished.
struct sg_group_run {
    int slot = -1;
    std::vector<sg_request *> members;
    void *dargs = nullptr;
    int pending = 0;
};

struct sg_server {
    int device = 0;
    int64_t budget = 0;
    int max_inflight = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<cudaStream_t> streams;
    int *err_host = nullptr;            // per slot: the request's device error word, copied after its solve (pinned)
    char *arg_host = nullptr;           // per slot: staging of a group's pass arguments (pinned)
    size_t arg_bytes = 0;               // per slot
    int group_limit = GROUP_MAX;        // 1: no grouping
    uint64_t groups_started = 0, grouped_requests = 0;
    std::vector<int> free_slots;
    std::deque<sg_request *> queue;
    std::vector<sg_request *> running;
    std::unordered_map<uint64_t, sg_request *> live;   // not yet retired by sg_poll / sg_wait
    int64_t bytes_in_use = 0, peak_bytes = 0;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, rejected = 0;
    std::vector<double> latency_ms;
    std::mutex mu;
    std::condition_variable wake;      // to the worker
    std::condition_variable finished;  // to waiters
    std::thread worker;
    bool stop = false;
};

namespace {

void CUDART_CB on_done(void *p)
{
    sg_request *r = (sg_request *)p;
    r->t_done = now_s();
    r->state.store(RQ_GPU_DONE);
    r->server->wake.notify_one();
}

// Finish a request whose GPU work completed (called with the lock held).
void finalize(sg_server *s, sg_request *r)
{
    sg_workspace_free(&r->ws, s->streams[r->slot], true);
    s->bytes_in_use -= r->bytes;
    // a bounded wait that ran out in one of the request's kernels (device error word;
    // a group's kernels report into its first member's word, copied to the slot's)
    if (r->result == SG_OK && s->err_host[r->slot] != 0) r->result = SG_ETIMEOUT;
    if (sg_group_run *g = r->group) {
        r->group = nullptr;
        if (--g->pending == 0) {
            if (g->dargs) cudaFreeAsync(g->dargs, s->streams[g->slot]);
            s->free_slots.push_back(g->slot);
            delete g;
        }
    } else {
        s->free_slots.push_back(r->slot);
    }
    r->slot = -1;
    if (r->result == SG_OK) {
        s->completed++;
        s->latency_ms.push_back(1e3 * (r->t_done - r->t_submit));
    } else {
        s->failed++;
    }
    r->state.store(RQ_FINISHED);
}

// Start a queued request on a free slot (lock held). Returns false when its
// workspace cannot be allocated now (it stays queued).
// The request's workspace, stream-ordered from the server's pool on `st`, its
// error word cleared; false (nothing held) when it cannot be allocated now.
bool alloc_ws(sg_server *s, sg_request *r, cudaStream_t st)
{
    memset(&r->ws, 0, sizeof(r->ws));
    sg_status a = SG_OK;
    {
        const sg_plan *p = r->plan;
        int64_t sizes[6] = {p->ws_fwd_bytes, p->ws_inv_bytes, p->ws_sfield_bytes, p->ws_tile_bytes,
                            p->ws_partial_bytes, 16};
        void **dst[6] = {&r->ws.work_fwd, &r->ws.work_inv, &r->ws.sfield, &r->ws.tile_w, (void **)&r->ws.partial,
                         (void **)&r->ws.err};
        for (int k = 0; k < 6 && a == SG_OK; ++k) {
            if (sizes[k] <= 0) continue;
            if (cudaMallocFromPoolAsync(dst[k], (size_t)sizes[k], s->pool, st) != cudaSuccess) {
                cudaGetLastError();
                *dst[k] = nullptr;
                a = SG_ENOMEM;
            }
        }
    }
    if (a == SG_OK && cudaMemsetAsync(r->ws.err, 0, 16, st) != cudaSuccess) a = SG_ECUDA;
    if (a != SG_OK) {
        sg_workspace_free(&r->ws, st, true);
        return false;
    }
    return true;
}

bool start(sg_server *s, sg_request *r)
{
    const int slot = s->free_slots.back();
    cudaStream_t st = s->streams[slot];
    if (!alloc_ws(s, r, st)) return false;
    s->free_slots.pop_back();
    r->slot = slot;
    s->bytes_in_use += r->bytes;
    s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
    r->t_start = now_s();
    r->state.store(RQ_RUNNING);
    s->err_host[slot] = 0;
    r->result = sg_force_ws(r->plan, &r->ws, r->sigma, r->dx, r->dy, r->fx, r->fy, st);
    if (r->result == SG_OK &&
        cudaMemcpyAsync(&s->err_host[slot], r->ws.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        r->result = SG_ECUDA;
    if (r->result != SG_OK || cudaLaunchHostFunc(st, on_done, r) != cudaSuccess) {
        if (r->result == SG_OK) r->result = SG_ECUDA;
        cudaGetLastError();
        cudaStreamSynchronize(st);
        r->t_done = now_s();
        r->state.store(RQ_GPU_DONE);
    }
    s->running.push_back(r);
    return true;
}

void CUDART_CB on_group_done(void *p)
{
    sg_group_run *g = (sg_group_run *)p;
    const double t = now_s();
    sg_server *s = g->members[0]->server;
    for (sg_request *r : g->members) {
        r->t_done = t;
        r->state.store(RQ_GPU_DONE);
    }
    s->wake.notify_one();
}

// Pack the members' pass arguments into the slot's pinned staging, copy them
// to a pool allocation and enqueue the grouped launches (lock held).
template <typename T>
sg_status group_launch(sg_server *s, sg_group_run *g, cudaStream_t st)
{
    const int m = (int)g->members.size();
    std::vector<sgk::uniform_passes<T>> us(m);
    int maxny = 0;
    for (int k = 0; k < m; ++k) {
        sg_request *r = g->members[k];
        const bool caller = r->plan->geom.slope_mode == SG_SLOPES_CALLER;
        us[k] = sgk::uniform_setup<T>(r->plan, &r->ws, 0, r->sigma, caller ? r->dx : nullptr,
                                      caller ? r->dy : nullptr, r->fx, r->fy, nullptr);
        if (us[k].rf.src.ny > maxny) maxny = us[k].rf.src.ny;
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t s0 = m * sizeof(sgk::row_fwd_args<T>), s1 = m * sizeof(sgk::edge_args<T>);
    const size_t s2 = m * sizeof(sgk::col_args<T>), s3 = m * sizeof(sgk::row_inv_args<T>);
    const size_t total = up(s0) + up(s1) + up(s2) + up(s3);
    if (total > s->arg_bytes) return SG_EINVAL;  // sized for GROUP_MAX members at creation
    char *h = s->arg_host + (size_t)g->slot * s->arg_bytes;
    for (int k = 0; k < m; ++k) {
        ((sgk::row_fwd_args<T> *)h)[k] = us[k].rf;
        ((sgk::edge_args<T> *)(h + up(s0)))[k] = us[k].ed;
        ((sgk::col_args<T> *)(h + up(s0) + up(s1)))[k] = us[k].col;
        ((sgk::row_inv_args<T> *)(h + up(s0) + up(s1) + up(s2)))[k] = us[k].ri;
    }
    char *d = nullptr;
    if (cudaMallocFromPoolAsync((void **)&d, total, s->pool, st) != cudaSuccess) {
        cudaGetLastError();
        return SG_ENOMEM;
    }
    g->dargs = d;
    SG_CUDA_TRY(cudaMemcpyAsync(d, h, total, cudaMemcpyHostToDevice, st));
    sgk::group_passes<T> gp;
    gp.u = us[0];
    gp.rf = (const sgk::row_fwd_args<T> *)d;
    gp.ed = (const sgk::edge_args<T> *)(d + up(s0));
    gp.col = (const sgk::col_args<T> *)(d + up(s0) + up(s1));
    gp.ri = (const sgk::row_inv_args<T> *)(d + up(s0) + up(s1) + up(s2));
    gp.bs = {m, maxny};
    gp.err = g->members[0]->ws.err;
    return sgk::group_enqueue<T>(gp, st);
}

// Start the requests `mem` (same group key; the queue's head first) together on
// a free slot (lock held). Returns false, holding nothing, when some member's
// workspace cannot be allocated now.
bool start_group(sg_server *s, const std::vector<sg_request *> &mem)
{
    const int slot = s->free_slots.back();
    cudaStream_t st = s->streams[slot];
    for (size_t k = 0; k < mem.size(); ++k) {
        if (!alloc_ws(s, mem[k], st)) {
            for (size_t q = 0; q < k; ++q) sg_workspace_free(&mem[q]->ws, st, true);
            return false;
        }
    }
    s->free_slots.pop_back();
    sg_group_run *g = new sg_group_run();
    g->slot = slot;
    g->members = mem;
    g->pending = (int)mem.size();
    const double t = now_s();
    for (sg_request *r : mem) {
        r->slot = slot;
        r->group = g;
        s->bytes_in_use += r->bytes;
        r->t_start = t;
        r->state.store(RQ_RUNNING);
        s->running.push_back(r);
    }
    s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
    s->err_host[slot] = 0;
    s->groups_started++;
    s->grouped_requests += mem.size();
    sg_status res = mem[0]->plan->prec == SG_FP64 ? group_launch<double>(s, g, st) : group_launch<float>(s, g, st);
    if (res == SG_OK &&
        cudaMemcpyAsync(&s->err_host[slot], mem[0]->ws.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        res = SG_ECUDA;
    if (res != SG_OK || cudaLaunchHostFunc(st, on_group_done, g) != cudaSuccess) {
        if (res == SG_OK) res = SG_ECUDA;
        cudaGetLastError();
        cudaStreamSynchronize(st);
        const double td = now_s();
        for (sg_request *r : mem) {
            r->result = res;
            r->t_done = td;
            r->state.store(RQ_GPU_DONE);
        }
    }
    return true;
}

// The head's group: queued requests with its key that fit the budget alongside
// it, in queue order, up to the group limit (lock held).
std::vector<sg_request *> collect_group(sg_server *s)
{
    std::vector<sg_request *> mem;
    sg_request *head = s->queue.front();
    mem.push_back(head);
    if (s->group_limit < 2 || !sgk::groupable(head->plan)) return mem;
    const auto key = sgk::group_key(head->plan);
    int64_t need = s->bytes_in_use + head->bytes;
    const size_t n = std::min(s->queue.size(), (size_t)GROUP_SCAN);
    for (size_t i = 1; i < n && (int)mem.size() < s->group_limit; ++i) {
        sg_request *q = s->queue[i];
        if (!sgk::groupable(q->plan) || sgk::group_key(q->plan) != key) continue;
        if (need + q->bytes > s->budget) continue;
        need += q->bytes;
        mem.push_back(q);
    }
    return mem;
}

void worker_main(sg_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        bool progressed = false;
        // completions
        for (size_t k = 0; k < s->running.size();) {
            sg_request *r = s->running[k];
            if (r->state.load() == RQ_GPU_DONE) {
                finalize(s, r);
                s->running[k] = s->running.back();
                s->running.pop_back();
                progressed = true;
            } else {
                ++k;
            }
        }
        if (progressed) s->finished.notify_all();
        // admissions, in arrival order (a head with queued requests of its group: together)
        while (!s->queue.empty() && !s->free_slots.empty() && !s->stop) {
            sg_request *r = s->queue.front();
            if (s->bytes_in_use + r->bytes > s->budget) break;
            const std::vector<sg_request *> grp = collect_group(s);
            if (grp.size() > 1 && start_group(s, grp)) {
                for (sg_request *q : grp) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), q));
                continue;
            }
            if (!start(s, r)) {
                if (!s->running.empty()) break;  // memory frees up when a running request ends
                // nothing running and still no memory: fail this request rather than wait forever
                s->queue.pop_front();
                r->result = SG_ENOMEM;
                r->state.store(RQ_FINISHED);
                s->failed++;
                s->finished.notify_all();
                continue;
            }
            s->queue.pop_front();
        }
        if (s->stop && s->running.empty()) break;
        s->wake.wait_for(lock, std::chrono::milliseconds(1));
    }
}

}  // namespace

extern "C" {

sg_status sg_server_create(size_t hbm_budget, int max_inflight, sg_server **out)
{
    if (!out || max_inflight < 1 || max_inflight > 256) return SG_EINVAL;
    sg_server *s = new (std::nothrow) sg_server();
    if (!s) return SG_ENOMEM;
    s->budget = hbm_budget ? (int64_t)hbm_budget : INT64_MAX;
    s->max_inflight = max_inflight;
    cudaError_t e = cudaGetDevice(&s->device);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool for the next request
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->err_host, sizeof(int) * max_inflight, cudaHostAllocDefault);
    if (e == cudaSuccess) memset(s->err_host, 0, sizeof(int) * max_inflight);
    {
        // a group's four argument arrays (FP64, the larger), each padded to 256 bytes
        auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
        s->arg_bytes = up(GROUP_MAX * sizeof(sgk::row_fwd_args<double>)) + up(GROUP_MAX * sizeof(sgk::edge_args<double>)) +
                       up(GROUP_MAX * sizeof(sgk::col_args<double>)) + up(GROUP_MAX * sizeof(sgk::row_inv_args<double>));
    }
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->arg_host, s->arg_bytes * max_inflight, cudaHostAllocDefault);
    for (int k = 0; k < max_inflight && e == cudaSuccess; ++k) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            s->streams.push_back(st);
            s->free_slots.push_back(k);
        }
    }
    if (e != cudaSuccess) {
        sg_set_last_cuda_error(e, "sg_server_create");
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        if (s->err_host) cudaFreeHost(s->err_host);
        if (s->arg_host) cudaFreeHost(s->arg_host);
        delete s;
        return SG_ECUDA;
    }
    std::reverse(s->free_slots.begin(), s->free_slots.end());
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SG_OK;
}

sg_status sg_server_destroy(sg_server *s)
{
    if (!s) return SG_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (sg_request *r : s->queue) {
            r->result = SG_ECANCELLED;
            r->state.store(RQ_FINISHED);
            s->cancelled++;
        }
        s->queue.clear();
        s->stop = true;
    }
    s->wake.notify_one();
    s->worker.join();
    for (auto &kv : s->live) delete kv.second;
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    cudaMemPoolDestroy(s->pool);
    cudaFreeHost(s->err_host);
    cudaFreeHost(s->arg_host);
    delete s;
    return SG_OK;
}

sg_status sg_server_set_group_limit(sg_server *s, int max_members)
{
    if (!s || max_members < 1 || max_members > GROUP_MAX) return SG_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    s->group_limit = max_members;
    return SG_OK;
}

sg_status sg_submit(sg_server *s, sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx,
                    void *fy, uint64_t *ticket)
{
    if (!s || !plan || !sigma || !fx || !fy || !ticket) return SG_EINVAL;
    if (plan->geom.slope_mode == SG_SLOPES_CALLER && (!deltax || !deltay)) return SG_EINVAL;
    if (plan->device != s->device) return SG_EINVAL;
    sg_request *r = new (std::nothrow) sg_request();
    if (!r) return SG_ENOMEM;
    r->plan = plan;
    r->sigma = sigma;
    r->dx = deltax;
    r->dy = deltay;
    r->fx = fx;
    r->fy = fy;
    r->bytes = sg_workspace_bytes(plan);
    r->server = s;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (r->bytes > s->budget) {
            s->rejected++;
            delete r;
            return SG_EBUDGET;
        }
        if (s->stop) {
            delete r;
            return SG_ECANCELLED;
        }
        r->ticket = s->next_ticket++;
        s->live[r->ticket] = r;
        s->queue.push_back(r);
        s->submitted++;
        *ticket = r->ticket;
    }
    s->wake.notify_one();
    return SG_OK;
}

// Report a finished request and retire its ticket (lock held).
static sg_status report(sg_server *s, sg_request *r, sg_status *result, double *latency_ms)
{
    if (result) *result = r->result;
    if (latency_ms) *latency_ms = r->result == SG_OK ? 1e3 * (r->t_done - r->t_submit) : 0.0;
    s->live.erase(r->ticket);
    delete r;
    return SG_OK;
}

sg_status sg_poll(sg_server *s, uint64_t ticket, sg_status *result, double *latency_ms)
{
    if (!s) return SG_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return SG_ENOTFOUND;
    sg_request *r = it->second;
    if (r->state.load() != RQ_FINISHED) return SG_EBUSY;
    return report(s, r, result, latency_ms);
}

sg_status sg_wait(sg_server *s, uint64_t ticket, double timeout_ms, sg_status *result, double *latency_ms)
{
    if (!s || !(timeout_ms >= 0.0)) return SG_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1e3));
    for (;;) {
        auto it = s->live.find(ticket);
        if (it == s->live.end()) return SG_ENOTFOUND;
        sg_request *r = it->second;
        if (r->state.load() == RQ_FINISHED) return report(s, r, result, latency_ms);
        if (s->finished.wait_until(lock, deadline) == std::cv_status::timeout) {
            if (r->state.load() == RQ_FINISHED) return report(s, r, result, latency_ms);
            return SG_ETIMEOUT;
        }
    }
}

sg_status sg_cancel(sg_server *s, uint64_t ticket)
{
    if (!s) return SG_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return SG_ENOTFOUND;
    sg_request *r = it->second;
    auto q = std::find(s->queue.begin(), s->queue.end(), r);
    if (q == s->queue.end()) return r->state.load() == RQ_FINISHED ? SG_OK : SG_EBUSY;
    s->queue.erase(q);
    r->result = SG_ECANCELLED;
    r->state.store(RQ_FINISHED);
    s->cancelled++;
    s->finished.notify_all();
    return SG_OK;
}

sg_status sg_server_get_stats(sg_server *s, sg_server_stats *out, int reset_latencies)
{
    if (!s || !out) return SG_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->cancelled = s->cancelled;
    out->rejected = s->rejected;
    out->queued = (int64_t)s->queue.size();
    out->running = (int64_t)s->running.size();
    out->bytes_in_use = s->bytes_in_use;
    out->peak_bytes = s->peak_bytes;
    std::vector<double> v = s->latency_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
        return v[std::min(i, v.size() - 1)];
    };
    out->latency_count = (int64_t)v.size();
    out->latency_p50_ms = pct(0.50);
    out->latency_p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->latency_mean_ms = v.empty() ? 0.0 : sum / (double)v.size();
    out->groups_started = s->groups_started;
    out->grouped_requests = s->grouped_requests;
    if (reset_latencies) s->latency_ms.clear();
    return SG_OK;
}

}  // extern "C"
