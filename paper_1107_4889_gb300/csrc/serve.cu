// serve.cu -- request server: continuous batching of independent coupled
// solves on one GPU (include/rbc.h, "Request server").
//
// Each admitted solve is an rbc_handle whose workspace is carved from the
// caller's arena (first fit over a free list with coalescing) and whose work
// runs on a stream of the server's pool.  A solve advances in ticks: one
// CUDA graph of tick_steps coupled steps followed by the budget reduction,
// which adds the work rate and momentum of the pass to the solve's device
// time-average sums once the pass count reaches average_from.  Up to two
// ticks per solve are in flight; the host only polls their events, so
// solves of different sizes progress independently and their kernels
// overlap on the device.  A finished solve reads its sums, frees its handle
// and arena block, and the next queued requests that fit are admitted:
// the polling thread reserves the arena block and a stream, and a worker
// thread runs rbc_init and the tick-graph captures (host work of
// milliseconds) while the running solves keep the device busy.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rbc.h"
#include "internal.h"

namespace {

constexpr int kLookahead = 16;  // queued requests considered per admission round
constexpr int kInFlight = 2;    // ticks per solve queued on its stream

// A request with its inputs copied; the pointers of r point into the vectors.
struct Owned {
    rbc_request r;
    std::vector<uint8_t> solid;
    std::vector<double> pos, quat, vel, om;
    double t_submit = 0.0;
    size_t bytes = 0;
};

// First-fit allocator over [0, size) in 256-byte granules.
struct Arena {
    std::map<size_t, size_t> free_;  // offset -> length, disjoint, coalesced
    size_t size = 0;
    void init(size_t n)
    {
        size = n & ~size_t(255);
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t *off)
    {
        n = (n + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n;
            const size_t at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) & ~size_t(255);
        auto it = free_.emplace(off, n).first;
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
};

struct Active {
    std::unique_ptr<Owned> req;
    rbc_handle *h = nullptr;
    size_t off = 0;
    int stream_slot = -1;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t tick = nullptr, last = nullptr;  // tick_steps steps; the remainder
    int64_t total = 0, launched = 0;
    cudaEvent_t ev[kInFlight] = {nullptr, nullptr};
    int head = 0, in_flight = 0;
    double t_admit = 0.0;
    int status = RBC_OK;
};

double seconds_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct rbc_server {
    char *base = nullptr;
    Arena arena;
    int max_active = 0, tick_steps = 0, device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<int> free_streams;
    std::deque<std::unique_ptr<Owned>> queue;
    std::vector<std::unique_ptr<Active>> active;
    std::deque<rbc_result> done;
    std::chrono::steady_clock::time_point t0;
    // admission worker: solves reserved by poll wait in to_init, come back
    // initialised (or failed) in ready; `pending` counts both and the one
    // being initialised
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Active>> to_init, ready;
    int pending = 0;
    bool stop = false;
};

namespace {

int fail(const std::string &msg, int code)
{
    rbc::set_thread_error(msg.c_str());
    return code;
}

void release(rbc_server *s, Active &a)
{
    for (auto &e : a.ev)
        if (e) {
            cudaEventSynchronize(e);
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (a.tick) cudaGraphExecDestroy(a.tick);
    if (a.last) cudaGraphExecDestroy(a.last);
    a.tick = a.last = nullptr;
    if (a.h) rbc_free(a.h);
    a.h = nullptr;
    if (a.req) s->arena.release(a.off, a.req->bytes);
    if (a.stream_slot >= 0) s->free_streams.push_back(a.stream_slot);
    a.stream_slot = -1;
}

void finish(rbc_server *s, Active &a)
{
    rbc_result res;
    std::memset(&res, 0, sizeof res);
    res.tag = a.req->r.tag;
    res.status = a.status;
    res.t_submit = a.req->t_submit;
    res.t_admit = a.t_admit;
    res.workspace_bytes = a.req->bytes;
    if (a.h && a.status == RBC_OK) {
        double acc[8];
        int flags[8];
        int rc = rbc::read_accum(a.h, acc, flags);
        if (rc == RBC_OK && (flags[0] || acc[6] > 0.0)) rc = RBC_EUNSTABLE;
        if (rc == RBC_OK && flags[1]) rc = RBC_ENOMEM;
        if (rc == RBC_OK && flags[2]) rc = RBC_ETIMEOUT;
        res.status = rc;
        res.steps = a.launched;
        res.samples = (int64_t)acc[1];
        if (acc[1] > 0.0) {
            res.mean_power = acc[0] / acc[1];
            for (int k = 0; k < 3; ++k) res.mean_p_fluid[k] = acc[2 + k] / acc[1];
        }
        res.max_u = acc[5];
    }
    release(s, a);
    res.t_done = seconds_since(s->t0);
    s->done.push_back(res);
}

// Queue the next tick of a solve on its stream.
int launch_tick(Active &a, int tick_steps)
{
    const int64_t n = std::min<int64_t>(tick_steps, a.total - a.launched);
    cudaGraphExec_t g = n == tick_steps ? a.tick : a.last;
    if (!g) return RBC_ECUDA;
    if (cudaGraphLaunch(g, a.stream) != cudaSuccess) return RBC_ECUDA;
    if (cudaEventRecord(a.ev[(a.head + a.in_flight) % kInFlight], a.stream) != cudaSuccess) return RBC_ECUDA;
    a.in_flight++;
    a.launched += n;
    rbc::advance_steps(a.h, n);
    return RBC_OK;
}

// Reserve a stream slot for a solve whose arena block is taken and hand it
// to the admission worker.
void admit(rbc_server *s, std::unique_ptr<Owned> req, size_t off)
{
    std::unique_ptr<Active> a(new Active());
    a->req = std::move(req);
    a->off = off;
    a->t_admit = seconds_since(s->t0);
    a->total = a->req->r.steps;
    a->stream_slot = s->free_streams.back();
    s->free_streams.pop_back();
    a->stream = s->streams[a->stream_slot];
    std::lock_guard<std::mutex> lock(s->mu);
    s->to_init.push_back(std::move(a));
    s->pending++;
    s->cv.notify_one();
}

// Worker side of admission: rbc_init in the reserved block (it captures the
// step graphs and synchronises only the solve's stream) and the tick
// graphs.  Errors are kept in the solve's status.
void initialise(rbc_server *s, Active &a)
{
    rbc_params p = a.req->r.params;
    p.stream = a.stream;
    int rc = rbc_init(&a.req->r.geom, &a.req->r.cells, &p, s->base + a.off, a.req->bytes, &a.h);
    const long long from = a.req->r.average_from;
    if (rc == RBC_OK && a.total >= s->tick_steps) rc = rbc::capture_ticks(a.h, s->tick_steps, from, &a.tick);
    if (rc == RBC_OK && a.total % s->tick_steps) rc = rbc::capture_ticks(a.h, a.total % s->tick_steps, from, &a.last);
    for (int k = 0; rc == RBC_OK && k < kInFlight; ++k)
        if (cudaEventCreateWithFlags(&a.ev[k], cudaEventDisableTiming) != cudaSuccess) rc = RBC_ECUDA;
    a.status = rc;
}

void worker_main(rbc_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::unique_ptr<Active> a;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv.wait(lock, [s] { return s->stop || !s->to_init.empty(); });
            if (s->stop) return;
            a = std::move(s->to_init.front());
            s->to_init.pop_front();
        }
        initialise(s, *a);
        std::lock_guard<std::mutex> lock(s->mu);
        s->ready.push_back(std::move(a));
    }
}

}  // namespace

extern "C" {

int rbc_server_create(void *arena, size_t arena_bytes, int max_active, int tick_steps, rbc_server **out)
{
    if (!out) return fail("out is NULL", RBC_EINVAL);
    *out = nullptr;
    if (!arena || (reinterpret_cast<uintptr_t>(arena) & 255u)) return fail("arena must be 256-byte aligned", RBC_EINVAL);
    if (max_active < 1 || max_active > 256) return fail("max_active must be 1..256", RBC_EINVAL);
    if (tick_steps < 2 || tick_steps > 100000 || tick_steps % 2)
        return fail("tick_steps must be even, 2..100000", RBC_EINVAL);
    rbc_server *s = new (std::nothrow) rbc_server();
    if (!s) return fail("host allocation failed", RBC_ENOMEM);
    s->base = static_cast<char *>(arena);
    s->arena.init(arena_bytes);
    s->max_active = max_active;
    s->tick_steps = tick_steps;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    for (int k = 0; k < max_active; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            rbc_server_free(s);
            return fail("stream creation failed", RBC_ECUDA);
        }
        s->streams.push_back(st);
        s->free_streams.push_back(max_active - 1 - k);
    }
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        rbc_server_free(s);
        return fail("could not start the admission thread", RBC_ENOMEM);
    }
    *out = s;
    return RBC_OK;
}

int rbc_server_submit(rbc_server *s, const rbc_request *r)
{
    if (!s || !r) return fail("NULL argument", RBC_EINVAL);
    if (r->steps < 1) return fail("steps must be >= 1", RBC_EINVAL);
    std::unique_ptr<Owned> o(new (std::nothrow) Owned());
    if (!o) return fail("host allocation failed", RBC_ENOMEM);
    o->r = *r;
    const rbc_geometry &g = r->geom;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return fail("bad lattice", RBC_EINVAL);
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    if (g.solid) {
        o->solid.assign(g.solid, g.solid + N);
        o->r.geom.solid = o->solid.data();
    }
    const int n = r->cells.n;
    if (n < 0) return fail("negative cell count", RBC_EINVAL);
    if (n > 0) {
        if (!r->cells.pos || !r->cells.quat) return fail("cell positions and quaternions are required", RBC_EINVAL);
        o->pos.assign(r->cells.pos, r->cells.pos + 3 * (size_t)n);
        o->quat.assign(r->cells.quat, r->cells.quat + 4 * (size_t)n);
        o->r.cells.pos = o->pos.data();
        o->r.cells.quat = o->quat.data();
        if (r->cells.vel) {
            o->vel.assign(r->cells.vel, r->cells.vel + 3 * (size_t)n);
            o->r.cells.vel = o->vel.data();
        }
        if (r->cells.omega_body) {
            o->om.assign(r->cells.omega_body, r->cells.omega_body + 3 * (size_t)n);
            o->r.cells.omega_body = o->om.data();
        }
    }
    int rc = rbc_workspace_size(&o->r.geom, &o->r.cells, &o->r.params, &o->bytes);
    if (rc != RBC_OK) return rc;
    if (((o->bytes + 255) & ~size_t(255)) > s->arena.size) return fail("request larger than the arena", RBC_ENOMEM);
    o->t_submit = seconds_since(s->t0);
    s->queue.push_back(std::move(o));
    return RBC_OK;
}

int rbc_server_poll(rbc_server *s, int *active, int *queued)
{
    if (!s) return fail("server is NULL", RBC_EINVAL);
    int err = RBC_OK;
    // progress of the running solves
    for (size_t i = 0; i < s->active.size();) {
        Active &a = *s->active[i];
        while (a.in_flight > 0) {
            const cudaError_t e = cudaEventQuery(a.ev[a.head]);
            if (e == cudaErrorNotReady) break;
            if (e != cudaSuccess) {
                a.status = RBC_ECUDA;
                err = RBC_ECUDA;
                a.in_flight = 0;
                break;
            }
            a.in_flight--;
            a.head = (a.head + 1) % kInFlight;
        }
        if (a.status == RBC_OK) {
            while (a.in_flight < kInFlight && a.launched < a.total) {
                const int rc = launch_tick(a, s->tick_steps);
                if (rc != RBC_OK) {
                    a.status = rc;
                    break;
                }
            }
        }
        if ((a.launched >= a.total && a.in_flight == 0) || a.status != RBC_OK) {
            finish(s, a);
            s->active.erase(s->active.begin() + (long)i);
        } else {
            ++i;
        }
    }
    // solves the worker has initialised start their first ticks
    std::deque<std::unique_ptr<Active>> ready;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        ready.swap(s->ready);
        s->pending -= (int)ready.size();
    }
    for (auto &a : ready) {
        for (int k = 0; a->status == RBC_OK && k < kInFlight && a->launched < a->total; ++k)
            a->status = launch_tick(*a, s->tick_steps);
        if (a->status != RBC_OK) {
            finish(s, *a);
            continue;
        }
        s->active.push_back(std::move(a));
    }
    // admission in arrival order; a request that does not fit yet is passed over
    int pending = 0;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        pending = s->pending;
    }
    int looked = 0;
    for (auto it = s->queue.begin(); it != s->queue.end() && looked < kLookahead;) {
        if ((int)s->active.size() + pending >= s->max_active || s->free_streams.empty()) break;
        size_t off = 0;
        if (s->arena.alloc((*it)->bytes, &off)) {
            std::unique_ptr<Owned> o = std::move(*it);
            it = s->queue.erase(it);
            admit(s, std::move(o), off);
            ++pending;
        } else {
            ++it;
            ++looked;
        }
    }
    if (active) *active = (int)s->active.size() + pending;
    if (queued) *queued = (int)s->queue.size();
    return err;
}

int rbc_server_results(rbc_server *s, rbc_result *out, int max, int *n)
{
    if (!s || !n || (max > 0 && !out)) return fail("NULL argument", RBC_EINVAL);
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return RBC_OK;
}

double rbc_server_clock(const rbc_server *s) { return s ? seconds_since(s->t0) : 0.0; }

void rbc_server_free(rbc_server *s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->worker.join();
    }
    for (auto &a : s->ready) release(s, *a);
    for (auto &a : s->to_init) release(s, *a);
    s->ready.clear();
    s->to_init.clear();
    for (auto &a : s->active) release(s, *a);
    s->active.clear();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete s;
}

}  // extern "C"
