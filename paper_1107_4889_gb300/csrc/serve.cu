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
    std::vector<double> pos, quat, vel, om, fext, text;
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
    bool released = false;  // arena block returned
};

double seconds_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// A pack: the solves of one class (storage type, walls, stress; all with
// cells and a row-staged lattice pass) advanced together, each kernel of the
// step launched once for all of them over device tables of their
// arguments.  Members change only between ticks.
struct Pack {
    long long key = -1;
    std::vector<std::unique_ptr<Active>> members, joining;
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};  // main, side (bins, Gay-Berne), side 2 (weights)
    cudaEvent_t fork = nullptr, join1 = nullptr, join2 = nullptr, done[2] = {nullptr, nullptr};
    cudaGraphExec_t pair = nullptr, budgets = nullptr;  // two packed steps; the members' budgets
    int in_flight = 0, head = 0;  // ticks queued (at most 2) and the oldest one's event
    size_t off = 0, bytes = 0;  // table region in the arena
    rbc::CellPackDesc cd;
    rbc::LbPackDesc ld;
    std::vector<char> host;
};

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
    std::vector<std::unique_ptr<Pack>> packs;
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
    if (a.req && !a.released) s->arena.release(a.off, a.req->bytes);
    a.released = true;
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
        // the final state, where the caller asked for it (the solve's work
        // has completed: its ticks are retired)
        const rbc_request &r = a.req->r;
        if (res.status == RBC_OK && (r.out_rho || r.out_u || r.out_cells))
            res.status = rbc_fields(a.h, r.out_rho, r.out_u, r.out_cells);
        if (res.status == RBC_OK && r.out_diag) res.status = rbc_cell_diag(a.h, r.out_diag);
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
    // packable solves run their full ticks in a pack
    const bool packable = rc == RBC_OK && rbc::handle_dev(a.h).nc > 0 && rbc::handle_dev(a.h).lb_grid > 0 &&
                          !rbc::handle_dev(a.h).compact;
    if (rc == RBC_OK && a.total >= s->tick_steps && !packable)
        rc = rbc::capture_ticks(a.h, s->tick_steps, from, &a.tick);
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

// class of a solve: storage type, walls, cells, stress output, and the
// shape-function box (the packed shape-list launch sizes its shared memory
// for one box)
long long pack_key(const rbc::Dev &d, const rbc::Params &p)
{
    return (((long long)p.box_dim * 65536 + p.sup_cap) * 4 + d.prec) * 8 + (d.walls ? 4 : 0) + (d.nc > 0 ? 2 : 0) +
           (d.S ? 1 : 0);
}

// packs hold dense lattices with cells (the packed lattice pass is row-staged)
bool packable(const Active &a)
{
    return a.h && rbc::handle_dev(a.h).nc > 0 && rbc::handle_dev(a.h).lb_grid > 0 && !rbc::handle_dev(a.h).compact;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Table region of a pack: per member one lattice and one cell entry, the
// block / batch starts of every packed launch, and the lattice pass's two
// work counters.
size_t pack_bytes(int cap)
{
    return align256(cap * rbc::lb_pack_entry_bytes()) + align256(cap * rbc::cell_pack_entry_bytes()) +
           (rbc::PACK_KINDS + 1) * align256((cap + 1) * sizeof(int)) + 256;
}

Pack *get_pack(rbc_server *s, long long key)
{
    for (auto &p : s->packs)
        if (p->key == key) return p.get();
    std::unique_ptr<Pack> p(new Pack());
    p->key = key;
    p->bytes = pack_bytes(s->max_active);
    if (!s->arena.alloc(p->bytes, &p->off)) return nullptr;
    bool ok = true;
    for (auto &st : p->st) ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t *e : {&p->fork, &p->join1, &p->join2, &p->done[0], &p->done[1]})
        ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    // the lattice pass's work counters start at zero (the pass leaves them so)
    const size_t work_off = p->off + p->bytes - 256;
    ok = ok && cudaMemsetAsync(s->base + work_off, 0, 256, p->st[0]) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(p->st[0]) == cudaSuccess;
    if (!ok) {
        for (auto &st : p->st)
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t e : {p->fork, p->join1, p->join2, p->done[0], p->done[1]})
            if (e) cudaEventDestroy(e);
        s->arena.release(p->off, p->bytes);
        return nullptr;
    }
    s->packs.push_back(std::move(p));
    return s->packs.back().get();
}

// Rebuild a pack's tables and capture its two graphs: a pair of packed
// steps (per step: the per-cell kernel, then the lattice pass beside the
// next step's shape lists, cell list and Gay-Berne forces, as in a single
// solve's step), launched tick_steps / 2 times per tick, and the members'
// budget reductions into their time-average sums, launched once per tick.
// Small graphs keep a membership change cheap.
int rebuild_pack(rbc_server *s, Pack &pk)
{
    const int n = (int)pk.members.size();
    if (pk.pair) cudaGraphExecDestroy(pk.pair);
    if (pk.budgets) cudaGraphExecDestroy(pk.budgets);
    pk.pair = pk.budgets = nullptr;
    if (n == 0) return RBC_OK;
    const size_t lbe = rbc::lb_pack_entry_bytes(), ce = rbc::cell_pack_entry_bytes();
    const size_t cap = (size_t)s->max_active;
    const size_t off_lb = 0, off_c = align256(cap * lbe), off_st = off_c + align256(cap * ce);
    const size_t st_stride = align256((cap + 1) * sizeof(int));
    pk.host.assign(pk.bytes - 256, 0);
    std::vector<int> starts((rbc::PACK_KINDS + 1) * (n + 1), 0);
    int *bstart = &starts[rbc::PACK_KINDS * (n + 1)];
    int stage_bytes = 0;
    for (int i = 0; i < n; ++i) {
        const rbc::Dev &d = rbc::handle_dev(pk.members[i]->h);
        const rbc::Params &p = rbc::handle_params(pk.members[i]->h);
        int nb = 0, sb = 0;
        if (!rbc::fill_lb_pack_entry(d, p, &pk.host[off_lb + i * lbe], &nb, &sb)) return RBC_EINVAL;
        rbc::fill_cell_pack_entry(d, p, &pk.host[off_c + i * ce]);
        bstart[i + 1] = bstart[i] + nb;
        stage_bytes = std::max(stage_bytes, sb);
        for (int k = 0; k < rbc::PACK_KINDS; ++k)
            starts[k * (n + 1) + i + 1] = starts[k * (n + 1) + i] + rbc::cell_pack_blocks(d.nc, d.nbins, k);
    }
    for (int k = 0; k <= rbc::PACK_KINDS; ++k)
        std::memcpy(&pk.host[off_st + k * st_stride], &starts[k * (n + 1)], (n + 1) * sizeof(int));
    char *dev = s->base + pk.off;
    if (cudaMemcpyAsync(dev, pk.host.data(), pk.host.size(), cudaMemcpyHostToDevice, pk.st[0]) != cudaSuccess)
        return RBC_ECUDA;
    pk.cd.tab = dev + off_c;
    for (int k = 0; k < rbc::PACK_KINDS; ++k) {
        pk.cd.start[k] = reinterpret_cast<const int *>(dev + off_st + k * st_stride);
        pk.cd.blocks[k] = starts[k * (n + 1) + n];
    }
    pk.cd.ninst = n;
    pk.ld.tab = dev + off_lb;
    pk.ld.bstart = reinterpret_cast<const int *>(dev + off_st + rbc::PACK_KINDS * st_stride);
    pk.ld.total = bstart[n];
    pk.ld.ninst = n;
    pk.ld.work = reinterpret_cast<int *>(dev + pk.bytes - 256);
    pk.ld.stage_bytes = stage_bytes;
    const rbc::Dev &d0 = rbc::handle_dev(pk.members[0]->h);
    const rbc::Params &p0 = rbc::handle_params(pk.members[0]->h);
    if (!rbc::prepare_lb_pack(d0, pk.ld)) return RBC_EINVAL;
    const bool alpha = d0.S != nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(pk.st[0], cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RBC_ECUDA;
    for (int k = 0; k < 2; ++k) {
        const int par = k & 1;
        rbc::launch_cells_packed(pk.cd, par, alpha, pk.st[0]);
        cudaEventRecord(pk.fork, pk.st[0]);
        cudaStreamWaitEvent(pk.st[1], pk.fork, 0);
        cudaStreamWaitEvent(pk.st[2], pk.fork, 0);
        rbc::launch_weights_packed(pk.cd, p0, par ^ 1, d0.side_prio, pk.st[2]);
        rbc::launch_bin_packed(pk.cd, d0.side_prio, pk.st[1]);
        rbc::launch_gb_packed(pk.cd, d0.side_prio, pk.st[1]);
        rbc::launch_lb_packed(d0, pk.ld, par, pk.st[0]);
        cudaEventRecord(pk.join1, pk.st[1]);
        cudaEventRecord(pk.join2, pk.st[2]);
        cudaStreamWaitEvent(pk.st[0], pk.join1, 0);
        cudaStreamWaitEvent(pk.st[0], pk.join2, 0);
    }
    if (cudaStreamEndCapture(pk.st[0], &g) != cudaSuccess) return RBC_ECUDA;
    cudaError_t e = cudaGraphInstantiate(&pk.pair, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return RBC_ECUDA;
    if (cudaStreamBeginCapture(pk.st[0], cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RBC_ECUDA;
    for (auto &m : pk.members)
        rbc::launch_budget(rbc::handle_dev(m->h), rbc::handle_params(m->h), 0, pk.st[0], true,
                           m->req->r.average_from);
    if (cudaStreamEndCapture(pk.st[0], &g) != cudaSuccess) return RBC_ECUDA;
    e = cudaGraphInstantiate(&pk.budgets, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? RBC_OK : RBC_ECUDA;
}

// Queue one tick of the pack: tick_steps / 2 launches of the step pair,
// the budgets, the tick's event.
int launch_pack_tick(rbc_server *s, Pack &pk)
{
    bool ok = true;
    for (int k = 0; ok && k < s->tick_steps / 2; ++k) ok = cudaGraphLaunch(pk.pair, pk.st[0]) == cudaSuccess;
    ok = ok && cudaGraphLaunch(pk.budgets, pk.st[0]) == cudaSuccess;
    ok = ok && cudaEventRecord(pk.done[(pk.head + pk.in_flight) % 2], pk.st[0]) == cudaSuccess;
    if (!ok) return RBC_ECUDA;
    pk.in_flight++;
    for (auto &m : pk.members) {
        m->launched += s->tick_steps;
        rbc::advance_steps(m->h, s->tick_steps);
    }
    return RBC_OK;
}

void fail_pack(rbc_server *s, Pack &pk, int rc)
{
    for (auto &m : pk.members) {
        m->status = rc;
        finish(s, *m);
    }
    pk.members.clear();
}

// Retire the pack's completed ticks.  With no tick queued (a tick
// boundary): retire finished members, hand members with fewer than a tick
// of steps left to their own streams, take in joining solves, rebuild if
// anything changed and queue the next tick.  With one tick queued, nobody
// waiting to join and every member at least a tick from its end, queue the
// following tick behind it so the device does not wait for the host.
int progress_pack(rbc_server *s, Pack &pk)
{
    while (pk.in_flight > 0) {
        const cudaError_t e = cudaEventQuery(pk.done[pk.head]);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) {
            pk.in_flight = 0;
            fail_pack(s, pk, RBC_ECUDA);
            return RBC_ECUDA;
        }
        pk.in_flight--;
        pk.head = (pk.head + 1) % 2;
    }
    if (pk.in_flight == 1 && pk.joining.empty()) {
        bool room = !pk.members.empty();
        for (auto &m : pk.members) room = room && m->status == RBC_OK && m->total - m->launched >= s->tick_steps;
        if (room) {
            const int rc = launch_pack_tick(s, pk);
            if (rc != RBC_OK) fail_pack(s, pk, rc);
            return rc;
        }
    }
    if (pk.in_flight > 0) return RBC_OK;
    bool changed = false;
    for (size_t i = 0; i < pk.members.size();) {
        Active &a = *pk.members[i];
        if (a.status != RBC_OK || a.launched >= a.total) {
            finish(s, a);
        } else if (a.total - a.launched < s->tick_steps) {
            a.status = launch_tick(a, s->tick_steps);  // the remainder, on the solve's own stream
            s->active.push_back(std::move(pk.members[i]));
        } else {
            ++i;
            continue;
        }
        pk.members.erase(pk.members.begin() + (long)i);
        changed = true;
    }
    for (auto &a : pk.joining) pk.members.push_back(std::move(a));
    if (!pk.joining.empty()) changed = true;
    pk.joining.clear();
    if (pk.members.empty()) return RBC_OK;
    if (changed || !pk.pair) {
        const int rc = rebuild_pack(s, pk);
        if (rc != RBC_OK) {
            fail_pack(s, pk, rc);
            return rc;
        }
    }
    const int rc = launch_pack_tick(s, pk);
    if (rc != RBC_OK) fail_pack(s, pk, rc);
    return rc;
}

int pack_count(const rbc_server *s)
{
    int n = 0;
    for (auto &p : s->packs) n += (int)(p->members.size() + p->joining.size());
    return n;
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
        if (r->cells.force_ext) {
            o->fext.assign(r->cells.force_ext, r->cells.force_ext + 3 * (size_t)n);
            o->r.cells.force_ext = o->fext.data();
        }
        if (r->cells.torque_ext) {
            o->text.assign(r->cells.torque_ext, r->cells.torque_ext + 3 * (size_t)n);
            o->r.cells.torque_ext = o->text.data();
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
    // packs advance between their ticks
    for (auto &pk : s->packs) {
        const int rc = progress_pack(s, *pk);
        if (rc != RBC_OK) err = rc;
    }
    // solves the worker has initialised join a pack (from its next tick) or
    // start their own ticks
    std::deque<std::unique_ptr<Active>> ready;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        ready.swap(s->ready);
        s->pending -= (int)ready.size();
    }
    for (auto &a : ready) {
        if (a->status == RBC_OK && packable(*a) && a->total >= s->tick_steps) {
            Pack *pk = get_pack(s, pack_key(rbc::handle_dev(a->h), rbc::handle_params(a->h)));
            if (pk) {
                pk->joining.push_back(std::move(a));
                if (pk->in_flight == 0) progress_pack(s, *pk);
                continue;
            }
            // no room for a pack's tables: this solve runs on its own
            a->status = rbc::capture_ticks(a->h, s->tick_steps, a->req->r.average_from, &a->tick);
        }
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
        if ((int)s->active.size() + pack_count(s) + pending >= s->max_active || s->free_streams.empty()) break;
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
    if (active) *active = (int)s->active.size() + pack_count(s) + pending;
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
    for (auto &pk : s->packs) {
        for (cudaEvent_t e : pk->done)
            if (e) cudaEventSynchronize(e);
        for (auto &a : pk->members) release(s, *a);
        for (auto &a : pk->joining) release(s, *a);
        if (pk->pair) cudaGraphExecDestroy(pk->pair);
        if (pk->budgets) cudaGraphExecDestroy(pk->budgets);
        for (auto &st : pk->st)
            if (st) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
            }
        for (cudaEvent_t e : {pk->fork, pk->join1, pk->join2, pk->done[0], pk->done[1]})
            if (e) cudaEventDestroy(e);
        s->arena.release(pk->off, pk->bytes);
    }
    s->packs.clear();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete s;
}

}  // extern "C"
