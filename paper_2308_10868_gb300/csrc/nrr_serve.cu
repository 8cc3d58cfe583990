// Serving: registrations submitted one by one and run with continuous
// batching on one GPU.
//
// The paper serves the operating room from a client/server setup whose
// server spreads each registration over remote clusters, with a work pool
// that tolerates failures (Sec. 4.1 "Ease-of-use", "Multi-Level Fault
// Tolerance").  On one GB300 a server is a scheduler thread in front of a
// set of CUDA streams ("slots"):
//   - nrr_submit queues a request (device-resident volumes, parameters) and
//     returns a ticket at once;
//   - the scheduler admits queued requests in arrival order whenever a slot
//     is free and the free device memory, less a reserve, covers the
//     request's scratch and result buffers; queued requests of the same
//     variant (dtype, block, radius) as the admitted one join it, up to 16:
//     each runs its own selection and box sums (the later ones on helper
//     streams of the slot, beside the first), and one match launch holds
//     all their jobs (each with its own volumes, sizes and tensor maps), so
//     a busy queue of small requests fills the GPU with one launch instead
//     of many partly filled ones; several admitted groups run at the same
//     time on different streams, so their kernels overlap on the device,
//     and a new group starts as soon as any earlier one finishes;
//   - each request runs the whole path (selection with a device-side count,
//     box sums, matching) on its slot stream, then a host callback stamps
//     its completion time and wakes the scheduler, which admits the next
//     queued request at once;
//   - request memory comes from a stream-ordered pool of the library's own
//     that keeps what it has mapped (a request of a size seen before maps
//     nothing), and admission counts the pool's mapped but unused bytes as
//     free;
//   - nrr_poll reports NRR_PENDING or the result (device pointers owned by
//     the library until nrr_release, the block count and the latencies).
// Failures are contained per request: an allocation or launch error marks
// that request failed (nrr_poll returns the status) and the server goes on.
// Host-side fault injection for tests: NRR_FAULT=alloc makes every
// admission's allocation fail; NRR_FAULT=alloc_once fails the next one only.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nrr_internal.h"

namespace nrr {
namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { QUEUED, RUNNING, DONE, FAILED };

struct Server;
struct Req {
    Server *srv;
    uint64_t ticket;
    nrr_request r;
    ReqState state = QUEUED;
    nrr_status status = NRR_OK;
    int slot = -1;
    void *mem = nullptr;
    size_t bytes = 0;
    int32_t cap = 0;
    int32_t *centers = nullptr, *d_n = nullptr, *disp = nullptr;
    double *ncc = nullptr;
    uint8_t *valid = nullptr;
    int32_t n_host = -1;  // count, read once at the first poll after completion
    std::atomic<int> finished{0};
    double t_submit = 0, t_admit = 0;
    std::atomic<double> t_done{0};
};

struct Server {
    int device = 0;
    int nslots = 0;
    size_t reserve = 0;
    int max_group = MATCH_MAX_JOBS;  // requests per match launch
    size_t max_queue = 65536;
    std::vector<cudaStream_t> slots;
    // per slot: streams on which a group's later requests run their
    // selection and box sums beside the first one's, and an event per
    // request that the group's match launch waits for
    static constexpr int HELPERS = 4;
    std::vector<cudaStream_t> helpers;   // [slot][HELPERS]
    std::vector<cudaEvent_t> ready;      // [slot][MATCH_MAX_JOBS]
    std::vector<std::vector<uint64_t>> slot_req;  // tickets running on each slot (empty = free)
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    cudaMemPool_t pool = nullptr;
    std::atomic<unsigned long long> events{0};  // submissions and completions
    bool stop = false;
    uint64_t next = 1;
    unsigned int *err = nullptr;
};

std::mutex g_server_mu;
Server *g_server = nullptr;

struct Layout {
    SelectPlan sp;
    size_t off_ws, off_box, off_centers, off_n, off_disp, off_ncc, off_valid, off_maps, total;
    int32_t cap;
};

Layout layout_of(const nrr_request &r)
{
    Layout L;
    L.sp = select_plan(r.dims, r.stride);
    long long cap = (long long)(0.5 + (double)L.sp.ng * r.frac) + 1;
    if (cap > L.sp.ng) cap = L.sp.ng;
    L.cap = (int32_t)(cap < 1 ? 1 : cap);
    size_t o = 0;
    L.off_ws = o;
    o += align_up(L.sp.bytes, 256);
    L.off_box = o;
    o += align_up(boxsum_bytes(r.dims, r.dtype), 256);
    L.off_centers = o;
    o += align_up((size_t)L.cap * 12, 256);
    L.off_n = o;
    o += 256;
    L.off_disp = o;
    o += align_up((size_t)L.cap * 12, 256);
    L.off_ncc = o;
    o += align_up((size_t)L.cap * 8, 256);
    L.off_valid = o;
    o += align_up((size_t)L.cap, 256);
    L.off_maps = o;  // the request's two tensor maps when it joins another's launch
    o += 256;
    L.total = o;
    return L;
}

bool fault(const char *what)
{
    static std::atomic<int> once_used{0};
    const char *f = getenv("NRR_FAULT");
    if (!f) return false;
    if (!strcmp(f, what)) return true;
    if (!strncmp(f, what, strlen(what)) && !strcmp(f + strlen(what), "_once")) return once_used.exchange(1) == 0;
    return false;
}

void CUDART_CB on_done(void *p)
{
    Req *q = (Req *)p;
    q->t_done.store(now_s());
    q->finished.store(1);
    // wake the scheduler to retire it and admit the next (no lock taken here:
    // the scheduler may hold its lock while it waits for a stream)
    q->srv->events.fetch_add(1);
    q->srv->cv.notify_all();
}

// The library's stream-ordered pool on `dev`: created once per process and
// kept (with every byte it has mapped, release threshold at the maximum), so
// that later requests and later servers reuse its memory.
cudaMemPool_t request_pool(int dev)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

// Bytes a request can still get: free device memory plus the pool's mapped
// bytes that no request uses.
size_t available_bytes(cudaMemPool_t pool)
{
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    uint64_t reserved = 0, used = 0;
    if (pool && cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
        fr += (size_t)(reserved - used);
    return fr;
}

// Prepare request q on slot k (server lock held): its memory, then its
// selection and box sums on the slot's stream; `follower` (it joins the
// launch of an earlier request of the same variant) also gets its tensor
// maps copied to its memory.  Fills its match job.  Returns 0 if memory is
// short right now (q stays queued), 1 if prepared, 2 if it failed (its
// status is set; nothing of it is left running).
int prepare(Server *S, Req *q, int k, cudaStream_t s, bool follower, MatchJob *job)
{
    const nrr_request &r = q->r;
    const Layout L = layout_of(r);
    const size_t fr = available_bytes(S->pool);
    if (fr < L.total + S->reserve) {
        bool busy = follower;
        for (auto &v : S->slot_req) busy |= !v.empty();
        if (busy) return 0;  // wait for running requests to free memory
        q->status = fail(NRR_E_NOMEM, "request needs %zu bytes, %zu free", L.total, fr);
        q->state = FAILED;  // would never fit
        return 2;
    }
    q->slot = k;
    q->t_admit = now_s();
    q->state = RUNNING;
    cudaError_t e = fault("alloc") ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync(&q->mem, L.total, S->pool, s);
    if (e != cudaSuccess) {
        q->mem = nullptr;
        q->status = cuda_fail(e, "request allocation");
        q->state = FAILED;
        return 2;
    }
    unsigned char *m = (unsigned char *)q->mem;
    q->bytes = L.total;
    q->cap = L.cap;
    q->centers = (int32_t *)(m + L.off_centers);
    q->d_n = (int32_t *)(m + L.off_n);
    q->disp = (int32_t *)(m + L.off_disp);
    q->ncc = (double *)(m + L.off_ncc);
    q->valid = (uint8_t *)(m + L.off_valid);
    nrr_status st = enqueue_select(r.d_select, r.d_mask, r.dims, r.block, r.stride, r.frac,
                                   q->centers, q->cap, q->d_n, m + L.off_ws, L.sp, s);
    if (st == NRR_OK) st = launch_boxsums(r.d_intraop, r.dtype, r.dims, r.block, m + L.off_box, s);
    *job = MatchJob{q->centers, q->d_n, q->cap, q->disp, q->ncc, q->valid};
    job->preop = r.d_preop;
    job->intraop = r.d_intraop;
    job->s1 = m + L.off_box;
    job->s2 = m + L.off_box + boxsum_s2_offset(r.dims, r.dtype);
    job->nx = r.dims.nx;
    job->ny = r.dims.ny;
    job->nz = r.dims.nz;
    if (st == NRR_OK && follower) {
        CUtensorMap maps[2];
        int wb[3], tb[3];
        match_boxes(r.dtype, r.block, r.block, r.block, r.radius, wb, tb);
        st = encode_volume_map(&maps[0], r.d_intraop, r.dtype, r.dims, wb[0], wb[1], wb[2]);
        if (st == NRR_OK) st = encode_volume_map(&maps[1], r.d_preop, r.dtype, r.dims, tb[0], tb[1], tb[2]);
        if (st == NRR_OK && cudaMemcpyAsync(m + L.off_maps, maps, sizeof maps, cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = fail(NRR_E_CUDA, "tensor map copy");
        job->mapJ = reinterpret_cast<const CUtensorMap *>(m + L.off_maps);
        job->mapI = job->mapJ + 1;
    }
    if (st != NRR_OK) {
        q->status = st;
        q->state = FAILED;
        cudaStreamSynchronize(s);  // nothing of this request may still run
        cudaFreeAsync(q->mem, s);
        q->mem = nullptr;
        return 2;
    }
    return 1;
}

bool same_variant(const nrr_request &a, const nrr_request &b)
{
    return a.dtype == b.dtype && a.block == b.block && a.radius[0] == b.radius[0] && a.radius[1] == b.radius[1] &&
           a.radius[2] == b.radius[2];
}

// Admit the request at the queue's front on free slot k, with queued
// requests of the same variant (dtype, block, radius) behind it, up to
// MATCH_MAX_JOBS in all: each runs its own selection and box sums on the
// slot's stream, then one match launch holds all their jobs (server lock
// held).  Returns false if the front request must wait for memory.
bool admit_group(Server *S, int k)
{
    const uint64_t t0 = S->queue.front();
    Req *q0 = S->reqs[t0];
    MatchJob jobs[MATCH_MAX_JOBS];
    std::vector<Req *> group;
    cudaStream_t s = S->slots[k];
    const int r0 = prepare(S, q0, k, s, false, &jobs[0]);
    if (r0 == 0) return false;
    S->queue.pop_front();
    if (r0 == 2) return true;
    group.push_back(q0);
    // followers: the next same-variant requests among the first queued ones
    constexpr size_t SCAN = 64;
    for (size_t pos = 0; pos < S->queue.size() && pos < SCAN && group.size() < (size_t)S->max_group;) {
        auto it = S->reqs.find(S->queue[pos]);
        if (it == S->reqs.end()) {  // released while queued
            S->queue.erase(S->queue.begin() + pos);
            continue;
        }
        Req *q = it->second;
        if (!same_variant(q->r, q0->r)) {
            ++pos;
            continue;
        }
        // a follower's selection and box sums run on a helper stream beside
        // the others'; the match launch waits for its event
        const size_t g = group.size();
        cudaStream_t hs = S->helpers[(size_t)k * Server::HELPERS + (g - 1) % Server::HELPERS];
        cudaEvent_t ev = S->ready[(size_t)k * MATCH_MAX_JOBS + g];
        if (cudaEventRecord(ev, s) != cudaSuccess || cudaStreamWaitEvent(hs, ev, 0) != cudaSuccess) break;
        const int r = prepare(S, q, k, hs, true, &jobs[g]);
        if (r == 0) break;
        S->queue.erase(S->queue.begin() + pos);
        if (r == 1) {
            if (cudaEventRecord(ev, hs) != cudaSuccess || cudaStreamWaitEvent(s, ev, 0) != cudaSuccess) {
                cudaStreamSynchronize(hs);  // nothing of it may still run
                q->status = fail(NRR_E_CUDA, "event");
                q->state = FAILED;
                cudaFreeAsync(q->mem, s);
                q->mem = nullptr;
                continue;
            }
            group.push_back(q);
        }
    }
    const nrr_request &r = q0->r;
    MatchLaunch a{};  // on the slot's stream, after every member's event
    a.preop = r.d_preop;
    a.intraop = r.d_intraop;
    a.s1 = jobs[0].s1;
    a.s2 = jobs[0].s2;
    a.dtype = r.dtype;
    a.dims = r.dims;
    a.block = r.block;
    for (int i = 0; i < 3; ++i) a.radius[i] = r.radius[i];
    a.n_jobs = (int)group.size();
    for (size_t g = 0; g < group.size(); ++g) a.jobs[g] = jobs[g];
    apply_tuning(a, r.dtype, r.block, r.radius);
    a.err = S->err;
    nrr_status st = launch_match(a, s);
    for (size_t g = 0; g < group.size() && st == NRR_OK; ++g)
        if (cudaLaunchHostFunc(s, on_done, group[g]) != cudaSuccess) st = fail(NRR_E_CUDA, "host callback");
    if (st != NRR_OK) {
        cudaStreamSynchronize(s);  // nothing of these requests may still run
        for (Req *q : group) {
            q->status = st;
            q->state = FAILED;
            cudaFreeAsync(q->mem, s);
            q->mem = nullptr;
        }
        return true;
    }
    for (Req *q : group) S->slot_req[k].push_back(q->ticket);
    return true;
}

void worker_main(Server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        const unsigned long long seen = S->events.load();
        // retire finished requests; a slot is free once all of its are
        for (int k = 0; k < S->nslots; ++k) {
            auto &v = S->slot_req[k];
            for (size_t i = 0; i < v.size();) {
                auto it = S->reqs.find(v[i]);
                if (it != S->reqs.end() && !it->second->finished.load()) {
                    ++i;
                    continue;
                }
                if (it != S->reqs.end()) it->second->state = DONE;
                v.erase(v.begin() + i);
                S->cv.notify_all();
            }
        }
        // admit in arrival order (with same-variant followers) while slots
        // and memory allow
        bool progressed = false;
        while (!S->queue.empty()) {
            int k = -1;
            for (int i = 0; i < S->nslots; ++i)
                if (S->slot_req[i].empty()) {
                    k = i;
                    break;
                }
            if (k < 0) break;
            if (S->reqs.find(S->queue.front()) == S->reqs.end()) {  // released while queued
                S->queue.pop_front();
                continue;
            }
            if (!admit_group(S, k)) break;
            progressed = true;
        }
        if (progressed) S->cv.notify_all();
        // woken by a submission or a completion (the short timeout covers a
        // wake-up sent between the check and the wait)
        S->cv.wait_for(lk, std::chrono::microseconds(200), [&] { return S->stop || S->events.load() != seen; });
    }
}

}  // namespace
}  // namespace nrr

using namespace nrr;

extern "C" {

nrr_status nrr_server_start(int32_t slots, size_t reserve_bytes)
{
    return nrr_server_start_ex(slots, reserve_bytes, MATCH_MAX_JOBS);
}

nrr_status nrr_server_start_ex(int32_t slots, size_t reserve_bytes, int32_t max_group)
{
    clear_error();
    if (slots < 1 || slots > 64) return fail(NRR_E_INVALID, "slots must be 1..64");
    if (max_group < 1 || max_group > MATCH_MAX_JOBS) return fail(NRR_E_INVALID, "max_group must be 1..%d", MATCH_MAX_JOBS);
    std::lock_guard<std::mutex> g(g_server_mu);
    if (g_server) return fail(NRR_E_INVALID, "server already running");
    Server *S = new Server();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return fail(NRR_E_CUDA, "cudaGetDevice");
    }
    nrr_status st = device_error_word(&S->err);
    if (st != NRR_OK) {
        delete S;
        return st;
    }
    S->pool = request_pool(S->device);
    if (!S->pool) {
        delete S;
        return fail(NRR_E_CUDA, "memory pool creation");
    }
    S->nslots = slots;
    S->reserve = reserve_bytes;
    S->max_group = max_group;
    S->slots.resize(slots);
    S->slot_req.assign(slots, std::vector<uint64_t>());
    S->helpers.assign((size_t)slots * Server::HELPERS, nullptr);
    S->ready.assign((size_t)slots * MATCH_MAX_JOBS, nullptr);
    bool ok = true;
    for (int k = 0; k < slots && ok; ++k) ok = cudaStreamCreateWithFlags(&S->slots[k], cudaStreamNonBlocking) == cudaSuccess;
    for (auto &h : S->helpers)
        if (ok) ok = cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &e : S->ready)
        if (ok) ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (auto &st : S->slots)
            if (st) cudaStreamDestroy(st);
        for (auto &h : S->helpers)
            if (h) cudaStreamDestroy(h);
        for (auto &e : S->ready)
            if (e) cudaEventDestroy(e);
        delete S;
        return fail(NRR_E_CUDA, "stream or event creation");
    }
    S->worker = std::thread(worker_main, S);
    g_server = S;
    return NRR_OK;
}

nrr_status nrr_server_stop(void)
{
    clear_error();
    Server *S;
    {
        std::lock_guard<std::mutex> g(g_server_mu);
        S = g_server;
        g_server = nullptr;
    }
    if (!S) return NRR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    S->worker.join();
    for (auto &st : S->slots) cudaStreamSynchronize(st);
    for (auto &h : S->helpers) cudaStreamSynchronize(h);
    for (auto &kv : S->reqs) {
        Req *q = kv.second;
        if (q->mem) cudaFree(q->mem);
        delete q;
    }
    for (auto &st : S->slots) cudaStreamDestroy(st);
    for (auto &h : S->helpers) cudaStreamDestroy(h);
    for (auto &e : S->ready) cudaEventDestroy(e);
    delete S;
    return NRR_OK;
}

nrr_status nrr_submit(const nrr_request *req, uint64_t *ticket)
{
    clear_error();
    if (!req || !ticket) return fail(NRR_E_INVALID, "NULL request or ticket");
    if (req->dtype != NRR_U16 && req->dtype != NRR_F32) return fail(NRR_E_INVALID, "unknown dtype");
    nrr_status st = check_select_args(req->dims, req->block, req->stride, req->frac);
    if (st != NRR_OK) return st;
    st = check_dims(req->dims, req->dtype, req->block);
    if (st != NRR_OK) return st;
    for (int i = 0; i < 3; ++i)
        if (req->radius[i] < 0 || req->radius[i] > MATCH_MAX_R) return fail(NRR_E_INVALID, "radius outside 0..%d", MATCH_MAX_R);
    if (!req->d_preop || !req->d_intraop || !req->d_mask || !req->d_select)
        return fail(NRR_E_INVALID, "NULL volume, mask or selection volume");
    std::lock_guard<std::mutex> g(g_server_mu);
    Server *S = g_server;
    if (!S) return fail(NRR_E_INVALID, "no server running (nrr_server_start)");
    Req *q = new Req();
    q->srv = S;
    q->r = *req;
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.size() >= S->max_queue) {
            delete q;
            return fail(NRR_E_CAPACITY, "request queue full");
        }
        q->ticket = S->next++;
        S->reqs[q->ticket] = q;
        S->queue.push_back(q->ticket);
        *ticket = q->ticket;
        S->events.fetch_add(1);
    }
    S->cv.notify_all();
    return NRR_OK;
}

nrr_status nrr_poll(uint64_t ticket, nrr_result *out)
{
    clear_error();
    std::lock_guard<std::mutex> g(g_server_mu);
    Server *S = g_server;
    if (!S) return fail(NRR_E_INVALID, "no server running");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(NRR_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second;
    if (q->state == RUNNING && q->finished.load()) q->state = DONE;
    if (q->state == FAILED) return fail(q->status, "request %llu failed", (unsigned long long)ticket);
    if (q->state != DONE) return NRR_PENDING;
    if (q->n_host < 0) {
        int32_t n = 0;
        cudaError_t e = cudaMemcpy(&n, q->d_n, sizeof(n), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "reading the block count");
        q->n_host = n;
    }
    if (out) {
        out->n_blocks = q->n_host;
        out->centers = q->centers;
        out->disp = q->disp;
        out->ncc = q->ncc;
        out->valid = q->valid;
        out->queued_s = q->t_admit - q->t_submit;
        out->latency_s = q->t_done.load() - q->t_submit;
    }
    return NRR_OK;
}

nrr_status nrr_release(uint64_t ticket)
{
    clear_error();
    std::lock_guard<std::mutex> g(g_server_mu);
    Server *S = g_server;
    if (!S) return fail(NRR_E_INVALID, "no server running");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(NRR_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second;
    if (q->state == RUNNING && !q->finished.load())
        return fail(NRR_E_INVALID, "request %llu still running", (unsigned long long)ticket);
    if (q->mem) cudaFreeAsync(q->mem, S->slots[q->slot >= 0 ? q->slot : 0]);
    S->reqs.erase(it);  // a queued request is simply dropped from the queue later
    delete q;
    return NRR_OK;
}

}  // extern "C"
