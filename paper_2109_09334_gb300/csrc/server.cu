// server.cu -- sfft_submit / sfft_poll / sfft_wait: several pairs in flight.
//
// A server holds `depth` slots, each a full plan (its own spectra, lag
// tables, M, rhs and solve workspace) plus staging buffers for requests in
// host memory, and three streams:
//   sc  copies of host requests' inputs to the slot's staging buffers;
//   sb  plan set-up; the build of each pair (row/column FFTs, gather, lag
//       sums, assembly) runs on its slot's own stream, so that builds of
//       different pairs overlap;
//   ss  (highest priority) the solves and the subtractions;
//   so  the copies of the results back to host requests, so that they
//       overlap the next group's solve and subtractions.
// Request s uses slot s mod depth.  Its build is enqueued at once; the
// requests are grouped `batch` at a time (batch <= depth), and when a group
// is complete (or on sfft_flush, or when a caller waits for one of its
// requests) one cooperative launch solves all of its systems together and
// the group's subtractions follow.  The solve is a latency-bound chain of
// grid-wide steps, so solving several systems in one launch costs little
// more than solving one.  Events order the streams:
//   built[i]: the slot's build stream -> ss (M, rhs of the slot ready);
//   done[i]:  ss or so -> sb, sc (the slot's previous pair is finished, so
//             its workspace and staging buffers may be overwritten);
//   subtracted[i]: ss -> so (a host request's results are ready to copy).
// A slot is reused only by a request of a later group, whose predecessor's
// group is complete and therefore flushed, so `done` is always recorded
// before anything waits on it.  Every pair runs the kernels of
// sfft_run_pair on its own slot, so its results are the same.
//
// Completion: every request records an event after its last operation (on
// ss, or on so for a host request).  The watermark (all requests below it
// are complete) advances over these events in submission order, so requests
// complete in submission order; it answers sfft_poll.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>

#include "internal.h"

namespace sfft {
namespace {

constexpr int kMaxDepth = 8;
constexpr int kRing = 64;  // completion events kept; submit waits beyond this
constexpr int kMaxPoolLanes = 64;  // configurations a pool holds at once

struct Slot {
    Plan *plan = nullptr;
    void *ref = nullptr, *sci = nullptr, *diff = nullptr;  // staging for host requests
    uint8_t *mask = nullptr;
    cudaEvent_t built = nullptr, done = nullptr, copied = nullptr, subtracted = nullptr;
    // the request built in this slot and not yet flushed
    bool host = false;
    const void *in_ref = nullptr, *in_sci = nullptr;  // device images the build read
    const uint8_t *in_mask = nullptr;
    double *x = nullptr;
    sfft_solve_info *info = nullptr;
    void *diff_out = nullptr;  // device difference image
    sfft_request req;          // the caller's request (host destinations)
};

}  // namespace

struct Server {
    sfft_config cfg;
    int depth = 0, batch = 1;
    size_t img_bytes = 0, pixels = 0;
    Slot slots[kMaxDepth];
    cudaStream_t sc = nullptr, sb = nullptr, ss = nullptr, so = nullptr;
    // one build stream per slot, so that the builds of different pairs overlap
    // on the GPU (their small kernels leave most SMs idle)
    cudaStream_t sbs[kMaxDepth] = {};
    cudaEvent_t input_ready = nullptr;
    cudaEvent_t ring[kRing] = {};
    uint64_t next_seq = 0;   // sequence number of the next request
    uint64_t flushed = 0;    // every request below it has its solve and subtraction enqueued
    uint64_t watermark = 0;  // every request below it has completed
    std::mutex mu;
    int refs = 0;  // callers waiting on it through a pool (guarded by the pool's lock)
    // Sticky failure: once a completion query reports a CUDA error, every
    // later submit, poll and wait returns it (the requests in flight can no
    // longer be known to complete).
    int err = SFFT_OK;
    // testing hook (sfft_server_debug_fail_queries): completion queries
    // report a CUDA error without asking the device
    bool fail_queries = false;
    // eager flushing (sfft_server_set_eager): an incomplete batch is solved
    // at once when everything flushed before it has completed
    bool eager = false;
};

namespace {

void server_free(Server *v) {
    for (int i = 0; i < kMaxDepth; ++i) {
        Slot &s = v->slots[i];
        if (s.plan) plan_free(s.plan);
        void *bufs[] = {s.ref, s.sci, s.diff, s.mask};
        for (void *b : bufs)
            if (b) cudaFree(b);
        cudaEvent_t evs[] = {s.built, s.done, s.copied, s.subtracted};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : v->ring)
        if (e) cudaEventDestroy(e);
    if (v->input_ready) cudaEventDestroy(v->input_ready);
    cudaStream_t sts[] = {v->sc, v->sb, v->ss, v->so};
    for (cudaStream_t s : sts)
        if (s) cudaStreamDestroy(s);
    for (cudaStream_t s : v->sbs)
        if (s) cudaStreamDestroy(s);
    delete v;
}

// Completion query of one request's event (through the testing hook).
cudaError_t query_done(Server *v, cudaEvent_t ev, bool block) {
    if (v->fail_queries) return cudaErrorLaunchFailure;
    return block ? cudaEventSynchronize(ev) : cudaEventQuery(ev);
}

// Advance the watermark over completed requests (caller holds mu).  Only
// flushed requests have their completion event recorded.  Returns SFFT_OK,
// or SFFT_ERR_CUDA (sticky) if a query reported an error.
int advance(Server *v) {
    if (v->err != SFFT_OK) return v->err;
    while (v->watermark < v->flushed) {
        const cudaError_t e = query_done(v, v->ring[v->watermark % kRing], false);
        if (e == cudaErrorNotReady) return SFFT_OK;
        if (e != cudaSuccess) {
            if (!v->fail_queries) cudaGetLastError();
            v->err = SFFT_ERR_CUDA;
            return v->err;
        }
        ++v->watermark;
    }
    return SFFT_OK;
}

int create_server(const sfft_config *cfg, int depth, int batch, Server **out) {
    Server *v = new (std::nothrow) Server();
    if (!v) return SFFT_ERR_OOM;
    v->cfg = *cfg;
    v->depth = depth;
    v->batch = batch;
    v->pixels = (size_t)cfg->n0 * cfg->n1;
    v->img_bytes = v->pixels * (cfg->dtype == SFFT_F64 ? sizeof(double) : sizeof(float));
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&v->sc, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&v->sb, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&v->ss, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&v->so, cudaStreamNonBlocking, lo);
    for (int i = 0; i < depth && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithPriority(&v->sbs[i], cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->input_ready, cudaEventDisableTiming);
    for (int k = 0; k < kRing && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&v->ring[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        server_free(v);
        return status_of(e);
    }
    for (int i = 0; i < depth; ++i) {
        Slot &s = v->slots[i];
        const int rc = plan_new(cfg, v->sb, &s.plan);
        if (rc != SFFT_OK) {
            s.plan = nullptr;
            server_free(v);
            return rc;
        }
        // four or more systems per solve launch: the 64-wide panels (half the
        // barriers and trailing passes, a longer chain per step; measured at
        // n = 1735: 8 systems 3.26 -> 2.77 ms, 4 even, 2 slower)
        if (batch >= 4) s.plan->solve_panel = 64;
        e = cudaMalloc(&s.ref, v->img_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s.sci, v->img_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s.diff, v->img_bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.mask, v->pixels);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.built, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.subtracted, cudaEventDisableTiming);
        // a fresh slot is free: let the first waits on `done` pass at once
        if (e == cudaSuccess) e = cudaEventRecord(s.done, v->ss);
        if (e != cudaSuccess) {
            cudaGetLastError();
            server_free(v);
            return status_of(e);
        }
    }
    e = cudaStreamSynchronize(v->sb);  // plan tables are ready
    if (e != cudaSuccess) {
        server_free(v);
        return status_of(e);
    }
    *out = v;
    return SFFT_OK;
}

// Enqueue the solve (one batched launch) and the subtraction of every
// request built but not yet flushed (caller holds mu).
int flush(Server *v) {
    const uint64_t first = v->flushed, end = v->next_seq;
    const int cnt = (int)(end - first);
    if (cnt == 0) return SFFT_OK;
    Plan *plans[kMaxDepth] = {};
    const double *M[kMaxDepth] = {}, *rhs[kMaxDepth] = {};
    double *x[kMaxDepth] = {};
    sfft_solve_info *info[kMaxDepth] = {};
    for (int k = 0; k < cnt; ++k) {
        Slot &s = v->slots[(first + k) % v->depth];
        plans[k] = s.plan;
        M[k] = s.plan->M_own;
        rhs[k] = s.plan->rhs_own;
        x[k] = s.x;
        info[k] = s.info;
    }
    // the group's builds ran on their slots' streams: wait for each
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < cnt && e == cudaSuccess; ++k)
        e = cudaStreamWaitEvent(v->ss, v->slots[(first + k) % v->depth].built, 0);
    if (e == cudaSuccess) e = solve_batch(plans, cnt, M, rhs, x, info, v->ss);
    for (int k = 0; k < cnt && e == cudaSuccess; ++k) {
        const uint64_t seq = first + k;
        Slot &s = v->slots[seq % v->depth];
        Plan *p = s.plan;
        if (s.in_mask) e = row_transform(p, s.in_ref, s.in_sci, nullptr, false, v->ss);
        if (e == cudaSuccess) e = subtract_from_rows(p, s.x, s.diff_out, v->ss);
        cudaStream_t last = v->ss;  // the stream of this request's last operation
        if (s.host) {  // results back to the host on so, overlapping the next group's work on ss
            const sfft_request &r = s.req;
            last = v->so;
            if (e == cudaSuccess) e = cudaEventRecord(s.subtracted, v->ss);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(v->so, s.subtracted, 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r.diff, s.diff, v->img_bytes, cudaMemcpyDeviceToHost, v->so);
            if (e == cudaSuccess && r.x)
                e = cudaMemcpyAsync(r.x, p->x_own, (size_t)p->n * sizeof(double), cudaMemcpyDeviceToHost, v->so);
            if (e == cudaSuccess && r.info)
                e = cudaMemcpyAsync(r.info, p->info_own, sizeof(sfft_solve_info), cudaMemcpyDeviceToHost, v->so);
        }
        if (e == cudaSuccess) e = cudaEventRecord(s.done, last);
        if (e == cudaSuccess) e = cudaEventRecord(v->ring[seq % kRing], last);
    }
    if (e != cudaSuccess) return status_of(e);
    v->flushed = end;
    return SFFT_OK;
}

int eager_flush(Server *v);

int submit(Server *v, const sfft_request *r, uint64_t *seq_out) {
    const bool host = r->memory == SFFT_REQ_HOST;
    if (v->err != SFFT_OK) return v->err;
    // keep at most kRing requests in flight: the ring slot must be free
    while (v->next_seq - v->watermark >= (uint64_t)kRing) {
        if (v->watermark >= v->flushed) {
            const int rc = flush(v);
            if (rc != SFFT_OK) return rc;
        }
        const cudaError_t e = query_done(v, v->ring[v->watermark % kRing], true);
        if (e != cudaSuccess) {
            v->err = SFFT_ERR_CUDA;
            return v->err;
        }
        const int rc = advance(v);
        if (rc != SFFT_OK) return rc;
    }
    const uint64_t seq = v->next_seq;
    // the request that used this slot before belongs to an earlier, full,
    // hence flushed batch (depth >= batch), so its `done` event is recorded
    Slot &s = v->slots[seq % v->depth];
    Plan *p = s.plan;
    const void *ref = r->ref, *sci = r->sci;
    const uint8_t *mask = r->mask;
    cudaError_t e = cudaSuccess;
    if (host) {
        e = cudaStreamWaitEvent(v->sc, s.done, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.ref, r->ref, v->img_bytes, cudaMemcpyHostToDevice, v->sc);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.sci, r->sci, v->img_bytes, cudaMemcpyHostToDevice, v->sc);
        if (e == cudaSuccess && r->mask) e = cudaMemcpyAsync(s.mask, r->mask, v->pixels, cudaMemcpyHostToDevice, v->sc);
        if (e == cudaSuccess) e = cudaEventRecord(s.copied, v->sc);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(v->sbs[seq % v->depth], s.copied, 0);
        ref = s.ref;
        sci = s.sci;
        mask = r->mask ? s.mask : nullptr;
    } else {
        // the inputs are ready in the caller's stream order
        e = cudaEventRecord(v->input_ready, (cudaStream_t)r->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(v->sbs[seq % v->depth], v->input_ready, 0);
    }
    // the slot's previous pair has finished with its workspace
    cudaStream_t sb = v->sbs[seq % v->depth];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sb, s.done, 0);
    if (e == cudaSuccess) e = build_system(p, ref, sci, mask, p->M_own, p->rhs_own, sb);
    if (e == cudaSuccess) e = cudaEventRecord(s.built, sb);
    if (e != cudaSuccess) return status_of(e);
    s.host = host;
    s.in_ref = ref;
    s.in_sci = sci;
    s.in_mask = mask;
    s.x = (!host && r->x) ? r->x : p->x_own;
    s.info = (!host && r->info) ? r->info : p->info_own;
    s.diff_out = host ? s.diff : r->diff;
    s.req = *r;
    v->next_seq = seq + 1;
    *seq_out = seq;
    if (v->next_seq - v->flushed >= (uint64_t)v->batch) return flush(v);
    return eager_flush(v);
}

// Continuous batching: with eager set, an incomplete batch is flushed as
// soon as every request flushed before it has completed, so a request never
// waits for batch partners while its server has nothing else in flight; when
// the server is busy, the requests that arrive meanwhile gather into one
// batch (caller holds mu).
int eager_flush(Server *v) {
    if (!v->eager || v->next_seq == v->flushed) return SFFT_OK;
    const int rc = advance(v);
    if (rc != SFFT_OK) return rc;
    return v->watermark == v->flushed ? flush(v) : SFFT_OK;
}

}  // namespace

// ---- pool: servers of several configurations under one byte budget --------

namespace {

struct Lane {
    uint64_t id = 0;
    sfft_config cfg{};
    Server *srv = nullptr;
    uint64_t bytes = 0;
    uint64_t last_use = 0;
};

bool same_config(const sfft_config &a, const sfft_config &b) { return memcmp(&a, &b, sizeof(sfft_config)) == 0; }

// every request of the lane has completed (caller holds the pool's lock)
bool lane_idle(Lane &l) {
    std::lock_guard<std::mutex> lock(l.srv->mu);
    // a lane whose completion query failed is never idle: its memory may
    // still be in use on the device
    if (advance(l.srv) != SFFT_OK) return false;
    return l.srv->flushed == l.srv->next_seq && l.srv->watermark == l.srv->next_seq;
}

uint64_t server_bytes(const Server *v) {
    uint64_t b = 0;
    for (int i = 0; i < v->depth; ++i) b += v->slots[i].plan->ws_bytes + 3 * v->img_bytes + v->pixels;
    return b;
}

}  // namespace

struct Pool {
    uint64_t budget = 0, used = 0, next_id = 1, clock = 0;
    int depth = 1, batch = 1;
    bool eager = false;  // lanes flush eagerly (sfft_pool_set_eager)
    Lane lanes[kMaxPoolLanes];
    int nlanes = 0;
    std::mutex mu;
};

namespace {

Lane *find_lane(Pool *pl, uint64_t id) {
    for (int k = 0; k < pl->nlanes; ++k)
        if (pl->lanes[k].id == id) return &pl->lanes[k];
    return nullptr;
}

void drop_lane(Pool *pl, int k) {
    Lane &l = pl->lanes[k];
    sfft_server_destroy((sfft_server_t)l.srv);
    pl->used -= l.bytes;
    pl->lanes[k] = pl->lanes[pl->nlanes - 1];
    --pl->nlanes;
}

// release idle lanes, least recently used first, until `need` more bytes fit
// (or a lane slot is needed); returns whether they fit
bool make_room(Pool *pl, uint64_t need, bool want_slot, uint64_t keep_id) {
    for (;;) {
        const bool fits = pl->used + need <= pl->budget && (!want_slot || pl->nlanes < kMaxPoolLanes);
        if (fits) return true;
        int victim = -1;
        for (int k = 0; k < pl->nlanes; ++k) {
            Lane &l = pl->lanes[k];
            if (l.id == keep_id || l.srv->refs > 0 || !lane_idle(l)) continue;
            if (victim < 0 || l.last_use < pl->lanes[victim].last_use) victim = k;
        }
        if (victim < 0) return false;
        drop_lane(pl, victim);
    }
}

}  // namespace

}  // namespace sfft

using namespace sfft;

extern "C" {

int sfft_server_create(const sfft_config *cfg, int32_t depth, int32_t batch, sfft_server_t *out) {
    if (!out) return SFFT_ERR_INVALID;
    *out = nullptr;
    if (!cfg || depth < 1 || depth > kMaxDepth || batch < 1 || batch > depth) return SFFT_ERR_INVALID;
    const int v = plan_validate(cfg);
    if (v) return v;
    Server *s = nullptr;
    const int rc = create_server(cfg, depth, batch, &s);
    if (rc == SFFT_OK) *out = (sfft_server_t)s;
    return rc;
}

int sfft_server_set_eager(sfft_server_t server, int32_t enable) {
    if (!server) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    std::lock_guard<std::mutex> lock(v->mu);
    v->eager = enable != 0;
    return eager_flush(v);
}

int sfft_server_debug_fail_queries(sfft_server_t server, int32_t enable) {
    if (!server) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    std::lock_guard<std::mutex> lock(v->mu);
    v->fail_queries = enable != 0;
    return SFFT_OK;
}

int sfft_server_destroy(sfft_server_t server) {
    if (!server) return SFFT_OK;
    Server *v = (Server *)server;
    {
        std::lock_guard<std::mutex> lock(v->mu);
        flush(v);
    }
    cudaStreamSynchronize(v->sc);
    cudaStreamSynchronize(v->sb);
    for (int i = 0; i < v->depth; ++i) cudaStreamSynchronize(v->sbs[i]);
    cudaStreamSynchronize(v->ss);
    cudaStreamSynchronize(v->so);
    server_free(v);
    return SFFT_OK;
}

int sfft_submit(sfft_server_t server, const sfft_request *req, sfft_ticket *ticket) {
    if (!server || !req || !ticket) return SFFT_ERR_INVALID;
    if (!req->ref || !req->sci || !req->diff) return SFFT_ERR_INVALID;
    if (req->memory != SFFT_REQ_DEVICE && req->memory != SFFT_REQ_HOST) return SFFT_ERR_INVALID;
    if (req->diff == req->ref || req->diff == req->sci) return SFFT_ERR_INVALID;
    if (req->memory == SFFT_REQ_DEVICE && !images_aligned(req->ref, req->sci, req->mask)) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    std::lock_guard<std::mutex> lock(v->mu);
    uint64_t seq = 0;
    const int rc = submit(v, req, &seq);
    if (rc == SFFT_OK) ticket->seq = seq;
    return rc;
}

int sfft_poll(sfft_server_t server, const sfft_ticket *ticket) {
    if (!server || !ticket) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    std::lock_guard<std::mutex> lock(v->mu);
    if (ticket->seq >= v->next_seq) return SFFT_ERR_INVALID;
    if (ticket->seq >= v->flushed) {
        const int rc = flush(v);
        if (rc != SFFT_OK) return rc;
    }
    const int rc = advance(v);
    if (rc != SFFT_OK) return rc;
    return ticket->seq < v->watermark ? SFFT_OK : SFFT_ERR_BUSY;
}

int sfft_wait(sfft_server_t server, const sfft_ticket *ticket, int64_t timeout_us) {
    if (!server || !ticket) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(v->mu);
            if (ticket->seq >= v->next_seq) return SFFT_ERR_INVALID;
            if (ticket->seq >= v->flushed) {
                const int rc = flush(v);
                if (rc != SFFT_OK) return rc;
            }
            const int rc = advance(v);
            if (rc != SFFT_OK) return rc;
            if (ticket->seq < v->watermark) return SFFT_OK;
        }
        if (timeout_us >= 0) {
            const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (us >= timeout_us) return SFFT_ERR_TIMEOUT;
        }
        std::this_thread::yield();
    }
}

int sfft_stream_wait_ticket(sfft_server_t server, const sfft_ticket *ticket, sfft_stream_t stream) {
    if (!server || !ticket) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    std::lock_guard<std::mutex> lock(v->mu);
    if (ticket->seq >= v->next_seq) return SFFT_ERR_INVALID;
    if (ticket->seq >= v->flushed) {
        const int rc = flush(v);
        if (rc != SFFT_OK) return rc;
    }
    // a ring event is reused only after the host has seen it complete
    if (ticket->seq + kRing < v->next_seq) return SFFT_OK;
    return status_of(cudaStreamWaitEvent((cudaStream_t)stream, v->ring[ticket->seq % kRing], 0));
}

int sfft_flush(sfft_server_t server) {
    if (!server) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    std::lock_guard<std::mutex> lock(v->mu);
    return flush(v);
}

int sfft_server_launch_count(sfft_server_t server, uint64_t *count) {
    if (!server || !count) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    std::lock_guard<std::mutex> lock(v->mu);
    uint64_t c = 0;
    for (int i = 0; i < v->depth; ++i) c += v->slots[i].plan->launches;
    *count = c;
    return SFFT_OK;
}

int sfft_server_workspace_bytes(sfft_server_t server, uint64_t *bytes) {
    if (!server || !bytes) return SFFT_ERR_INVALID;
    Server *v = (Server *)server;
    uint64_t b = 0;
    for (int i = 0; i < v->depth; ++i) b += v->slots[i].plan->ws_bytes + 3 * v->img_bytes + v->pixels;
    *bytes = b;
    return SFFT_OK;
}


int sfft_pool_create(uint64_t budget_bytes, int32_t depth, int32_t batch, sfft_pool_t *out) {
    if (!out) return SFFT_ERR_INVALID;
    *out = nullptr;
    if (budget_bytes == 0 || depth < 1 || depth > kMaxDepth || batch < 1 || batch > depth) return SFFT_ERR_INVALID;
    Pool *pl = new (std::nothrow) Pool();
    if (!pl) return SFFT_ERR_OOM;
    pl->budget = budget_bytes;
    pl->depth = depth;
    pl->batch = batch;
    *out = (sfft_pool_t)pl;
    return SFFT_OK;
}

int sfft_pool_destroy(sfft_pool_t pool) {
    if (!pool) return SFFT_OK;
    Pool *pl = (Pool *)pool;
    {
        std::lock_guard<std::mutex> lock(pl->mu);
        while (pl->nlanes > 0) drop_lane(pl, pl->nlanes - 1);
    }
    delete pl;
    return SFFT_OK;
}

int sfft_pool_submit(sfft_pool_t pool, const sfft_config *cfg, const sfft_request *req, sfft_pool_ticket *ticket) {
    if (!pool || !cfg || !req || !ticket) return SFFT_ERR_INVALID;
    if (!req->ref || !req->sci || !req->diff) return SFFT_ERR_INVALID;
    if (req->memory != SFFT_REQ_DEVICE && req->memory != SFFT_REQ_HOST) return SFFT_ERR_INVALID;
    if (req->memory == SFFT_REQ_DEVICE && !images_aligned(req->ref, req->sci, req->mask)) return SFFT_ERR_INVALID;
    const int v = plan_validate(cfg);
    if (v) return v;
    Pool *pl = (Pool *)pool;
    std::lock_guard<std::mutex> lock(pl->mu);
    Lane *lane = nullptr;
    for (int k = 0; k < pl->nlanes; ++k)
        if (same_config(pl->lanes[k].cfg, *cfg)) lane = &pl->lanes[k];
    if (!lane) {
        // admission: the new lane's workspace must fit the budget
        if (!make_room(pl, 0, true, 0)) return SFFT_ERR_BUSY;
        Server *srv = nullptr;
        int rc = create_server(cfg, pl->depth, pl->batch, &srv);
        if (rc == SFFT_ERR_OOM) {  // the device itself is full: release idle lanes and retry once
            if (!make_room(pl, pl->budget, true, 0)) return SFFT_ERR_BUSY;
            rc = create_server(cfg, pl->depth, pl->batch, &srv);
        }
        if (rc != SFFT_OK) return rc;
        const uint64_t bytes = server_bytes(srv);
        if (!make_room(pl, bytes, true, 0)) {
            sfft_server_destroy((sfft_server_t)srv);
            return SFFT_ERR_BUSY;
        }
        srv->eager = pl->eager;
        lane = &pl->lanes[pl->nlanes++];
        lane->id = pl->next_id++;
        lane->cfg = *cfg;
        lane->srv = srv;
        lane->bytes = bytes;
        pl->used += bytes;
    }
    lane->last_use = ++pl->clock;
    sfft_ticket t;
    const int rc = sfft_submit((sfft_server_t)lane->srv, req, &t);
    if (rc != SFFT_OK) return rc;
    ticket->lane = lane->id;
    ticket->seq = t.seq;
    return SFFT_OK;
}

int sfft_pool_wait(sfft_pool_t pool, const sfft_pool_ticket *ticket, int64_t timeout_us) {
    if (!pool || !ticket) return SFFT_ERR_INVALID;
    Pool *pl = (Pool *)pool;
    Server *srv = nullptr;
    {
        std::lock_guard<std::mutex> lock(pl->mu);
        if (ticket->lane == 0 || ticket->lane >= pl->next_id) return SFFT_ERR_INVALID;
        if (pl->eager) {  // before blocking: start the open batches of idle lanes
            for (int k = 0; k < pl->nlanes; ++k) {
                Server *o = pl->lanes[k].srv;
                std::lock_guard<std::mutex> lk(o->mu);
                eager_flush(o);
            }
        }
        Lane *l = find_lane(pl, ticket->lane);
        if (!l) return SFFT_OK;  // a lane is released only once all its requests have completed
        srv = l->srv;
        ++srv->refs;  // the lane is not released while this wait uses it
    }
    sfft_ticket t{ticket->seq};
    const int rc = sfft_wait((sfft_server_t)srv, &t, timeout_us);
    std::lock_guard<std::mutex> lock(pl->mu);
    --srv->refs;
    return rc;
}

int sfft_pool_poll(sfft_pool_t pool, const sfft_pool_ticket *ticket) {
    if (!pool || !ticket) return SFFT_ERR_INVALID;
    Pool *pl = (Pool *)pool;
    std::lock_guard<std::mutex> lock(pl->mu);
    if (ticket->lane == 0 || ticket->lane >= pl->next_id) return SFFT_ERR_INVALID;
    Lane *l = find_lane(pl, ticket->lane);
    if (!l) return SFFT_OK;
    sfft_ticket t{ticket->seq};
    return sfft_poll((sfft_server_t)l->srv, &t);
}

int sfft_pool_set_eager(sfft_pool_t pool, int32_t enable) {
    if (!pool) return SFFT_ERR_INVALID;
    Pool *pl = (Pool *)pool;
    std::lock_guard<std::mutex> lock(pl->mu);
    pl->eager = enable != 0;
    int rc = SFFT_OK;
    for (int k = 0; k < pl->nlanes; ++k) {
        Server *o = pl->lanes[k].srv;
        std::lock_guard<std::mutex> lk(o->mu);
        o->eager = pl->eager;
        const int r = eager_flush(o);
        if (rc == SFFT_OK) rc = r;
    }
    return rc;
}

int sfft_pool_usage(sfft_pool_t pool, uint64_t *bytes, int32_t *lanes) {
    if (!pool || !bytes || !lanes) return SFFT_ERR_INVALID;
    Pool *pl = (Pool *)pool;
    std::lock_guard<std::mutex> lock(pl->mu);
    *bytes = pl->used;
    *lanes = pl->nlanes;
    return SFFT_OK;
}

}  // extern "C"
