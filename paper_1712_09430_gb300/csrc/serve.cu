// Request loop with continuous batching (Sec. 3.2: independent events share
// the GPU "as long as the GPU memory suffices").
//
// tpc_stream_submit admits a request when the free part of the serving arena
// covers its reservation and a slot is free; the input is copied to pinned
// host memory before the call returns.  Admitted requests wait in a FIFO.
// Whenever fewer than max_inflight batches run, all pending requests (up to
// max_batch_events events) form the next batch (with a batching policy set,
// only once enough work is pending while another batch runs): one H2D per request, the
// batched stages of tpc_track_sectors on the batch's own stream, and a D2H
// of the counters and of an estimated output (fetch the rest if the estimate
// was short, Sec. 3.1).  Requests that arrive while batches run join the
// next one.  tpc_stream_poll drives the loop and hands out each request's
// slice of its batch's output.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <thread>

#include "tpc_serve.h"

using namespace tpc;

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Request {
    uint64_t ticket = 0, tag = 0;
    int n_events = 0;
    int N = 0;
    std::vector<int32_t> row_counts;
    size_t pin_off = 0, pin_bytes = 0;  // input copy in the pinned staging
    const tpc_cluster* src = nullptr;   // caller's buffer when submitted without a copy
    size_t reserve = 0;                 // arena bytes reserved at admission
    int state = 0;                      // 0 pending, 1 in flight, 2 done, 3 failed
    int batch = -1;
    int err = TPC_OK;
    // slice of the batch output (rebased to the request on the device)
    int e0 = 0, cl0 = 0;                // first event / cluster of the request in the batch
    int m0 = 0, m1 = 0;                 // track range
    int h0 = 0, h1 = 0;                 // hit range
    bool viewed = false;                // handed out by tpc_stream_poll_view
    std::chrono::steady_clock::time_point t_submit;  // admission time (batching policy)
};

struct Batch {
    int id = -1;
    bool busy = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t start = nullptr;        // timing: first H2D of the batch
    size_t arena_off = 0, arena_bytes = 0;
    BatchShape sh;
    DevPtrs p{};
    std::vector<uint64_t> tickets;
    // pinned per-batch host buffers
    int* plan = nullptr;                // row counts, row offsets, bin offsets
    size_t plan_cap = 0;
    int* counters = nullptr;            // [kNumCounters]
    tpc_track* tracks = nullptr;
    int* hits = nullptr;
    tpc_fit* fits = nullptr;            // with params.refit
    tpc_merge* merges = nullptr;        // with params.merge
    tpc_t0* t0s = nullptr;              // with params.t0
    size_t tracks_cap = 0, hits_cap = 0, fits_cap = 0, merges_cap = 0, t0s_cap = 0;
    int est_tracks = 0, est_hits = 0;   // what the D2H enqueued
    int open_results = 0;               // requests of the batch not yet polled
};

// First-fit allocator over [0, size) with coalescing.
struct Arena {
    size_t size = 0;
    std::vector<std::pair<size_t, size_t>> free;  // (offset, bytes), sorted
    void init(size_t s)
    {
        size = s;
        free.clear();
        if (s) free.push_back({0, s});
    }
    bool alloc(size_t bytes, size_t* off)
    {
        for (size_t i = 0; i < free.size(); i++) {
            if (free[i].second >= bytes) {
                *off = free[i].first;
                free[i].first += bytes;
                free[i].second -= bytes;
                if (!free[i].second) free.erase(free.begin() + (long)i);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        auto it = std::lower_bound(free.begin(), free.end(), std::make_pair(off, size_t(0)));
        it = free.insert(it, {off, bytes});
        size_t i = (size_t)(it - free.begin());
        if (i + 1 < free.size() && free[i].first + free[i].second == free[i + 1].first) {
            free[i].second += free[i + 1].second;
            free.erase(free.begin() + (long)i + 1);
        }
        if (i > 0 && free[i - 1].first + free[i - 1].second == free[i].first) {
            free[i - 1].second += free[i].second;
            free.erase(free.begin() + (long)i);
        }
    }
};

bool fault(const char* name)
{
    const char* v = std::getenv(name);
    return v && *v && std::strcmp(v, "0") != 0;
}

}  // namespace

struct ServeState {
    size_t arena_bytes = 0;        // 0: choose at first submit
    int max_batch_events = 64;
    int64_t max_batch_clusters = TPC_STREAM_BATCH_CLUSTERS;  // 0: no limit
    int max_inflight = 2;
    // batching policy: while a batch runs, the next one forms only once the
    // pending requests hold min_batch_clusters clusters or the oldest has
    // waited max_wait_us (0: whenever a slot is free)
    int64_t min_batch_clusters = 0;
    int max_wait_us = 0;
    int max_requests = 4096;
    int flags = 0;                 // TPC_STREAM_NO_COPY
    void* arena_base = nullptr;
    Arena arena;                   // device workspace of running batches
    size_t reserved = 0;           // admission: sum of reservations of live requests
    char* pin = nullptr;           // pinned input staging
    Arena pin_arena;
    std::deque<uint64_t> pending;
    std::deque<uint64_t> finished;  // tickets in the order their batches finished (tpc_stream_poll_any)
    std::map<uint64_t, Request> req;
    std::vector<Batch> batches;    // slots
    uint64_t next_ticket = 1;
    int next_batch = 0;
    int inflight = 0;
    double tracks_per_cluster = 0.012, hits_per_cluster = 0.9;  // D2H estimate, adapted
    tpc_stream_stats stats{};
};

namespace {
double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}
}  // namespace

static int grow_pinned(tpc_tracker* tr, void** ptr, size_t* cap, size_t want);

static int serve_init(tpc_tracker* tr)
{
    ServeState* S = tr->serve;
    if (S->arena_base) return TPC_OK;
    if (!S->arena_bytes) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, "cudaMemGetInfo");
        S->arena_bytes = std::min<size_t>(fr / 2, (size_t)24 << 30);
    }
    if (fault("TPC_FAULT_ALLOC") || cudaMalloc(&S->arena_base, S->arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        S->arena_base = nullptr;
        return tr->fail(TPC_ERR_NOMEM, "cannot allocate the serving arena");
    }
    S->arena.init(S->arena_bytes);
    // the tracker's pinned plan buffer, which every batch's shape is planned
    // in, sized for a full batch now (growing it later synchronizes the device)
    if (tpc_reserve_plan(tr, (int64_t)S->max_batch_events * tr->geom.n_sectors * tr->geom.n_rows) != TPC_OK) {
        cudaFree(S->arena_base);
        S->arena_base = nullptr;
        return TPC_ERR_NOMEM;
    }
    const size_t pin_bytes = std::max<size_t>(S->arena_bytes / 8, (size_t)64 << 20);
    if (cudaMallocHost(&S->pin, pin_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(S->arena_base);
        S->arena_base = nullptr;
        return tr->fail(TPC_ERR_NOMEM, "cannot allocate pinned staging");
    }
    S->pin_arena.init(pin_bytes);
    // slots: running batches plus finished ones whose results wait for polls
    S->batches.resize((size_t)(2 * S->max_inflight + 2));
    for (auto& b : S->batches) {
        if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&b.done) != cudaSuccess || cudaEventCreate(&b.start) != cudaSuccess ||
            cudaMallocHost(&b.counters, sizeof(int) * kNumCounters) != cudaSuccess)
            return tr->fail(TPC_ERR_DEVICE, "cannot create serving streams");
    }
    // With a cluster limit per batch, every slot's pinned buffers are sized
    // for a full batch now: growing them while serving would mean
    // cudaFreeHost / cudaMallocHost, which synchronize the device and stall
    // every batch in flight.  Hits of a batch never exceed its clusters;
    // tracks are sized for 2 % of them (central and min-bias events make
    // about 1.1 %), beyond which the estimate-then-fetch path still works.
    if (S->max_batch_clusters > 0) {
        const size_t cap = (size_t)S->max_batch_clusters;
        const size_t nt = cap / 50 + 1024, nh = cap + 4096;
        const size_t R = (size_t)S->max_batch_events * tr->geom.n_sectors * tr->geom.n_rows;
        const size_t plan = (3 * R + 2 + 3 * (size_t)S->max_batch_events + 2) * sizeof(int);
        for (auto& b : S->batches) {
            if (grow_pinned(tr, reinterpret_cast<void**>(&b.plan), &b.plan_cap, plan) != TPC_OK ||
                grow_pinned(tr, reinterpret_cast<void**>(&b.tracks), &b.tracks_cap, sizeof(tpc_track) * nt) != TPC_OK ||
                grow_pinned(tr, reinterpret_cast<void**>(&b.hits), &b.hits_cap, sizeof(int) * nh) != TPC_OK ||
                (tr->params.refit &&
                 grow_pinned(tr, reinterpret_cast<void**>(&b.fits), &b.fits_cap, sizeof(tpc_fit) * nt) != TPC_OK) ||
                (tr->params.merge &&
                 grow_pinned(tr, reinterpret_cast<void**>(&b.merges), &b.merges_cap, sizeof(tpc_merge) * nt) != TPC_OK) ||
                (tr->params.t0 &&
                 grow_pinned(tr, reinterpret_cast<void**>(&b.t0s), &b.t0s_cap, sizeof(tpc_t0) * nt) != TPC_OK))
                return TPC_ERR_NOMEM;
        }
    }
    return TPC_OK;
}

static int grow_pinned(tpc_tracker* tr, void** ptr, size_t* cap, size_t want)
{
    if (want <= *cap) return TPC_OK;
    cudaFreeHost(*ptr);
    *ptr = nullptr;
    const size_t old = *cap;
    *cap = 0;
    // grow at least twofold: pinned reallocation is slow and can synchronize
    // the device, so it must stay rare under a growing load
    size_t n = std::max(want + want / 4, 2 * old) + 4096;
    if (cudaMallocHost(ptr, n) != cudaSuccess) {
        cudaGetLastError();
        return tr->fail(TPC_ERR_NOMEM, "pinned result buffer");
    }
    *cap = n;
    return TPC_OK;
}

// Launch all pending requests (up to max_batch_events events) as one batch.
static int launch_batch_impl(tpc_tracker* tr);

static int launch_batch(tpc_tracker* tr)
{
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = launch_batch_impl(tr);
    const double ms = ms_since(t0);
    tr->serve->stats.host_launch_ms += ms;
    tr->serve->stats.max_launch_ms = std::max(tr->serve->stats.max_launch_ms, ms);
    return rc;
}

static int launch_batch_impl(tpc_tracker* tr)
{
    ServeState* S = tr->serve;
    Batch* b = nullptr;
    for (auto& x : S->batches)
        if (!x.busy) { b = &x; break; }
    if (S->pending.empty()) return TPC_OK;
    if (!b) return TPC_BUSY;  // every slot holds results not yet polled
    // take requests in arrival order
    std::vector<uint64_t> take;
    int ev = 0;
    int64_t ncl = 0;
    for (uint64_t t : S->pending) {
        const Request& r = S->req[t];
        if (!take.empty() && (ev + r.n_events > S->max_batch_events ||
                              (S->max_batch_clusters > 0 && ncl + r.N > S->max_batch_clusters)))
            break;
        take.push_back(t);
        ev += r.n_events;
        ncl += r.N;
    }
    const int NR = tr->geom.n_rows, NS = tr->geom.n_sectors;
    const size_t R = (size_t)ev * NS * NR;
    // the batch's pinned host buffer: row counts [R], plan [2 (R + 1)], first
    // event of each event's request [ev], first (track, hit) of each event
    // [2 (ev + 1)] (filled by the device)
    if (grow_pinned(tr, reinterpret_cast<void**>(&b->plan), &b->plan_cap,
                    (3 * R + 2 + 3 * (size_t)ev + 2) * sizeof(int)) != TPC_OK)
        return TPC_ERR_NOMEM;
    int* counts = b->plan;
    size_t pos = 0;
    for (uint64_t t : take) {
        const Request& r = S->req[t];
        std::memcpy(counts + pos, r.row_counts.data(), r.row_counts.size() * sizeof(int));
        pos += r.row_counts.size();
    }
    BatchShape sh;
    int rc = tpc_shape(tr, counts, ev, &sh);  // fills tr->plan_host
    if (rc != TPC_OK) return rc;
    std::memcpy(counts + R, tr->plan_host + R, (R + 1) * 2 * sizeof(int));
    const size_t bytes = align256(tpc_layout(tr, sh, nullptr, nullptr));
    size_t off = 0;
    if (!S->arena.alloc(bytes, &off)) return TPC_BUSY;  // wait for a running batch
    b->id = S->next_batch++;
    b->busy = true;
    b->arena_off = off;
    b->arena_bytes = bytes;
    b->sh = sh;
    b->tickets = take;
    tpc_layout(tr, sh, &b->p, static_cast<char*>(S->arena_base) + off);
    b->p.req_first_event = b->p.req_area;
    int* req_first = counts + 3 * R + 2;
    const DevPtrs& p = b->p;
    cudaStream_t s = b->stream;
    int e0 = 0, cl0 = 0;
    cudaError_t e = cudaEventRecord(b->start, s);
    S->stats.batches++;
    S->stats.events += ev;
    S->stats.clusters += sh.N;
    S->stats.max_batch_events = std::max<int64_t>(S->stats.max_batch_events, ev);
    for (uint64_t t : take) {
        Request& r = S->req[t];
        r.state = 1;
        r.batch = (int)(b - S->batches.data());
        r.e0 = e0;
        r.cl0 = cl0;
        for (int q = 0; q < r.n_events; q++) req_first[e0 + q] = e0;
        const void* src = r.src ? static_cast<const void*>(r.src) : S->pin + r.pin_off;
        if (r.N && e == cudaSuccess)
            e = cudaMemcpyAsync(const_cast<float4*>(p.clusters) + cl0, src, (size_t)r.N * 16,
                                cudaMemcpyHostToDevice, s);
        e0 += r.n_events;
        cl0 += r.N;
    }
    S->pending.erase(S->pending.begin(), S->pending.begin() + (long)take.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<int*>(p.row_cnt), counts, (3 * R + 2) * sizeof(int),
                            cudaMemcpyHostToDevice, s);  // counts and plan, adjacent on both sides
    if (e == cudaSuccess && ev > 0)
        e = cudaMemcpyAsync(p.req_area, req_first, (size_t)ev * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, cudaGetErrorString(e));
    S->inflight++;
    if (sh.N > 0) {
        rc = tpc_enqueue(tr, p, sh, s, false);
        if (rc != TPC_OK) return rc;
        // estimated output, fetched right after the last kernel (Sec. 3.1)
        b->est_tracks = std::min<int>(sh.t_cap, (int)(S->tracks_per_cluster * sh.N * 1.3) + 256);
        b->est_hits = std::min<int>(sh.N, (int)(S->hits_per_cluster * sh.N * 1.3) + 4096);
        if (S->max_batch_clusters > 0) {
            // buffers sized when serving started: an estimate beyond them is
            // left to the fetch of the rest rather than a reallocation
            b->est_tracks = std::min<int>(b->est_tracks, (int)(b->tracks_cap / sizeof(tpc_track)));
            b->est_hits = std::min<int>(b->est_hits, (int)(b->hits_cap / sizeof(int)));
        }
        if (grow_pinned(tr, reinterpret_cast<void**>(&b->tracks), &b->tracks_cap,
                        sizeof(tpc_track) * (size_t)b->est_tracks) != TPC_OK ||
            grow_pinned(tr, reinterpret_cast<void**>(&b->hits), &b->hits_cap,
                        sizeof(int) * (size_t)b->est_hits) != TPC_OK)
            return TPC_ERR_NOMEM;
        if (tr->params.refit &&
            grow_pinned(tr, reinterpret_cast<void**>(&b->fits), &b->fits_cap,
                        sizeof(tpc_fit) * (size_t)b->est_tracks) != TPC_OK)
            return TPC_ERR_NOMEM;
        if (tr->params.merge &&
            grow_pinned(tr, reinterpret_cast<void**>(&b->merges), &b->merges_cap,
                        sizeof(tpc_merge) * (size_t)b->est_tracks) != TPC_OK)
            return TPC_ERR_NOMEM;
        if (tr->params.t0 &&
            grow_pinned(tr, reinterpret_cast<void**>(&b->t0s), &b->t0s_cap,
                        sizeof(tpc_t0) * (size_t)b->est_tracks) != TPC_OK)
            return TPC_ERR_NOMEM;
        e = cudaMemcpyAsync(b->counters, p.counters, sizeof(int) * kNumCounters, cudaMemcpyDeviceToHost, s);
        // first (track, hit) of every event, to slice the output per request
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(req_first + ev, p.ev_first, ((size_t)ev + 1) * sizeof(int2),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->tracks, p.out_tracks, sizeof(tpc_track) * (size_t)b->est_tracks,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->hits, p.out_hits, sizeof(int) * (size_t)b->est_hits,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && tr->params.refit)
            e = cudaMemcpyAsync(b->fits, p.out_fits, sizeof(tpc_fit) * (size_t)b->est_tracks,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && tr->params.merge)
            e = cudaMemcpyAsync(b->merges, p.out_merges, sizeof(tpc_merge) * (size_t)b->est_tracks,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && tr->params.t0)
            e = cudaMemcpyAsync(b->t0s, p.out_t0s, sizeof(tpc_t0) * (size_t)b->est_tracks,
                                cudaMemcpyDeviceToHost, s);
    } else {
        std::memset(b->counters, 0, sizeof(int) * kNumCounters);
        std::memset(req_first + ev, 0, sizeof(int2) * ((size_t)ev + 1));
        b->est_tracks = b->est_hits = 0;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->done, s);
    if (e != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, cudaGetErrorString(e));
    return TPC_OK;
}

// A finished batch: fetch the rest if the estimate was short, slice the
// output per request, free the device workspace.
static void finish_batch(tpc_tracker* tr, Batch& b)
{
    ServeState* S = tr->serve;
    const auto t_host = std::chrono::steady_clock::now();
    {
        float gms = 0.0f;
        if (cudaEventElapsedTime(&gms, b.start, b.done) == cudaSuccess) S->stats.gpu_ms += gms;
        else cudaGetLastError();
    }
    int err = TPC_OK;
    const int* c = b.counters;
    const int M = b.sh.N ? c[C_M] : 0, MH = b.sh.N ? c[C_MH] : 0;
    if (b.sh.N && (c[C_ERR] & E_INPUT)) err = TPC_ERR_INVALID;
    if (b.sh.N && (c[C_ERR] & E_TIMEOUT)) err = TPC_ERR_TIMEOUT;
    if (b.sh.N && (c[C_ERR] & E_SHAPE)) err = TPC_ERR_DEVICE;
    if (err == TPC_OK && (M > b.est_tracks || MH > b.est_hits)) {
        // the estimate was short: fetch the remainder now
        S->stats.refetches++;
        void* tp = b.tracks;
        void* hp = b.hits;
        size_t tc = b.tracks_cap, hc = b.hits_cap;
        std::vector<tpc_track> keep_t(b.tracks, b.tracks + std::min(M, b.est_tracks));
        std::vector<int> keep_h(b.hits, b.hits + std::min(MH, b.est_hits));
        if (grow_pinned(tr, &tp, &tc, sizeof(tpc_track) * (size_t)M) != TPC_OK ||
            grow_pinned(tr, &hp, &hc, sizeof(int) * (size_t)MH) != TPC_OK) {
            err = TPC_ERR_NOMEM;
        } else {
            b.tracks = static_cast<tpc_track*>(tp);
            b.hits = static_cast<int*>(hp);
            b.tracks_cap = tc;
            b.hits_cap = hc;
            if (cudaMemcpy(b.tracks, b.p.out_tracks, sizeof(tpc_track) * (size_t)M, cudaMemcpyDeviceToHost) !=
                    cudaSuccess ||
                cudaMemcpy(b.hits, b.p.out_hits, sizeof(int) * (size_t)MH, cudaMemcpyDeviceToHost) != cudaSuccess)
                err = TPC_ERR_DEVICE;
            if (err == TPC_OK && tr->params.refit) {
                void* fp = b.fits;
                size_t fc = b.fits_cap;
                if (grow_pinned(tr, &fp, &fc, sizeof(tpc_fit) * (size_t)M) != TPC_OK) {
                    err = TPC_ERR_NOMEM;
                } else {
                    b.fits = static_cast<tpc_fit*>(fp);
                    b.fits_cap = fc;
                    if (cudaMemcpy(b.fits, b.p.out_fits, sizeof(tpc_fit) * (size_t)M, cudaMemcpyDeviceToHost) !=
                        cudaSuccess)
                        err = TPC_ERR_DEVICE;
                }
            }
            if (err == TPC_OK && tr->params.t0) {
                void* tp0 = b.t0s;
                size_t tc0 = b.t0s_cap;
                if (grow_pinned(tr, &tp0, &tc0, sizeof(tpc_t0) * (size_t)M) != TPC_OK) {
                    err = TPC_ERR_NOMEM;
                } else {
                    b.t0s = static_cast<tpc_t0*>(tp0);
                    b.t0s_cap = tc0;
                    if (cudaMemcpy(b.t0s, b.p.out_t0s, sizeof(tpc_t0) * (size_t)M, cudaMemcpyDeviceToHost) !=
                        cudaSuccess)
                        err = TPC_ERR_DEVICE;
                }
            }
            if (err == TPC_OK && tr->params.merge) {
                void* mp = b.merges;
                size_t mc = b.merges_cap;
                if (grow_pinned(tr, &mp, &mc, sizeof(tpc_merge) * (size_t)M) != TPC_OK) {
                    err = TPC_ERR_NOMEM;
                } else {
                    b.merges = static_cast<tpc_merge*>(mp);
                    b.merges_cap = mc;
                    if (cudaMemcpy(b.merges, b.p.out_merges, sizeof(tpc_merge) * (size_t)M,
                                   cudaMemcpyDeviceToHost) != cudaSuccess)
                        err = TPC_ERR_DEVICE;
                }
            }
        }
    }
    if (b.sh.N > 0) {  // adapt the estimate to what central/min-bias events produce
        S->tracks_per_cluster = std::max(S->tracks_per_cluster * 0.9, (double)M / b.sh.N);
        S->hits_per_cluster = std::max(S->hits_per_cluster * 0.9, (double)MH / b.sh.N);
    }
    // tracks are in canonical order, grouped by event, so by request; the
    // device wrote the first (track, hit) of every event
    b.open_results = 0;
    const int ev = b.sh.n_events;
    const int2* evf = reinterpret_cast<const int2*>(b.plan + 3 * (size_t)b.sh.R + 2 + ev);
    for (uint64_t t : b.tickets) {
        Request& r = S->req[t];
        r.err = err;
        r.state = err == TPC_OK ? 2 : 3;
        const int2 f0 = evf[r.e0], f1 = evf[r.e0 + r.n_events];
        r.m0 = err == TPC_OK ? f0.x : 0;
        r.m1 = err == TPC_OK ? f1.x : 0;
        r.h0 = err == TPC_OK ? f0.y : 0;
        r.h1 = err == TPC_OK ? f1.y : 0;
        if (r.pin_bytes) S->pin_arena.release(r.pin_off, r.pin_bytes);
        r.pin_bytes = 0;
        b.open_results++;
        S->finished.push_back(t);
    }
    if (S->finished.size() > 4 * (size_t)S->max_requests) {  // drop tickets taken by per-ticket polls
        std::deque<uint64_t> keep;
        for (uint64_t t : S->finished) {
            auto it = S->req.find(t);
            if (it != S->req.end() && !it->second.viewed) keep.push_back(t);
        }
        S->finished.swap(keep);
    }
    S->arena.release(b.arena_off, b.arena_bytes);
    S->inflight--;
    S->stats.host_finish_ms += ms_since(t_host);
}

// With a batch already running: is the pending work worth a batch of its
// own now (enough clusters, a full batch, or the oldest request waited long
// enough)?  Otherwise it waits and joins a larger batch.
static bool batch_ready(const ServeState* S)
{
    int64_t ncl = 0;
    int ev = 0;
    for (uint64_t t : S->pending) {
        const Request& r = S->req.at(t);
        ncl += r.N;
        ev += r.n_events;
    }
    if (ncl >= S->min_batch_clusters || ev >= S->max_batch_events) return true;
    if (S->max_batch_clusters > 0 && ncl >= S->max_batch_clusters) return true;
    const Request& oldest = S->req.at(S->pending.front());
    const auto waited = std::chrono::duration_cast<std::chrono::microseconds>(
        std::chrono::steady_clock::now() - oldest.t_submit);
    return waited.count() >= S->max_wait_us;
}

static int progress(tpc_tracker* tr)
{
    ServeState* S = tr->serve;
    for (auto& b : S->batches) {
        if (!b.busy || b.open_results) continue;
        if (b.tickets.empty()) continue;
        cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, cudaGetErrorString(q));
        finish_batch(tr, b);
        if (!b.open_results) {
            b.busy = false;
            b.tickets.clear();
        }
    }
    while (!S->pending.empty() && S->inflight < S->max_inflight) {
        if (S->inflight > 0 && S->min_batch_clusters > 0 && !batch_ready(S)) break;
        int rc = launch_batch(tr);
        if (rc == TPC_BUSY) break;  // arena fragmented: wait for a running batch
        if (rc != TPC_OK) return rc;
    }
    return TPC_OK;
}

void tpc_serve_shutdown(tpc_tracker* tr)
{
    ServeState* S = tr->serve;
    if (!S) return;
    for (auto& b : S->batches) {
        if (b.stream) cudaStreamSynchronize(b.stream);
        if (b.stream) cudaStreamDestroy(b.stream);
        if (b.done) cudaEventDestroy(b.done);
        if (b.start) cudaEventDestroy(b.start);
        cudaFreeHost(b.plan);
        cudaFreeHost(b.counters);
        cudaFreeHost(b.tracks);
        cudaFreeHost(b.hits);
        cudaFreeHost(b.fits);
        cudaFreeHost(b.merges);
        cudaFreeHost(b.t0s);
    }
    cudaFree(S->arena_base);
    cudaFreeHost(S->pin);
    delete S;
    tr->serve = nullptr;
}

bool tpc_serve_busy(const tpc_tracker* tr) { return tr->serve && !tr->serve->req.empty(); }

extern "C" int tpc_stream_configure(tpc_tracker* tr, size_t arena_bytes, int max_batch_events,
                                    int max_inflight, int flags, int64_t max_batch_clusters)
{
    if (!tr) return TPC_ERR_INVALID;
    if (tr->serve && (tr->serve->arena_base || !tr->serve->req.empty()))
        return tr->fail(TPC_BUSY, "serving already started");
    if (max_batch_events < 1 || max_inflight < 1 || max_inflight > 8 || max_batch_clusters < 0)
        return tr->fail(TPC_ERR_INVALID, "max_batch_events >= 1, max_inflight in [1, 8], max_batch_clusters >= 0");
    if (!tr->serve) tr->serve = new ServeState();
    tr->serve->arena_bytes = arena_bytes;
    tr->serve->max_batch_events = max_batch_events;
    tr->serve->max_inflight = max_inflight;
    tr->serve->flags = flags;
    tr->serve->max_batch_clusters = max_batch_clusters;
    return TPC_OK;
}

extern "C" int tpc_stream_set_batching(tpc_tracker* tr, int64_t min_batch_clusters, int max_wait_us)
{
    if (!tr) return TPC_ERR_INVALID;
    if (min_batch_clusters < 0 || max_wait_us < 0)
        return tr->fail(TPC_ERR_INVALID, "min_batch_clusters and max_wait_us must be >= 0");
    if (!tr->serve) tr->serve = new ServeState();
    tr->serve->min_batch_clusters = min_batch_clusters;
    tr->serve->max_wait_us = max_wait_us;
    return TPC_OK;
}

namespace {
// The longest tpc_stream_submit call after serving was set up, kept in the
// stats on every return.
struct SubmitTimer {
    tpc_tracker* tr;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    ~SubmitTimer()
    {
        if (tr && tr->serve) tr->serve->stats.max_submit_ms = std::max(tr->serve->stats.max_submit_ms, ms_since(t0));
    }
};
}  // namespace

extern "C" int tpc_stream_submit(tpc_tracker* tr, const tpc_cluster* clusters, const int32_t* row_counts,
                                 int n_events, uint64_t tag, uint64_t* ticket)
{
    if (!tr) return TPC_ERR_INVALID;
    if (!row_counts || !ticket || n_events < 1) return tr->fail(TPC_ERR_INVALID, "NULL argument or n_events < 1");
    if (cudaSetDevice(tr->dev) != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, "cudaSetDevice");
    if (!tr->serve) tr->serve = new ServeState();
    int rc = serve_init(tr);  // the first submit allocates the arena and staging
    if (rc != TPC_OK) return rc;
    const SubmitTimer timer{tr};  // from here: the submit itself
    ServeState* S = tr->serve;
    rc = progress(tr);
    if (rc != TPC_OK) return rc;
    BatchShape sh;
    rc = tpc_shape(tr, row_counts, n_events, &sh);
    if (rc != TPC_OK) return rc;
    if (sh.N > 0 && !clusters) return tr->fail(TPC_ERR_INVALID, "NULL clusters");
    if (n_events > S->max_batch_events) return tr->fail(TPC_ERR_INVALID, "more events than max_batch_events");
    // admission: the request's own workspace (input + ~3x internal buffers,
    // Sec. 4.1) must fit the free part of the arena, and a slot must be free
    const size_t reserve = align256(tpc_layout(tr, sh, nullptr, nullptr)) + ((size_t)1 << 20);
    if (reserve > S->arena.size) return tr->fail(TPC_ERR_NOMEM, "request larger than the serving arena");
    if (fault("TPC_FAULT_ADMIT") || S->reserved + reserve > S->arena.size ||
        (int)S->req.size() >= S->max_requests)
        return TPC_BUSY;
    size_t pin_off = 0;
    const bool no_copy = (S->flags & TPC_STREAM_NO_COPY) != 0;
    const size_t pin_bytes = no_copy ? 0 : align256((size_t)sh.N * 16);
    if (pin_bytes && !S->pin_arena.alloc(pin_bytes, &pin_off)) return TPC_BUSY;
    if (pin_bytes) std::memcpy(S->pin + pin_off, clusters, (size_t)sh.N * 16);
    Request r;
    r.ticket = S->next_ticket++;
    r.tag = tag;
    r.n_events = n_events;
    r.N = sh.N;
    r.row_counts.assign(row_counts, row_counts + sh.R);
    r.pin_off = pin_off;
    r.pin_bytes = pin_bytes;
    r.src = no_copy ? clusters : nullptr;
    r.reserve = reserve;
    r.t_submit = std::chrono::steady_clock::now();
    S->reserved += reserve;
    S->req[r.ticket] = std::move(r);
    S->pending.push_back(S->next_ticket - 1);
    *ticket = S->next_ticket - 1;
    rc = progress(tr);
    return rc == TPC_OK ? TPC_OK : rc;
}

// Drive the loop until the ticket's batch is done or the time runs out.
static int wait_ticket(tpc_tracker* tr, uint64_t ticket, int timeout_us, Request** out)
{
    ServeState* S = tr->serve;
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max(0, timeout_us));
    while (true) {
        int rc = progress(tr);
        if (rc != TPC_OK) return rc;
        auto it = S->req.find(ticket);
        if (it == S->req.end()) return TPC_ERR_UNKNOWN_TICKET;
        if (it->second.state >= 2) {
            *out = &it->second;
            return TPC_OK;
        }
        if (std::chrono::steady_clock::now() >= t_end) return TPC_PENDING;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Forget a finished request; its batch slot frees with its last request.
static void release_ticket(tpc_tracker* tr, uint64_t ticket)
{
    ServeState* S = tr->serve;
    auto it = S->req.find(ticket);
    Batch& b = S->batches[(size_t)it->second.batch];
    S->reserved -= it->second.reserve;
    S->req.erase(it);
    if (--b.open_results == 0) {
        b.busy = false;
        b.tickets.clear();
        progress(tr);
    }
}

extern "C" int tpc_stream_poll(tpc_tracker* tr, uint64_t ticket, tpc_output* out, int timeout_us)
{
    if (!tr) return TPC_ERR_INVALID;
    if (!out) return tr->fail(TPC_ERR_INVALID, "NULL output");
    if (!tr->serve) return TPC_ERR_UNKNOWN_TICKET;
    if (cudaSetDevice(tr->dev) != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, "cudaSetDevice");
    ServeState* S = tr->serve;
    Request* r = nullptr;
    int rc = wait_ticket(tr, ticket, timeout_us, &r);
    if (rc != TPC_OK) return rc;
    Batch& b = S->batches[(size_t)r->batch];
    const int result = r->err;
    if (result == TPC_OK) {
        const int M = r->m1 - r->m0, MH = r->h1 - r->h0;
        out->n_tracks = M;
        out->n_hits = MH;
        if (M > out->cap_tracks || MH > out->cap_hits)
            return tr->fail(TPC_ERR_OUTPUT_TRUNCATED, "output capacity too small");
        if (out->mem_kind != TPC_MEM_HOST)
            return tr->fail(TPC_ERR_INVALID, "stream results are returned in host memory");
        const auto t_copy = std::chrono::steady_clock::now();
        if (M) std::memcpy(out->tracks, b.tracks + r->m0, sizeof(tpc_track) * (size_t)M);
        if (MH) std::memcpy(out->hit_ids, b.hits + r->h0, sizeof(int32_t) * (size_t)MH);
        if (M && out->fits && tr->params.refit)
            std::memcpy(out->fits, b.fits + r->m0, sizeof(tpc_fit) * (size_t)M);
        if (M && out->merges && tr->params.merge)
            std::memcpy(out->merges, b.merges + r->m0, sizeof(tpc_merge) * (size_t)M);
        if (M && out->t0s && tr->params.t0) std::memcpy(out->t0s, b.t0s + r->m0, sizeof(tpc_t0) * (size_t)M);
        S->stats.host_copy_ms += ms_since(t_copy);
    }
    release_ticket(tr, ticket);
    return result == TPC_OK ? TPC_OK : tr->fail(result, "batch failed");
}

extern "C" int tpc_stream_poll_view(tpc_tracker* tr, uint64_t ticket, tpc_stream_view* view, int timeout_us)
{
    if (!tr) return TPC_ERR_INVALID;
    if (!view) return tr->fail(TPC_ERR_INVALID, "NULL view");
    if (!tr->serve) return TPC_ERR_UNKNOWN_TICKET;
    if (cudaSetDevice(tr->dev) != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, "cudaSetDevice");
    ServeState* S = tr->serve;
    Request* r = nullptr;
    int rc = wait_ticket(tr, ticket, timeout_us, &r);
    if (rc != TPC_OK) return rc;
    if (r->err != TPC_OK) {
        const int result = r->err;
        release_ticket(tr, ticket);
        return tr->fail(result, "batch failed");
    }
    const Batch& b = S->batches[(size_t)r->batch];
    view->tracks = b.tracks + r->m0;
    view->hit_ids = b.hits + r->h0;
    view->fits = tr->params.refit ? b.fits + r->m0 : nullptr;
    view->merges = tr->params.merge ? b.merges + r->m0 : nullptr;
    view->t0s = tr->params.t0 ? b.t0s + r->m0 : nullptr;
    view->n_tracks = r->m1 - r->m0;
    view->n_hits = r->h1 - r->h0;
    r->viewed = true;
    return TPC_OK;
}

extern "C" int tpc_stream_poll_any(tpc_tracker* tr, uint64_t* ticket, tpc_stream_view* view, int timeout_us)
{
    if (!tr) return TPC_ERR_INVALID;
    if (!ticket || !view) return tr->fail(TPC_ERR_INVALID, "NULL ticket or view");
    if (!tr->serve) return TPC_PENDING;
    if (cudaSetDevice(tr->dev) != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, "cudaSetDevice");
    ServeState* S = tr->serve;
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max(0, timeout_us));
    while (true) {
        int rc = progress(tr);
        if (rc != TPC_OK) return rc;
        while (!S->finished.empty()) {
            const uint64_t t = S->finished.front();
            S->finished.pop_front();
            auto it = S->req.find(t);
            if (it == S->req.end() || it->second.viewed) continue;  // taken by a per-ticket poll
            Request& r = it->second;
            *ticket = t;
            if (r.err != TPC_OK) {
                const int result = r.err;
                release_ticket(tr, t);
                return tr->fail(result, "batch failed");
            }
            const Batch& b = S->batches[(size_t)r.batch];
            view->tracks = b.tracks + r.m0;
            view->hit_ids = b.hits + r.h0;
            view->fits = tr->params.refit ? b.fits + r.m0 : nullptr;
            view->merges = tr->params.merge ? b.merges + r.m0 : nullptr;
            view->t0s = tr->params.t0 ? b.t0s + r.m0 : nullptr;
            view->n_tracks = r.m1 - r.m0;
            view->n_hits = r.h1 - r.h0;
            r.viewed = true;
            return TPC_OK;
        }
        if (std::chrono::steady_clock::now() >= t_end) return TPC_PENDING;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" int tpc_stream_release(tpc_tracker* tr, uint64_t ticket)
{
    if (!tr) return TPC_ERR_INVALID;
    if (!tr->serve) return TPC_ERR_UNKNOWN_TICKET;
    ServeState* S = tr->serve;
    auto it = S->req.find(ticket);
    if (it == S->req.end()) return TPC_ERR_UNKNOWN_TICKET;
    if (it->second.state < 2) return tr->fail(TPC_ERR_INVALID, "ticket still pending");
    if (cudaSetDevice(tr->dev) != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, "cudaSetDevice");
    release_ticket(tr, ticket);
    return TPC_OK;
}

extern "C" int tpc_stream_get_stats(const tpc_tracker* tr, tpc_stream_stats* stats)
{
    if (!tr || !stats) return TPC_ERR_INVALID;
    if (!tr->serve) {
        *stats = tpc_stream_stats{};
        return TPC_OK;
    }
    *stats = tr->serve->stats;
    return TPC_OK;
}
