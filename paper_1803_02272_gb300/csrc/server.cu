// Serving: a resident reference set answers query batches with distance rows (the
// rectangular form of `disseq` in section 2.2, used to place new reads into the map of
// a sample, and the read-vs-reference-database distances of the supervised annotation).
//
// Continuous batching with shortest-remaining-work-first dispatch:
//  * gbd_server_submit validates and copies a request on the host and queues it; it
//    returns at once with a ticket (or EBUDGET if the request can never fit).
//  * A worker thread admits queued requests in arrival order while their footprint (the
//    output rows plus the packed queries) fits the HBM budget beside the requests in
//    flight.  An admitted request's queries are copied and packed on the device once
//    (ingest stream), and the request is cut into chunks of about kChunkPairs pairs.
//  * At most kSlots chunk batches are on the GPU at a time.  Whenever a slot frees, the
//    worker fills the next batch with chunks of the admitted requests with the least
//    remaining work first, up to kChunkPairs pairs, and launches it (one launch of the
//    systolic kernel per rows-per-lane bucket) on the slot's stream, so batches overlap
//    and a small request never waits behind more than one batch of a large one.
//  * A host callback at the end of a batch's stream work counts its chunks done; the
//    last chunk of a request marks it done and returns its budget.
// Every pair is computed independently by the same kernels whatever else is in the
// batch, so a request's rows are identical alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "gbd_internal.cuh"
#include "sw_systolic.cuh"

namespace gbd {
namespace {

enum ReqState { REQ_QUEUED = 0, REQ_ACTIVE = 1, REQ_DONE = 2, REQ_FAILED = 3 };

// Pairs per chunk batch: about 0.15 s of GPU work when few pairs wait, an eighth of the
// waiting work up to 64 Mi pairs otherwise (a newly arrived small request waits at most
// for a slot to free, so the batch length bounds its latency), and up to 256 Mi pairs
// when a backlog of kBacklog requests or more is waiting: a batch's launches then hold
// more queries per length bucket, so their work units are longer (twice the cost
// model's piece) and the per-unit pipeline fill and the launch tails cost a smaller
// share than in one launch per request.
constexpr uint64_t kChunkPairs = 12u << 20;
constexpr uint64_t kMaxChunkPairs = 64u << 20;
constexpr uint64_t kBacklogChunkPairs = 256u << 20;
constexpr size_t kBacklog = 8;
constexpr double kBacklogPieceScale = 2.0;
constexpr double kAgeSeconds = 1.0;    // waiting time that halves a request's sort key
constexpr int kSlots = 2;                     // chunk batches in flight

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> seq;        // validated bytes, offsets rebased to 0
    std::vector<uint64_t> off;
    std::vector<uint16_t> len;
    uint64_t nq = 0;
    uint32_t max_len = 0, stride = 1;
    uint16_t *d_rows = nullptr;
    uint64_t footprint = 0;
    int state = REQ_QUEUED;
    std::string error;
    // device side, once admitted
    std::vector<void *> dev;         // allocations to free after the last chunk
    uint32_t *d_words = nullptr;
    uint16_t *d_len = nullptr;
    cudaEvent_t packed = nullptr;
    uint64_t next_query = 0;         // first query not yet dispatched
    uint64_t chunks_inflight = 0;
    std::chrono::steady_clock::time_point submitted;
};

struct Piece {
    Request *req;
    uint64_t q0, q1;                 // query range of the request
};

struct Batch {
    std::vector<Piece> pieces;
    struct gbd_server *srv = nullptr;
    int slot = 0;
};

}  // namespace
}  // namespace gbd

using namespace gbd;

struct gbd_server {
    gbd_ctx *ctx = nullptr;
    const gbd_set *ref = nullptr;
    cudaStream_t slots[kSlots] = {};
    gbd::StreamSet slot_aux[kSlots];           // a second stream per slot for bucket launches
    bool slot_busy[kSlots] = {};
    cudaStream_t ingest = nullptr;             // packing and batch uploads
    cudaEvent_t uploaded[kSlots] = {};         // a slot's uploads are complete
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;               // submitted, not admitted
    std::vector<Request *> active;             // admitted, not finished
    std::vector<std::vector<void *>> garbage;  // device memory of finished requests
    std::unordered_map<uint64_t, std::unique_ptr<Request>> table;
    uint64_t budget = 0, used = 0, next_ticket = 1;
    bool stop = false;
};

namespace gbd {
namespace {

bool valid_base(uint8_t c)
{
    const uint8_t u = c | 0x20;
    return u == 'a' || u == 'c' || u == 'g' || u == 't';
}

bool use_systolic_scores(const gbd_params &p)
{
    return p.kernel != GBD_KERNEL_GENERAL && p.match == 1 && p.mismatch == -1 && p.gap == 1 && p.gap_open >= 0 &&
           p.gap_open <= kSystolicMaxGapOpen;
}

// Called with srv->mu held: one chunk of r finished (or failed with `err`).
void chunk_finished(gbd_server *srv, Request *r, const std::string &err)
{
    if (!err.empty() && r->error.empty()) r->error = err;
    --r->chunks_inflight;
    if (r->chunks_inflight == 0 && (r->next_query >= r->nq || !r->error.empty())) {
        r->state = r->error.empty() ? REQ_DONE : REQ_FAILED;
        r->next_query = r->nq;
        srv->used -= r->footprint;
        srv->garbage.push_back(std::move(r->dev));
        r->dev.clear();
        srv->active.erase(std::remove(srv->active.begin(), srv->active.end(), r), srv->active.end());
    }
}

void CUDART_CB batch_done(void *arg)
{
    // Runs on a CUDA callback thread once the batch's stream work has finished: no CUDA
    // calls here, only bookkeeping.
    Batch *b = static_cast<Batch *>(arg);
    gbd_server *srv = b->srv;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (const Piece &p : b->pieces) chunk_finished(srv, p.req, std::string());
        srv->slot_busy[b->slot] = false;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
    delete b;
}

// Copies and packs an admitted request's queries on the ingest stream.
std::string admit(gbd_server *srv, Request *r)
{
    cudaStream_t st = srv->ingest;
    std::string err;
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && err.empty()) err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaSuccess;
    };
    uint8_t *d_seq = nullptr;
    uint64_t *d_off = nullptr;
    unsigned long long *d_err = nullptr;
    const size_t nbytes = std::max<size_t>(r->seq.size(), 1);
    if (cu(cudaMallocAsync((void **)&d_seq, nbytes, st), "cudaMallocAsync")) r->dev.push_back(d_seq);
    if (cu(cudaMallocAsync((void **)&d_off, (r->nq + 1) * 8, st), "cudaMallocAsync")) r->dev.push_back(d_off);
    if (cu(cudaMallocAsync((void **)&r->d_words, r->nq * r->stride * 4, st), "cudaMallocAsync"))
        r->dev.push_back(r->d_words);
    if (cu(cudaMallocAsync((void **)&r->d_len, r->nq * 2, st), "cudaMallocAsync")) r->dev.push_back(r->d_len);
    if (cu(cudaMallocAsync((void **)&d_err, 8, st), "cudaMallocAsync")) r->dev.push_back(d_err);
    if (!err.empty()) return err;
    if (!r->seq.empty()) cu(cudaMemcpyAsync(d_seq, r->seq.data(), r->seq.size(), cudaMemcpyHostToDevice, st), "H2D");
    cu(cudaMemcpyAsync(d_off, r->off.data(), (r->nq + 1) * 8, cudaMemcpyHostToDevice, st), "H2D");
    if (err.empty()) cu(launch_pack(d_seq, d_off, r->nq, r->stride, r->d_words, r->d_len, d_err, st), "pack");
    if (err.empty() && cu(cudaEventCreateWithFlags(&r->packed, cudaEventDisableTiming), "cudaEventCreate"))
        cu(cudaEventRecord(r->packed, st), "cudaEventRecord");
    return err;
}

// Launches one batch of pieces on stream st; returns an error message or "".
std::string launch_batch(gbd_server *srv, const std::vector<Piece> &pieces, cudaStream_t st,
                         const StreamSet *aux, cudaEvent_t uploaded)
{
    gbd_ctx *ctx = srv->ctx;
    const gbd_set *ref = srv->ref;
    cudaStream_t up = srv->ingest;
    const bool systolic = use_systolic_scores(ctx->params);
    std::vector<GeneralJob> general;
    std::vector<SysJob> jobs;
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    std::vector<void *> to_free;
    std::string err;
    for (const Piece &p : pieces) {
        Request *r = p.req;
        if (r->packed && cudaStreamWaitEvent(st, r->packed, 0) != cudaSuccess) return "cudaStreamWaitEvent failed";
        SysJob J{};
        J.Q = {r->d_words, r->d_len, r->nq, r->stride};
        J.S = ref->view();
        J.sub_perm = nullptr;
        J.out = r->d_rows;
        J.ld = ref->n;
        J.row0 = 0;
        J.col0 = 0;
        J.mode = OUT_RECT;
        J.conversion = ctx->params.conversion;
        J.gap_open = ctx->params.gap_open;
        J.out_len = out_extent(ctx, r->nq * ref->n);
        const uint32_t job = (uint32_t)jobs.size();
        jobs.push_back(J);
        std::vector<uint32_t> long_rows;
        for (uint64_t i = p.q0; i < p.q1; ++i) {
            if (systolic && r->len[i] <= kSystolicMaxQuery) {
                entries.push_back({job, (uint32_t)i, 0u, (uint32_t)ref->n});
                rows.push_back((uint8_t)systolic_rows(r->len[i]));
            } else {
                long_rows.push_back((uint32_t)i);
            }
        }
        if (!long_rows.empty()) {
            uint32_t *d_list = nullptr;
            if (cudaMallocAsync((void **)&d_list, long_rows.size() * 4, up) != cudaSuccess) return "cudaMallocAsync failed";
            to_free.push_back(d_list);
            if (cudaMemcpyAsync(d_list, long_rows.data(), long_rows.size() * 4, cudaMemcpyHostToDevice, up) !=
                cudaSuccess)
                return "H2D failed";
            GeneralJob gj{J.Q, J.S, 0, r->nq, 0, ref->n, ref->n, OUT_RECT, r->d_rows};
            gj.rows = d_list;
            gj.nrows = long_rows.size();
            gj.out_len = J.out_len;
            general.push_back(gj);
        }
    }
    // Uploads go through the ingest stream, which is idle, so the worker never blocks on
    // a host copy queued behind the batch still running on this slot's stream.
    SysJob *d_jobs = nullptr;
    SysPlan plan;
    if (!entries.empty()) {
        // pieces from the cost model: a small batch gets short pieces and still covers
        // every SM
        if (cudaMallocAsync((void **)&d_jobs, jobs.size() * sizeof(SysJob), up) != cudaSuccess)
            return "cudaMallocAsync failed";
        to_free.push_back(d_jobs);
        if (cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(SysJob), cudaMemcpyHostToDevice, up) !=
            cudaSuccess)
            return "H2D failed";
        const double scale = (uint64_t)entries.size() * ref->n > kMaxChunkPairs ? kBacklogPieceScale : 1.0;
        if (build_plan(entries, rows, plan, false, up, 0, ref->mean_len, ctx->sm_count, scale) != GBD_OK)
            return gbd_last_error();
    }
    if (cudaEventRecord(uploaded, up) != cudaSuccess || cudaStreamWaitEvent(st, uploaded, 0) != cudaSuccess)
        err = "upload event failed";
    const Scoring sc{ctx->params.match, ctx->params.mismatch, ctx->params.gap, ctx->params.conversion,
                     ctx->params.gap_open};
    for (const GeneralJob &gj : general)
        if (err.empty() && run_general(gj, sc, ctx->sm_count, st) != GBD_OK) err = gbd_last_error();
    if (err.empty() && !entries.empty() &&
        run_systolic(d_jobs, plan, ctx->sm_count, st, aux, 1, ctx->params.gap_open > 0) != GBD_OK)
        err = gbd_last_error();
    plan.stream_ordered = true;
    free_plan(plan, st);
    for (void *p : to_free) cudaFreeAsync(p, st);
    return err;
}

// Next batch: chunks of the admitted requests, least remaining work first.
std::vector<Piece> next_pieces(gbd_server *srv)
{
    std::vector<Request *> cand;
    for (Request *r : srv->active)
        if (r->next_query < r->nq && r->error.empty()) cand.push_back(r);
    // Shortest remaining work first, aged: a request's remaining queries count as
    // remaining / (1 + waited / kAgeSeconds), so a large request that has waited long
    // enough is served before newer small ones instead of starving.
    const auto now = std::chrono::steady_clock::now();
    auto key = [&](const Request *r) {
        const double waited = std::chrono::duration<double>(now - r->submitted).count();
        return (double)(r->nq - r->next_query) / (1.0 + waited / kAgeSeconds);
    };
    std::sort(cand.begin(), cand.end(), [&](const Request *a, const Request *b) {
        const double ka = key(a), kb = key(b);
        return ka < kb || (ka == kb && a->ticket < b->ticket);
    });
    std::vector<Piece> out;
    const uint64_t n_ref = srv->ref->n;
    uint64_t waiting = 0;
    for (Request *r : cand) waiting += (r->nq - r->next_query) * n_ref;
    const uint64_t cap = cand.size() >= kBacklog ? kBacklogChunkPairs : kMaxChunkPairs;
    const uint64_t chunk = std::min(cap, std::max(kChunkPairs, waiting / 8));
    uint64_t room = std::max<uint64_t>(chunk / n_ref, 1);         // queries in this batch
    for (Request *r : cand) {
        if (room == 0) break;
        const uint64_t take = std::min<uint64_t>(room, r->nq - r->next_query);
        out.push_back({r, r->next_query, r->next_query + take});
        r->next_query += take;
        ++r->chunks_inflight;
        room -= take;
    }
    return out;
}

void worker_main(gbd_server *srv)
{
    cudaSetDevice(srv->ctx->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        // free device memory of finished requests (their kernels have completed)
        if (!srv->garbage.empty()) {
            std::vector<std::vector<void *>> g;
            g.swap(srv->garbage);
            lk.unlock();
            for (auto &v : g)
                for (void *p : v) cudaFreeAsync(p, srv->ingest);
            lk.lock();
        }
        // admit in arrival order while the budget allows (a request always fits when
        // nothing else is admitted: submit rejected those that never fit)
        bool progressed = false;
        while (!srv->queue.empty()) {
            Request *r = srv->queue.front();
            if (srv->used + r->footprint > srv->budget && srv->used > 0) break;
            srv->queue.pop_front();
            srv->used += r->footprint;
            r->state = REQ_ACTIVE;
            srv->active.push_back(r);
            lk.unlock();
            std::string err = admit(srv, r);
            lk.lock();
            if (!err.empty()) {
                r->error = err;
                ++r->chunks_inflight;
                chunk_finished(srv, r, err);
                srv->cv_done.notify_all();
            }
            progressed = true;
        }
        // dispatch into every free slot
        for (int s = 0; s < kSlots; ++s) {
            if (srv->slot_busy[s]) continue;
            std::vector<Piece> pieces = next_pieces(srv);
            if (pieces.empty()) break;
            srv->slot_busy[s] = true;
            lk.unlock();
            cudaStream_t st = srv->slots[s];
            std::string err;
            try {
                err = launch_batch(srv, pieces, st, &srv->slot_aux[s], srv->uploaded[s]);
            } catch (const std::exception &e) {
                err = std::string("server batch: ") + e.what();
            }
            Batch *b = new Batch{pieces, srv, s};
            cudaError_t e = cudaSuccess;
            if (err.empty()) e = cudaLaunchHostFunc(st, batch_done, b);
            lk.lock();
            if (!err.empty() || e != cudaSuccess) {
                // launch failed: drain the stream before releasing the pieces
                lk.unlock();
                cudaStreamSynchronize(st);
                lk.lock();
                const std::string msg = err.empty() ? std::string(cudaGetErrorString(e)) : err;
                for (const Piece &p : pieces) chunk_finished(srv, p.req, msg);
                srv->slot_busy[s] = false;
                delete b;
                srv->cv_done.notify_all();
            }
            progressed = true;
        }
        if (progressed) continue;
        bool busy = false;
        for (int s = 0; s < kSlots; ++s) busy = busy || srv->slot_busy[s];
        if (srv->stop && srv->active.empty() && srv->queue.empty() && !busy) break;
        srv->cv_work.wait(lk);
    }
}

}  // namespace
}  // namespace gbd

extern "C" {

int gbd_server_create(gbd_ctx *ctx, const gbd_set *ref, gbd_server **out)
{
    if (!out) return fail(GBD_EINVAL, "gbd_server_create: out is NULL");
    *out = nullptr;
    if (!ctx || !ref) return fail(GBD_EINVAL, "gbd_server_create: NULL context or reference set");
    if (ref->n == 0) return fail(GBD_EINVAL, "gbd_server_create: empty reference set");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    std::unique_ptr<gbd_server> srv(new gbd_server());
    srv->ctx = ctx;
    srv->ref = ref;
    size_t free_b = 0, total_b = 0;
    GBD_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    srv->budget = ctx->params.hbm_budget ? ctx->params.hbm_budget : (uint64_t)(0.9 * (double)free_b);
    for (int i = 0; i < kSlots; ++i) {
        GBD_CUDA_TRY(cudaStreamCreateWithFlags(&srv->slots[i], cudaStreamNonBlocking));
        GBD_CUDA_TRY(cudaStreamCreateWithFlags(&srv->slot_aux[i].aux[0], cudaStreamNonBlocking));
        GBD_CUDA_TRY(cudaEventCreateWithFlags(&srv->slot_aux[i].fork, cudaEventDisableTiming));
        GBD_CUDA_TRY(cudaEventCreateWithFlags(&srv->slot_aux[i].join[0], cudaEventDisableTiming));
    }
    GBD_CUDA_TRY(cudaStreamCreateWithFlags(&srv->ingest, cudaStreamNonBlocking));
    for (int i = 0; i < kSlots; ++i) GBD_CUDA_TRY(cudaEventCreateWithFlags(&srv->uploaded[i], cudaEventDisableTiming));
    srv->worker = std::thread(worker_main, srv.get());
    *out = srv.release();
    return GBD_OK;
}

int gbd_server_submit(gbd_server *srv, const uint8_t *seq, const uint64_t *offsets, uint64_t nq,
                      uint16_t *d_rows, uint64_t *ticket)
{
    if (!srv || !offsets || !ticket) return fail(GBD_EINVAL, "gbd_server_submit: NULL argument");
    if (nq == 0) return fail(GBD_EINVAL, "gbd_server_submit: empty request");
    if (!d_rows) return fail(GBD_EINVAL, "gbd_server_submit: d_rows is NULL");
    std::unique_ptr<Request> r(new Request());
    r->nq = nq;
    r->d_rows = d_rows;
    r->off.resize(nq + 1);
    r->len.resize(nq);
    const uint64_t base = offsets[0];
    for (uint64_t i = 0; i < nq; ++i) {
        if (offsets[i + 1] < offsets[i]) return fail(GBD_EINVAL, "gbd_server_submit: offsets decrease");
        const uint64_t L = offsets[i + 1] - offsets[i];
        if (L > 65535) return fail(GBD_EINVAL, "gbd_server_submit: read longer than 65535");
        r->len[i] = (uint16_t)L;
        r->max_len = std::max<uint32_t>(r->max_len, (uint32_t)L);
        r->off[i] = offsets[i] - base;
    }
    r->off[nq] = offsets[nq] - base;
    const uint64_t nbytes = r->off[nq];
    if (nbytes > 0 && !seq) return fail(GBD_EINVAL, "gbd_server_submit: seq is NULL");
    r->seq.assign(seq + base, seq + base + nbytes);
    for (uint64_t k = 0; k < nbytes; ++k)
        if (!valid_base(r->seq[k]))
            return fail(GBD_EINVAL, "gbd_server_submit: byte at position " + std::to_string(k) +
                                        " is not one of A, C, G, T");
    r->stride = std::max<uint32_t>(1, (r->max_len + kBasesPerWord - 1) / kBasesPerWord);
    r->footprint = nq * srv->ref->n * 2 + nbytes + (nq + 1) * 8 + nq * (r->stride * 4 + 2) + 64 * nq;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (r->footprint > srv->budget)
            return fail(GBD_EBUDGET, "gbd_server_submit: request needs " + std::to_string(r->footprint) +
                                         " bytes, above the server budget of " + std::to_string(srv->budget));
        r->ticket = srv->next_ticket++;
        r->submitted = std::chrono::steady_clock::now();
        *ticket = r->ticket;
        srv->queue.push_back(r.get());
        srv->table.emplace(r->ticket, std::move(r));
    }
    srv->cv_work.notify_all();
    return GBD_OK;
}

static int report(gbd_server *srv, uint64_t ticket, int *done)
{
    auto it = srv->table.find(ticket);
    if (it == srv->table.end()) return fail(GBD_ENOTFOUND, "gbd_server: unknown ticket " + std::to_string(ticket));
    Request *r = it->second.get();
    if (r->state == REQ_DONE || r->state == REQ_FAILED) {
        const bool ok = r->state == REQ_DONE;
        const std::string msg = r->error;
        if (r->packed) cudaEventDestroy(r->packed);
        srv->table.erase(it);                       // a finished ticket is reported once
        if (done) *done = 1;
        if (!ok) return fail(GBD_ECUDA, "gbd_server request failed: " + msg);
        return GBD_OK;
    }
    if (done) *done = 0;
    return GBD_OK;
}

int gbd_server_poll(gbd_server *srv, uint64_t ticket, int *done)
{
    if (!srv || !done) return fail(GBD_EINVAL, "gbd_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    return report(srv, ticket, done);
}

int gbd_server_wait(gbd_server *srv, uint64_t ticket)
{
    if (!srv) return fail(GBD_EINVAL, "gbd_server_wait: NULL server");
    const uint32_t tmo = srv->ctx->params.timeout_us ? srv->ctx->params.timeout_us : 60000000u;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(tmo);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        auto it = srv->table.find(ticket);
        if (it == srv->table.end()) return fail(GBD_ENOTFOUND, "gbd_server_wait: unknown ticket " + std::to_string(ticket));
        const int st = it->second->state;
        if (st == REQ_DONE || st == REQ_FAILED) return report(srv, ticket, nullptr);
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = srv->table.find(ticket);
            if (it2 != srv->table.end() && (it2->second->state == REQ_DONE || it2->second->state == REQ_FAILED))
                return report(srv, ticket, nullptr);
            return fail(GBD_ETIMEDOUT, "gbd_server_wait: ticket " + std::to_string(ticket) + " not done after " +
                                           std::to_string(tmo) + " us");
        }
    }
}

void gbd_server_destroy(gbd_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->ctx->device);
    for (auto &v : srv->garbage)
        for (void *p : v) cudaFreeAsync(p, srv->ingest);
    for (auto &kv : srv->table)
        if (kv.second->packed) cudaEventDestroy(kv.second->packed);
    for (int i = 0; i < kSlots; ++i) {
        if (srv->slots[i]) {
            cudaStreamSynchronize(srv->slots[i]);
            cudaStreamDestroy(srv->slots[i]);
        }
        StreamSet &a = srv->slot_aux[i];
        if (a.aux[0]) {
            cudaStreamSynchronize(a.aux[0]);
            cudaStreamDestroy(a.aux[0]);
        }
        if (a.fork) cudaEventDestroy(a.fork);
        if (a.join[0]) cudaEventDestroy(a.join[0]);
    }
    if (srv->ingest) {
        cudaStreamSynchronize(srv->ingest);
        cudaStreamDestroy(srv->ingest);
    }
    for (int i = 0; i < kSlots; ++i)
        if (srv->uploaded[i]) cudaEventDestroy(srv->uploaded[i]);
    delete srv;
}

}  // extern "C"
