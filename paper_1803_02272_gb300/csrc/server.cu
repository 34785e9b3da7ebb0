// Serving: a resident reference set answers query batches with distance rows (the
// rectangular form of `disseq` in section 2.2, used to place new reads into the map of
// a sample, and the read-vs-reference-database distances of the supervised annotation).
//
// Continuous batching:
//  * gbd_server_submit validates and copies a request on the host and queues it; it
//    returns at once with a ticket (or EBUDGET if the request can never fit).
//  * A worker thread admits queued requests in arrival order while their footprint (the
//    output rows plus the packed queries and the work plan) fits the HBM budget beside
//    the requests in flight.  Everything admitted in one round becomes one batch: the
//    queries of all its requests are packed on the device and scheduled as one plan --
//    one launch of the systolic kernel per rows-per-lane bucket -- with one job per
//    request, so each request's rows go to its own output buffer.
//  * Batches rotate over four compute streams, so a batch admitted while others are
//    running starts on the SMs they free.  A host callback at the end
//    of a batch's stream work marks its requests done and returns their budget.
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

enum ReqState { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> seq;        // validated bytes, offsets rebased to 0
    std::vector<uint64_t> off;
    std::vector<uint16_t> len;
    uint64_t nq = 0;
    uint32_t max_len = 0;
    uint16_t *d_rows = nullptr;
    uint64_t footprint = 0;
    int state = REQ_QUEUED;
    std::string error;
};

struct Batch {
    std::vector<Request *> reqs;
    struct gbd_server *srv = nullptr;
};

}  // namespace
}  // namespace gbd

using namespace gbd;

struct gbd_server {
    gbd_ctx *ctx = nullptr;
    const gbd_set *ref = nullptr;
    static constexpr int kStreams = 4;
    cudaStream_t streams[kStreams] = {};
    int next_stream = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> table;
    uint64_t budget = 0, used = 0, next_ticket = 1;
    int inflight = 0;
    bool stop = false;
};

namespace gbd {
namespace {

bool valid_base(uint8_t c)
{
    const uint8_t u = c | 0x20;
    return u == 'a' || u == 'c' || u == 'g' || u == 't';
}

void CUDART_CB batch_done(void *arg)
{
    // Runs on a CUDA callback thread once the batch's work on its stream has finished:
    // no CUDA calls here, only bookkeeping.
    Batch *b = static_cast<Batch *>(arg);
    gbd_server *srv = b->srv;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (Request *r : b->reqs) {
            r->state = r->error.empty() ? REQ_DONE : REQ_FAILED;
            srv->used -= r->footprint;
        }
        --srv->inflight;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
    delete b;
}

// Packs every query of the batch and launches its plan on `st`; returns a message on
// failure (the requests are then failed).
std::string launch_batch(gbd_server *srv, const std::vector<Request *> &reqs, cudaStream_t st)
{
    gbd_ctx *ctx = srv->ctx;
    const gbd_set *ref = srv->ref;
    const size_t nr = reqs.size();
    std::vector<SysJob> jobs(nr);
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    std::vector<void *> to_free;
    std::string err;
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && err.empty()) err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaSuccess;
    };
    uint64_t total_pairs = 0;
    for (size_t k = 0; k < nr && err.empty(); ++k) {
        Request *r = reqs[k];
        const uint32_t stride = std::max<uint32_t>(1, (r->max_len + kBasesPerWord - 1) / kBasesPerWord);
        uint8_t *d_seq = nullptr;
        uint64_t *d_off = nullptr;
        uint32_t *d_words = nullptr;
        uint16_t *d_len = nullptr;
        unsigned long long *d_err = nullptr;
        const size_t nbytes = std::max<size_t>(r->seq.size(), 1);
        if (!cu(cudaMallocAsync((void **)&d_seq, nbytes, st), "cudaMallocAsync")) break;
        to_free.push_back(d_seq);
        if (!cu(cudaMallocAsync((void **)&d_off, (r->nq + 1) * 8, st), "cudaMallocAsync")) break;
        to_free.push_back(d_off);
        if (!cu(cudaMallocAsync((void **)&d_words, r->nq * stride * 4, st), "cudaMallocAsync")) break;
        to_free.push_back(d_words);
        if (!cu(cudaMallocAsync((void **)&d_len, r->nq * 2, st), "cudaMallocAsync")) break;
        to_free.push_back(d_len);
        if (!cu(cudaMallocAsync((void **)&d_err, 8, st), "cudaMallocAsync")) break;
        to_free.push_back(d_err);
        if (!r->seq.empty() &&
            !cu(cudaMemcpyAsync(d_seq, r->seq.data(), r->seq.size(), cudaMemcpyHostToDevice, st), "H2D"))
            break;
        if (!cu(cudaMemcpyAsync(d_off, r->off.data(), (r->nq + 1) * 8, cudaMemcpyHostToDevice, st), "H2D")) break;
        if (!cu(launch_pack(d_seq, d_off, r->nq, stride, d_words, d_len, d_err, st), "pack")) break;
        SysJob &J = jobs[k];
        J = SysJob{};
        J.Q = {d_words, d_len, r->nq, stride};
        J.S = ref->view();
        J.sub_perm = nullptr;
        J.out = r->d_rows;
        J.ld = ref->n;
        J.row0 = 0;
        J.col0 = 0;
        J.mode = OUT_RECT;
        J.conversion = ctx->params.conversion;
        std::vector<uint32_t> long_rows;
        const gbd_params &pp = ctx->params;
        const bool systolic = pp.kernel != GBD_KERNEL_GENERAL && pp.match == 1 && pp.mismatch == -1 &&
                              pp.gap == 1;
        for (uint64_t i = 0; i < r->nq; ++i) {
            if (systolic && r->len[i] <= kSystolicMaxQuery) {
                entries.push_back({(uint32_t)k, (uint32_t)i, 0u, (uint32_t)ref->n});
                rows.push_back((uint8_t)systolic_rows(r->len[i]));
            } else {
                long_rows.push_back((uint32_t)i);
            }
        }
        total_pairs += r->nq * ref->n;
        if (!long_rows.empty()) {
            uint32_t *d_rows_list = nullptr;
            if (!cu(cudaMallocAsync((void **)&d_rows_list, long_rows.size() * 4, st), "cudaMallocAsync")) break;
            to_free.push_back(d_rows_list);
            if (!cu(cudaMemcpyAsync(d_rows_list, long_rows.data(), long_rows.size() * 4,
                                    cudaMemcpyHostToDevice, st), "H2D"))
                break;
            GeneralJob gj{J.Q, J.S, 0, r->nq, 0, ref->n, ref->n, OUT_RECT, r->d_rows};
            gj.rows = d_rows_list;
            gj.nrows = long_rows.size();
            const Scoring sc{ctx->params.match, ctx->params.mismatch, ctx->params.gap, ctx->params.conversion};
            if (run_general(gj, sc, ctx->sm_count, st) != GBD_OK) err = gbd_last_error();
        }
    }
    if (err.empty() && !entries.empty()) {
        // small batches: shorter pieces so the batch still spreads over every SM
        const uint64_t warps = (uint64_t)systolic_resident_warps(ctx->sm_count);
        uint64_t piece = total_pairs / std::max<uint64_t>(1, 4 * warps);
        piece = std::min<uint64_t>(kSystolicPiece, std::max<uint64_t>(64, piece));
        SysJob *d_jobs = nullptr;
        if (cu(cudaMallocAsync((void **)&d_jobs, nr * sizeof(SysJob), st), "cudaMallocAsync")) {
            to_free.push_back(d_jobs);
            if (cu(cudaMemcpyAsync(d_jobs, jobs.data(), nr * sizeof(SysJob), cudaMemcpyHostToDevice, st), "H2D")) {
                SysPlan plan;
                if (build_plan(entries, rows, plan, false, st, (uint32_t)piece) != GBD_OK ||
                    run_systolic(d_jobs, plan, ctx->sm_count, st) != GBD_OK)
                    err = gbd_last_error();
                free_plan(plan, st);
            }
        }
    }
    for (void *p : to_free) cudaFreeAsync(p, st);
    return err;
}

void worker_main(gbd_server *srv)
{
    cudaSetDevice(srv->ctx->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        // admit in arrival order while the budget allows (a request always fits when
        // nothing else is in flight: submit rejected those that never fit)
        std::vector<Request *> batch;
        while (!srv->queue.empty()) {
            Request *r = srv->queue.front();
            if (srv->used + r->footprint > srv->budget && (srv->used > 0 || !batch.empty())) break;
            srv->queue.pop_front();
            srv->used += r->footprint;
            r->state = REQ_RUNNING;
            batch.push_back(r);
        }
        if (!batch.empty()) {
            const int si = srv->next_stream;
            srv->next_stream = (si + 1) % gbd_server::kStreams;
            ++srv->inflight;
            lk.unlock();
            cudaStream_t st = srv->streams[si];
            std::string err;
            try {
                err = launch_batch(srv, batch, st);
            } catch (const std::exception &e) {
                err = std::string("server batch: ") + e.what();
            }
            Batch *b = new Batch{batch, srv};
            if (!err.empty()) {
                // published as failed by batch_done, after the stream work has drained
                lk.lock();
                for (Request *r : batch) r->error = err;
                lk.unlock();
            }
            cudaError_t e = cudaLaunchHostFunc(st, batch_done, b);
            lk.lock();
            if (e != cudaSuccess) {
                for (Request *r : batch) {
                    r->state = REQ_FAILED;
                    if (r->error.empty()) r->error = cudaGetErrorString(e);
                    srv->used -= r->footprint;
                }
                --srv->inflight;
                delete b;
                srv->cv_done.notify_all();
            }
            continue;
        }
        if (srv->stop && srv->inflight == 0) break;
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
    for (int i = 0; i < gbd_server::kStreams; ++i)
        GBD_CUDA_TRY(cudaStreamCreateWithFlags(&srv->streams[i], cudaStreamNonBlocking));
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
    const uint32_t stride = std::max<uint32_t>(1, (r->max_len + kBasesPerWord - 1) / kBasesPerWord);
    r->footprint = nq * srv->ref->n * 2 + nbytes + (nq + 1) * 8 + nq * (stride * 4 + 2) + 64 * nq;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (r->footprint > srv->budget)
            return fail(GBD_EBUDGET, "gbd_server_submit: request needs " + std::to_string(r->footprint) +
                                         " bytes, above the server budget of " + std::to_string(srv->budget));
        r->ticket = srv->next_ticket++;
        *ticket = r->ticket;
        srv->queue.push_back(r.get());
        srv->table.emplace(r->ticket, std::move(r));
    }
    srv->cv_work.notify_all();
    return GBD_OK;
}

static int report(gbd_server *srv, std::unique_lock<std::mutex> &lk, uint64_t ticket, int *done)
{
    auto it = srv->table.find(ticket);
    if (it == srv->table.end()) return fail(GBD_ENOTFOUND, "gbd_server: unknown ticket " + std::to_string(ticket));
    Request *r = it->second.get();
    if (r->state == REQ_DONE || r->state == REQ_FAILED) {
        const bool ok = r->state == REQ_DONE;
        const std::string msg = r->error;
        srv->table.erase(it);                       // a finished ticket is reported once
        if (done) *done = 1;
        if (!ok) return fail(GBD_ECUDA, "gbd_server request failed: " + msg);
        return GBD_OK;
    }
    if (done) *done = 0;
    (void)lk;
    return GBD_OK;
}

int gbd_server_poll(gbd_server *srv, uint64_t ticket, int *done)
{
    if (!srv || !done) return fail(GBD_EINVAL, "gbd_server_poll: NULL argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    return report(srv, lk, ticket, done);
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
        if (st == REQ_DONE || st == REQ_FAILED) return report(srv, lk, ticket, nullptr);
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = srv->table.find(ticket);
            if (it2 != srv->table.end() && (it2->second->state == REQ_DONE || it2->second->state == REQ_FAILED))
                return report(srv, lk, ticket, nullptr);
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
    for (int i = 0; i < gbd_server::kStreams; ++i) {
        if (srv->streams[i]) {
            cudaStreamSynchronize(srv->streams[i]);
            cudaStreamDestroy(srv->streams[i]);
        }
    }
    delete srv;
}

}  // extern "C"
