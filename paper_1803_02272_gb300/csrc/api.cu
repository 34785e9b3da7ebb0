// C ABI of the library: contexts, packed read sets, and the all-pairs / rectangle /
// batched entry points.  Serving lives in server.cu.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>

#include "gbd_internal.cuh"
#include "sw_systolic.cuh"

namespace gbd {

static thread_local std::string t_last_error;
static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_set_ids{0};

void note_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const std::string &msg) { t_last_error = msg; }

int fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    set_error(m);
    return GBD_ECUDA;
}

static bool is_device_pointer(const void *p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

Scoring scoring_of(const gbd_ctx *ctx)
{
    return {ctx->params.match, ctx->params.mismatch, ctx->params.gap, ctx->params.conversion,
            ctx->params.gap_open};
}

// The systolic kernel is specialised to match +1, mismatch -1, gap extension 1; it takes
// a gap opening penalty up to kSystolicMaxGapOpen (0 = linear gaps).
static bool default_scores(const gbd_params &p)
{
    return p.match == 1 && p.mismatch == -1 && p.gap == 1 && p.gap_open >= 0 &&
           p.gap_open <= kSystolicMaxGapOpen;
}

static bool use_systolic(const gbd_ctx *ctx)
{
    return ctx->params.kernel != GBD_KERNEL_GENERAL && default_scores(ctx->params);
}

// Systolic entries and long-read rows of a set's triangle (built once per set).
static int build_tri_schedule(gbd_set *set, cudaStream_t st)
{
    TriSchedule &sc = set->sched;
    if (sc.built) return GBD_OK;
    const uint64_t n = set->n;
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    std::vector<uint32_t> long_rows;
    std::vector<uint64_t> long_prefix(1, 0);
    for (uint64_t i = 0; i + 1 < n; ++i) {
        if (set->h_len[i] <= kSystolicMaxQuery) {
            entries.push_back({0u, (uint32_t)i, (uint32_t)(i + 1), (uint32_t)(n - 1 - i)});
            rows.push_back((uint8_t)systolic_rows(set->h_len[i]));
        } else {
            long_rows.push_back((uint32_t)i);
            long_prefix.push_back(long_prefix.back() + (n - 1 - i));
        }
    }
    sc.nlong = long_rows.size();
    if (sc.nlong) {
        GBD_CUDA_TRY(cudaMalloc((void **)&sc.d_long_rows, sc.nlong * sizeof(uint32_t)));
        GBD_CUDA_TRY(cudaMalloc((void **)&sc.d_long_prefix, (sc.nlong + 1) * sizeof(uint64_t)));
        GBD_CUDA_TRY(cudaMemcpyAsync(sc.d_long_rows, long_rows.data(), sc.nlong * sizeof(uint32_t),
                                     cudaMemcpyHostToDevice, st));
        GBD_CUDA_TRY(cudaMemcpyAsync(sc.d_long_prefix, long_prefix.data(),
                                     (sc.nlong + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    }
    int rc = build_plan(entries, rows, sc.plan, true, st, 0, set->mean_len, set->ctx->sm_count);
    if (rc != GBD_OK) return rc;
    GBD_CUDA_TRY(cudaStreamSynchronize(st));
    sc.long_units = long_prefix.back();
    sc.built = true;
    return GBD_OK;
}

// Rows of the triangle whose read is too long to be a systolic query.
static int long_rows_general(gbd_ctx *ctx, const gbd_set *set, uint16_t *d_tri, cudaStream_t st)
{
    const TriSchedule &sc = set->sched;
    if (sc.nlong == 0 || sc.long_units == 0) return GBD_OK;
    GeneralJob gj{set->view(), set->view(), 0, set->n, 0, set->n, 0, OUT_TRI_ROWS, d_tri};
    gj.rows = sc.d_long_rows;
    gj.nrows = sc.nlong;
    gj.row_prefix = sc.d_long_prefix;
    gj.units_total = sc.long_units;
    gj.out_len = out_extent(ctx, set->n * (set->n - 1) / 2);
    return run_general(gj, scoring_of(ctx), ctx->sm_count, st);
}

// Copies a host array into stream-ordered device memory freed by the caller.
template <typename T>
static int upload(const T *h, size_t count, T **d, cudaStream_t st)
{
    *d = nullptr;
    if (count == 0) return GBD_OK;
    GBD_CUDA_TRY(cudaMallocAsync((void **)d, count * sizeof(T), st));
    GBD_CUDA_TRY(cudaMemcpyAsync(*d, h, count * sizeof(T), cudaMemcpyHostToDevice, st));
    return GBD_OK;
}

// Triangle of one set through the systolic kernel (+ the general kernel for the pairs
// of reads longer than the systolic query limit).
static int all_pairs_systolic(gbd_ctx *ctx, gbd_set *set, uint16_t *d_tri, cudaStream_t st)
{
    int rc = build_tri_schedule(set, st);
    if (rc != GBD_OK) return rc;
    const TriSchedule &sc = set->sched;
    SysJob job{};
    job.Q = job.S = set->view();
    job.sub_perm = nullptr;
    job.out = d_tri;
    job.n = set->n;
    job.mode = OUT_TRI;
    job.conversion = ctx->params.conversion;
    job.gap_open = ctx->params.gap_open;
    job.out_len = out_extent(ctx, set->n * (set->n - 1) / 2);
    SysJob *d_job = nullptr;
    if ((rc = upload(&job, 1, &d_job, st)) != GBD_OK) return rc;
    rc = run_systolic(d_job, sc.plan, ctx->sm_count, st, &ctx->streams, kDefaultAuxStreams, job.gap_open > 0);
    cudaFreeAsync(d_job, st);
    if (rc != GBD_OK) return rc;
    return long_rows_general(ctx, set, d_tri, st);
}

// All pairs of one set into the dense triangle.
static int all_pairs_impl(gbd_ctx *ctx, const gbd_set *set, uint16_t *d_tri, cudaStream_t st)
{
    if (use_systolic(ctx)) return all_pairs_systolic(ctx, const_cast<gbd_set *>(set), d_tri, st);
    const uint64_t n = set->n;
    GeneralJob job{set->view(), set->view(), 0, n, 0, n, 0, OUT_TRI, d_tri};
    job.out_len = out_extent(ctx, n * (n - 1) / 2);
    return run_general(job, scoring_of(ctx), ctx->sm_count, st);
}

// Rectangle A[a0,a1) x B[b0,b1) into d_out (leading dimension ld).
static int tile_impl(gbd_ctx *ctx, const gbd_set *A, uint64_t a0, uint64_t a1, const gbd_set *B,
                     uint64_t b0, uint64_t b1, uint16_t *d_out, uint64_t ld, cudaStream_t st)
{
    const uint64_t rect_len = out_extent(ctx, (a1 - a0 - 1) * ld + (b1 - b0));
    if (!use_systolic(ctx)) {
        GeneralJob job{A->view(), B->view(), a0, a1, b0, b1, ld, OUT_RECT, d_out};
        job.out_len = rect_len;
        return run_general(job, scoring_of(ctx), ctx->sm_count, st);
    }
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    std::vector<uint32_t> long_rows;
    for (uint64_t r = a0; r < a1; ++r) {
        if (A->h_len[r] <= kSystolicMaxQuery) {
            entries.push_back({0u, (uint32_t)r, (uint32_t)b0, (uint32_t)(b1 - b0)});
            rows.push_back((uint8_t)systolic_rows(A->h_len[r]));
        } else {
            long_rows.push_back((uint32_t)r);
        }
    }
    int rc = GBD_OK;
    if (!entries.empty()) {
        SysJob job{};
        job.Q = A->view();
        job.S = B->view();
        job.sub_perm = nullptr;
        job.out = d_out;
        job.ld = ld;
        job.row0 = a0;
        job.col0 = b0;
        job.mode = OUT_RECT;
        job.conversion = ctx->params.conversion;
        job.gap_open = ctx->params.gap_open;
        job.out_len = rect_len;
        SysJob *d_job = nullptr;
        SysPlan plan;
        if ((rc = upload(&job, 1, &d_job, st)) != GBD_OK) return rc;
        if ((rc = build_plan(entries, rows, plan, false, st, 0, B->mean_len, ctx->sm_count)) != GBD_OK)
            return rc;
        rc = run_systolic(d_job, plan, ctx->sm_count, st, &ctx->streams, kDefaultAuxStreams, job.gap_open > 0);
        cudaFreeAsync(d_job, st);
        free_plan(plan, st);
        if (rc != GBD_OK) return rc;
    }
    if (!long_rows.empty()) {
        uint32_t *d_rows = nullptr;
        if ((rc = upload(long_rows.data(), long_rows.size(), &d_rows, st)) != GBD_OK) return rc;
        GeneralJob gj{A->view(), B->view(), a0, a1, b0, b1, ld, OUT_RECT, d_out};
        gj.rows = d_rows;
        gj.nrows = long_rows.size();
        gj.out_len = rect_len;
        rc = run_general(gj, scoring_of(ctx), ctx->sm_count, st);
        cudaFreeAsync(d_rows, st);
    }
    return rc;
}

// Distances of the rows [a0, a1) of a set against the reads after each row: row r's
// pairs (r, j), j > r, go to out[(r - a0) * ld + (j - a0 - 1)] (the entries before
// column r + 1 - a0 - 1 of each row are not written, or hold pairs with j <= r).
static int band_impl(gbd_ctx *ctx, const gbd_set *set, uint64_t a0, uint64_t a1, uint16_t *out, uint64_t ld,
                     cudaStream_t st)
{
    const uint64_t n = set->n;
    if (a1 <= a0 || a0 + 1 >= n) return GBD_OK;
    const uint64_t band_len = out_extent(ctx, (a1 - a0) * ld);
    if (!use_systolic(ctx)) {
        GeneralJob job{set->view(), set->view(), a0, a1, a0 + 1, n, ld, OUT_RECT, out};
        job.out_len = band_len;
        return run_general(job, scoring_of(ctx), ctx->sm_count, st);
    }
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    std::vector<uint32_t> long_rows;
    for (uint64_t r = a0; r < a1 && r + 1 < n; ++r) {
        if (set->h_len[r] <= kSystolicMaxQuery) {
            entries.push_back({0u, (uint32_t)r, (uint32_t)(r + 1), (uint32_t)(n - r - 1)});
            rows.push_back((uint8_t)systolic_rows(set->h_len[r]));
        } else {
            long_rows.push_back((uint32_t)r);
        }
    }
    int rc = GBD_OK;
    if (!entries.empty()) {
        SysJob job{};
        job.Q = job.S = set->view();
        job.sub_perm = nullptr;
        job.out = out;
        job.ld = ld;
        job.row0 = a0;
        job.col0 = a0 + 1;
        job.mode = OUT_RECT;
        job.conversion = ctx->params.conversion;
        job.gap_open = ctx->params.gap_open;
        job.out_len = band_len;
        SysJob *d_job = nullptr;
        SysPlan plan;
        if ((rc = upload(&job, 1, &d_job, st)) != GBD_OK) return rc;
        if ((rc = build_plan(entries, rows, plan, false, st, 0, set->mean_len, ctx->sm_count)) != GBD_OK)
            return rc;
        rc = run_systolic(d_job, plan, ctx->sm_count, st, &ctx->streams, kDefaultAuxStreams, job.gap_open > 0);
        cudaFreeAsync(d_job, st);
        free_plan(plan, st);
        if (rc != GBD_OK) return rc;
    }
    if (!long_rows.empty()) {
        // whole rows of the rectangle [a0, a1) x [a0 + 1, n): the pairs with j <= r land in
        // the row's unused entries
        uint32_t *d_rows = nullptr;
        if ((rc = upload(long_rows.data(), long_rows.size(), &d_rows, st)) != GBD_OK) return rc;
        GeneralJob gj{set->view(), set->view(), a0, a1, a0 + 1, n, ld, OUT_RECT, out};
        gj.rows = d_rows;
        gj.nrows = long_rows.size();
        gj.out_len = band_len;
        rc = run_general(gj, scoring_of(ctx), ctx->sm_count, st);
        cudaFreeAsync(d_rows, st);
    }
    return rc;
}

// Listed triangle rows of a set through the general kernel, into `out`, which holds the
// triangle's entries from index `base` on (len entries).
static int tri_rows_general(gbd_ctx *ctx, const gbd_set *set, const std::vector<uint32_t> &rows_h,
                            uint16_t *out, uint64_t base, uint64_t len, cudaStream_t st)
{
    const uint64_t n = set->n;
    std::vector<uint64_t> prefix(1, 0);
    for (uint32_t r : rows_h) prefix.push_back(prefix.back() + (n - 1 - r));
    if (prefix.back() == 0) return GBD_OK;
    uint32_t *d_rows = nullptr;
    uint64_t *d_prefix = nullptr;
    int rc = upload(rows_h.data(), rows_h.size(), &d_rows, st);
    if (rc == GBD_OK) rc = upload(prefix.data(), prefix.size(), &d_prefix, st);
    if (rc == GBD_OK) {
        GeneralJob gj{set->view(), set->view(), 0, n, 0, n, 0, OUT_TRI_ROWS, out};
        gj.rows = d_rows;
        gj.nrows = rows_h.size();
        gj.row_prefix = d_prefix;
        gj.units_total = prefix.back();
        gj.out_base = base;
        gj.out_len = len;
        rc = run_general(gj, scoring_of(ctx), ctx->sm_count, st);
    }
    if (d_rows) cudaFreeAsync(d_rows, st);
    if (d_prefix) cudaFreeAsync(d_prefix, st);
    return rc;
}

// Rows [a0, a1) of a set's triangle into `out`: the band is the contiguous run of the
// row-major triangle from k(a0, a0 + 1) on, and `out` holds just that run.
static int tri_band_impl(gbd_ctx *ctx, const gbd_set *set, uint64_t a0, uint64_t a1, uint16_t *out, cudaStream_t st)
{
    const uint64_t n = set->n;
    const uint64_t base = a0 * n - a0 * (a0 + 1) / 2;
    const uint64_t len = out_extent(ctx, a1 * n - a1 * (a1 + 1) / 2 - base);
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    std::vector<uint32_t> general_rows;
    const bool systolic = use_systolic(ctx);
    for (uint64_t r = a0; r < a1 && r + 1 < n; ++r) {
        if (systolic && set->h_len[r] <= kSystolicMaxQuery) {
            entries.push_back({0u, (uint32_t)r, (uint32_t)(r + 1), (uint32_t)(n - 1 - r)});
            rows.push_back((uint8_t)systolic_rows(set->h_len[r]));
        } else {
            general_rows.push_back((uint32_t)r);
        }
    }
    int rc = GBD_OK;
    if (!entries.empty()) {
        SysJob job{};
        job.Q = job.S = set->view();
        job.sub_perm = nullptr;
        job.out = out;
        job.n = n;
        job.mode = OUT_TRI;
        job.conversion = ctx->params.conversion;
        job.gap_open = ctx->params.gap_open;
        job.out_len = len;
        job.out_base = base;
        SysJob *d_job = nullptr;
        SysPlan plan;
        if ((rc = upload(&job, 1, &d_job, st)) != GBD_OK) return rc;
        rc = build_plan(entries, rows, plan, false, st, 0, set->mean_len, ctx->sm_count);
        if (rc == GBD_OK)
            rc = run_systolic(d_job, plan, ctx->sm_count, st, &ctx->streams, kDefaultAuxStreams, job.gap_open > 0);
        cudaFreeAsync(d_job, st);
        free_plan(plan, st);
        if (rc != GBD_OK) return rc;
    }
    if (!general_rows.empty()) rc = tri_rows_general(ctx, set, general_rows, out, base, len, st);
    return rc;
}

// Default entries of the band scratch of gbd_threshold_components without a triangle (512 MB).
constexpr uint64_t kBandEntries = 1ull << 28;

static int check_threshold(const gbd_threshold *th)
{
    if (!th) return fail(GBD_EINVAL, "NULL threshold");
    if (th->den == 0) return fail(GBD_EINVAL, "threshold den must be positive");
    return GBD_OK;
}


// Last captured batch: its inputs, persistent job table and plan, and the graph.
// Online autotuner of the batched launch.  A candidate sets the shape of the launch group:
// the work-unit size (the cost model's piece times `scale`) and the number of streams the
// per-bucket launches alternate over (1 + naux).  Coordinate descent over the first calls
// with a new list of samples, each timed with events: scales 1, 0.5 and 2 with two
// streams, then the best scale with one and with three streams; the next call keeps the
// fastest candidate.
struct TuneCand {
    double scale;
    int naux;
};
constexpr int kTrials = 5;
constexpr TuneCand kFirstCands[3] = {{1.0, 1}, {0.5, 1}, {2.0, 1}};

struct BatchGraph {
    std::vector<uint64_t> ids;
    std::vector<uint16_t *> outs;
    int conversion = 0;
    SysJob *d_jobs = nullptr;
    SysPlan plan;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;
    // inputs of the plan, kept to rebuild it with another candidate
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    double mean_len = 0.0;
    // autotuner state
    TuneCand cands[kTrials] = {kFirstCands[0], kFirstCands[1], kFirstCands[2], {1.0, 0}, {1.0, 2}};
    int trial = 0;                    // candidate being timed; kTrials = tuning finished
    bool timing = false;              // events t0/t1 bracket the last launch
    double trial_ms[kTrials] = {0, 0, 0, 0, 0};
    int current = 0;                  // candidate of the recorded graph
    int chosen = -1;                  // fastest candidate, once tuning has finished
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    int gap_open = 0;
    bool matches(const gbd_set *const *samples, uint64_t ns, uint16_t *const *d_tris, int conv, int go) const
    {
        if (ids.size() != ns || conversion != conv || gap_open != go) return false;
        for (uint64_t s = 0; s < ns; ++s)
            if (ids[s] != samples[s]->id || outs[s] != d_tris[s]) return false;
        return true;
    }
};

void free_batch_cache(gbd_ctx *ctx)
{
    BatchGraph *bg = static_cast<BatchGraph *>(ctx->batch_cache);
    if (!bg) return;
    if (bg->exec) cudaGraphExecDestroy(bg->exec);
    if (bg->graph) cudaGraphDestroy(bg->graph);
    if (bg->d_jobs) cudaFree(bg->d_jobs);
    free_plan(bg->plan, nullptr);
    if (bg->t0) cudaEventDestroy(bg->t0);
    if (bg->t1) cudaEventDestroy(bg->t1);
    delete bg;
    ctx->batch_cache = nullptr;
}

// Builds the batch's job table and plan (persistent) and records its launch group on the
// context's capture stream.
static int record_batch_graph(gbd_ctx *ctx, BatchGraph *bg, const gbd_set *const *samples, uint64_t ns,
                              uint16_t *const *d_tris, int cand);

static int capture_batch(gbd_ctx *ctx, BatchGraph *bg, const gbd_set *const *samples, uint64_t ns,
                         uint16_t *const *d_tris)
{
    std::vector<SysJob> jobs(ns);
    std::vector<SysEntry> entries;
    std::vector<uint8_t> rows;
    double len_sum = 0.0, n_sum = 0.0;
    for (uint64_t s = 0; s < ns; ++s) {
        const gbd_set *set = samples[s];
        bg->ids.push_back(set->id);
        bg->outs.push_back(d_tris[s]);
        SysJob &job = jobs[s];
        job = SysJob{};
        job.Q = job.S = set->view();
        job.sub_perm = nullptr;
        job.out = d_tris[s];
        job.n = set->n;
        job.mode = OUT_TRI;
        job.conversion = ctx->params.conversion;
        job.gap_open = ctx->params.gap_open;
        job.out_len = out_extent(ctx, set->n < 2 ? 0 : set->n * (set->n - 1) / 2);
        for (uint64_t i = 0; i + 1 < set->n; ++i) {
            if (set->h_len[i] > kSystolicMaxQuery) continue;
            entries.push_back({(uint32_t)s, (uint32_t)i, (uint32_t)(i + 1), (uint32_t)(set->n - 1 - i)});
            rows.push_back((uint8_t)systolic_rows(set->h_len[i]));
        }
        len_sum += set->mean_len * (double)set->n;
        n_sum += (double)set->n;
    }
    bg->conversion = ctx->params.conversion;
    bg->gap_open = ctx->params.gap_open;
    {
        std::vector<size_t> order(entries.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](size_t x, size_t y) { return entries[x].nsub > entries[y].nsub; });
        std::vector<SysEntry> e2(entries.size());
        std::vector<uint8_t> r2(entries.size());
        for (size_t i = 0; i < order.size(); ++i) { e2[i] = entries[order[i]]; r2[i] = rows[order[i]]; }
        entries.swap(e2);
        rows.swap(r2);
    }
    if (ns > 0) {
        GBD_CUDA_TRY(cudaMalloc((void **)&bg->d_jobs, ns * sizeof(SysJob)));
        GBD_CUDA_TRY(cudaMemcpy(bg->d_jobs, jobs.data(), ns * sizeof(SysJob), cudaMemcpyHostToDevice));
    }
    bg->mean_len = n_sum > 0 ? len_sum / n_sum : 0.0;
    bg->entries.swap(entries);
    bg->rows.swap(rows);
    GBD_CUDA_TRY(cudaEventCreate(&bg->t0));
    GBD_CUDA_TRY(cudaEventCreate(&bg->t1));
    return record_batch_graph(ctx, bg, samples, ns, d_tris, 0);
}

// (Re)builds the plan with candidate `cand`'s piece scale and records the launch group,
// over its number of streams, as a graph.  The previous graph, if any, must have finished.
static int record_batch_graph(gbd_ctx *ctx, BatchGraph *bg, const gbd_set *const *samples, uint64_t ns,
                              uint16_t *const *d_tris, int cand)
{
    cudaStream_t cap = ctx->capture;
    if (bg->exec) { cudaGraphExecDestroy(bg->exec); bg->exec = nullptr; }
    if (bg->graph) { cudaGraphDestroy(bg->graph); bg->graph = nullptr; }
    free_plan(bg->plan, nullptr);
    bg->current = cand;
    const TuneCand &c = bg->cands[cand];
    int rc = build_plan(bg->entries, bg->rows, bg->plan, true, cap, 0, bg->mean_len, ctx->sm_count, c.scale);
    if (rc != GBD_OK) return rc;
    const uint64_t launches0 = gbd_kernel_launches();
    GBD_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    rc = run_systolic(bg->d_jobs, bg->plan, ctx->sm_count, cap, &ctx->streams, c.naux, ctx->params.gap_open > 0);
    for (uint64_t s = 0; s < ns && rc == GBD_OK; ++s) rc = long_rows_general(ctx, samples[s], d_tris[s], cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (rc != GBD_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    bg->graph = g;
    GBD_CUDA_TRY(cudaGraphInstantiate(&bg->exec, g, 0));
    // the capture counted the kernels it recorded; every replay runs them again
    bg->kernels = gbd_kernel_launches() - launches0;
    return GBD_OK;
}

}  // namespace gbd

using namespace gbd;

extern "C" {

const char *gbd_last_error(void) { return t_last_error.c_str(); }

void gbd_default_params(gbd_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->match = 1;
    p->mismatch = -1;
    p->gap = 1;
    p->conversion = GBD_CONV_MAX;
    p->kernel = GBD_KERNEL_AUTO;
    p->hbm_budget = 0;
    p->timeout_us = 0;
}

uint64_t gbd_params_size(void) { return sizeof(gbd_params); }

int gbd_create(gbd_ctx **out, int device, const gbd_params *p)
{
    if (!out) return fail(GBD_EINVAL, "gbd_create: out is NULL");
    *out = nullptr;
    gbd_params prm;
    gbd_default_params(&prm);
    if (p) prm = *p;
    if (prm.gap < 0) return fail(GBD_EINVAL, "gbd_create: gap penalty must be >= 0");
    if (prm.gap_open < 0) return fail(GBD_EINVAL, "gbd_create: gap opening penalty must be >= 0");
    if (prm.conversion < GBD_CONV_MAX || prm.conversion > GBD_CONV_NORM)
        return fail(GBD_EINVAL, "gbd_create: unknown conversion");
    if (prm.kernel < GBD_KERNEL_AUTO || prm.kernel > GBD_KERNEL_SYSTOLIC)
        return fail(GBD_EINVAL, "gbd_create: unknown kernel choice");
    if (prm.kernel == GBD_KERNEL_SYSTOLIC && !default_scores(prm))
        return fail(GBD_EINVAL, "gbd_create: the systolic kernel supports match +1, mismatch -1, gap "
                                "extension 1 and a gap opening penalty up to 1000 only");
    int ndev = 0;
    GBD_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(GBD_EINVAL, "gbd_create: no such device");
    GBD_CUDA_TRY(cudaSetDevice(device));
    gbd_ctx *ctx = new (std::nothrow) gbd_ctx();
    if (!ctx) return fail(GBD_ENOMEM, "gbd_create: out of host memory");
    ctx->device = device;
    ctx->params = prm;
    cudaError_t e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    for (int k = 0; k < StreamSet::kMaxAux && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&ctx->streams.aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->streams.join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->streams.fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_fail(e, "gbd_create");
    }
    // Scratch comes from the device's default stream-ordered pool; with its default
    // release threshold (0) every synchronisation hands the memory back and the next call
    // maps it again (milliseconds for the 512 MB edge list).  Keep up to 4 GiB reserved
    // (only ever raised, never lowered).
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = 0;
        const uint64_t want = 4ull << 30;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess && keep < want)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, (void *)&want);
    }
    cudaGetLastError();
    *out = ctx;
    return GBD_OK;
}

void gbd_destroy(gbd_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_batch_cache(ctx);
    free_mds_cache(ctx);
    for (cudaStream_t st : {ctx->streams.aux[0], ctx->streams.aux[1], ctx->capture}) {
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    }
    if (ctx->streams.fork) cudaEventDestroy(ctx->streams.fork);
    for (cudaEvent_t ev : ctx->streams.join)
        if (ev) cudaEventDestroy(ev);
    delete ctx;
}

int gbd_trim(gbd_ctx *ctx)
{
    if (!ctx) return fail(GBD_EINVAL, "gbd_trim: NULL context");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    GBD_CUDA_TRY(cudaDeviceSynchronize());
    free_batch_cache(ctx);
    free_mds_cache(ctx);
    return GBD_OK;
}

int gbd_load_reads(gbd_ctx *ctx, const uint8_t *seq, const uint64_t *offsets, uint64_t n,
                   gbd_set **out, void *stream)
{
    if (!ctx || !out) return fail(GBD_EINVAL, "gbd_load_reads: NULL context or output");
    *out = nullptr;
    if (!offsets) return fail(GBD_EINVAL, "gbd_load_reads: offsets is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    const bool dev_off = is_device_pointer(offsets);
    std::vector<uint64_t> hoff(n + 1);
    if (dev_off) {
        GBD_CUDA_TRY(cudaMemcpyAsync(hoff.data(), offsets, (n + 1) * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, st));
        GBD_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        std::memcpy(hoff.data(), offsets, (n + 1) * sizeof(uint64_t));
    }
    gbd_set *set = new (std::nothrow) gbd_set();
    if (!set) return fail(GBD_ENOMEM, "gbd_load_reads: out of host memory");
    set->ctx = ctx;
    set->device = ctx->device;
    set->n = n;
    set->h_len.resize(n);
    uint32_t max_len = 0;
    double sum = 0.0, sumsq = 0.0;
    for (uint64_t r = 0; r < n; ++r) {
        if (hoff[r + 1] < hoff[r]) {
            delete set;
            return fail(GBD_EINVAL, "gbd_load_reads: offsets decrease at read " + std::to_string(r));
        }
        const uint64_t L = hoff[r + 1] - hoff[r];
        if (L > 65535) {
            delete set;
            return fail(GBD_EINVAL, "gbd_load_reads: read " + std::to_string(r) + " is longer than 65535");
        }
        set->h_len[r] = (uint16_t)L;
        max_len = std::max<uint32_t>(max_len, (uint32_t)L);
        sum += (double)L;
        sumsq += (double)L * (double)L;
    }
    set->max_len = max_len;
    set->stride = std::max<uint32_t>(1, (max_len + kBasesPerWord - 1) / kBasesPerWord);
    set->pair_cells = (sum * sum - sumsq) * 0.5;
    set->mean_len = n ? sum / (double)n : 0.0;
    set->id = g_set_ids.fetch_add(1, std::memory_order_relaxed) + 1;
    const uint64_t nbytes = hoff[n] - hoff[0];
    if (nbytes > 0 && !seq) {
        delete set;
        return fail(GBD_EINVAL, "gbd_load_reads: seq is NULL");
    }
    if (n == 0) {
        *out = set;
        return GBD_OK;
    }

    cudaError_t e = cudaSuccess;
    uint8_t *d_seq_tmp = nullptr;
    uint64_t *d_off_tmp = nullptr;
    unsigned long long *d_err = nullptr;
    unsigned long long h_err = ~0ull;
    const uint8_t *d_seq = seq;
    const uint64_t *d_off = offsets;
    auto cleanup = [&]() {
        if (d_seq_tmp) cudaFreeAsync(d_seq_tmp, st);
        if (d_off_tmp) cudaFreeAsync(d_off_tmp, st);
        if (d_err) cudaFreeAsync(d_err, st);
    };
    do {
        if ((e = cudaMalloc((void **)&set->d_words, n * set->stride * sizeof(uint32_t))) != cudaSuccess) break;
        if ((e = cudaMalloc((void **)&set->d_len, n * sizeof(uint16_t))) != cudaSuccess) break;
        if ((e = cudaMallocAsync((void **)&d_err, sizeof(unsigned long long), st)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(d_err, 0xff, sizeof(unsigned long long), st)) != cudaSuccess) break;
        if (!dev_off) {
            if ((e = cudaMallocAsync((void **)&d_off_tmp, (n + 1) * sizeof(uint64_t), st)) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(d_off_tmp, hoff.data(), (n + 1) * sizeof(uint64_t),
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
            d_off = d_off_tmp;
        }
        if (nbytes > 0 && !is_device_pointer(seq)) {
            if ((e = cudaMallocAsync((void **)&d_seq_tmp, nbytes, st)) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(d_seq_tmp, seq + hoff[0], nbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
            // the kernel indexes seq with absolute offsets: shift the base pointer back
            d_seq = d_seq_tmp - hoff[0];
        }
        if ((e = launch_pack(d_seq, d_off, n, set->stride, set->d_words, set->d_len, d_err, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&h_err, d_err, sizeof h_err, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        e = cudaStreamSynchronize(st);
    } while (0);
    cleanup();
    if (e != cudaSuccess) {
        gbd_free_set(set);
        return cuda_fail(e, "gbd_load_reads");
    }
    if (h_err != ~0ull) {
        gbd_free_set(set);
        return fail(GBD_EINVAL, "gbd_load_reads: byte at position " + std::to_string(h_err) +
                                    " is not one of A, C, G, T");
    }
    *out = set;
    return GBD_OK;
}

void gbd_free_set(gbd_set *set)
{
    if (!set) return;
    cudaSetDevice(set->device);
    if (set->d_words) cudaFree(set->d_words);
    if (set->d_len) cudaFree(set->d_len);
    if (set->sched.d_long_rows) cudaFree(set->sched.d_long_rows);
    if (set->sched.d_long_prefix) cudaFree(set->sched.d_long_prefix);
    gbd::free_plan(set->sched.plan, nullptr);
    delete set;
}

uint64_t gbd_set_size(const gbd_set *set) { return set ? set->n : 0; }
uint32_t gbd_set_max_len(const gbd_set *set) { return set ? set->max_len : 0; }
double gbd_set_pair_cells(const gbd_set *set) { return set ? set->pair_cells : 0.0; }

int gbd_all_pairs(gbd_ctx *ctx, const gbd_set *set, uint16_t *d_tri, uint64_t tri_len, void *stream)
{
    if (!ctx || !set) return fail(GBD_EINVAL, "gbd_all_pairs: NULL context or set");
    const uint64_t n = set->n;
    const uint64_t need = n < 2 ? 0 : n * (n - 1) / 2;
    if (tri_len != need)
        return fail(GBD_EINVAL, "gbd_all_pairs: tri_len is " + std::to_string(tri_len) +
                                    ", expected n(n-1)/2 = " + std::to_string(need));
    if (need == 0) return GBD_OK;
    if (!d_tri) return fail(GBD_EINVAL, "gbd_all_pairs: d_tri is NULL");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    return all_pairs_impl(ctx, set, d_tri, (cudaStream_t)stream);
}

int gbd_all_pairs_to_host(gbd_ctx *ctx, const gbd_set *set, uint16_t *h_tri, uint64_t tri_len,
                          uint64_t band_entries, void *stream)
{
    if (!ctx || !set) return fail(GBD_EINVAL, "gbd_all_pairs_to_host: NULL context or set");
    const uint64_t n = set->n;
    const uint64_t need = n < 2 ? 0 : n * (n - 1) / 2;
    if (tri_len != need)
        return fail(GBD_EINVAL, "gbd_all_pairs_to_host: tri_len is " + std::to_string(tri_len) +
                                    ", expected n(n-1)/2 = " + std::to_string(need));
    if (need == 0) return GBD_OK;
    if (!h_tri) return fail(GBD_EINVAL, "gbd_all_pairs_to_host: h_tri is NULL");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    cudaStream_t cp = ctx->streams.aux[1];          // copies; the bands' launches use aux[0]
    // each band: whole rows, at most `cap` entries (at least one row)
    uint64_t cap = band_entries ? band_entries : kBandEntries;
    cap = std::min<uint64_t>(std::max<uint64_t>(cap, n - 1), need);
    uint16_t *buf[2] = {nullptr, nullptr};
    cudaEvent_t computed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    int rc = GBD_OK;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMallocAsync((void **)&buf[k], cap * sizeof(uint16_t), st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&computed[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "gbd_all_pairs_to_host: staging set-up");
    uint64_t band = 0;
    for (uint64_t a0 = 0; rc == GBD_OK && a0 + 1 < n; ++band) {
        uint64_t a1 = a0, len = 0;
        while (a1 + 1 < n && len + (n - 1 - a1) <= cap) len += n - 1 - a1++;
        const int k = (int)(band & 1);
        // the buffer's previous band must have reached the host before it is overwritten
        if (band >= 2 && (e = cudaStreamWaitEvent(st, copied[k], 0)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaStreamWaitEvent");
            break;
        }
        rc = tri_band_impl(ctx, set, a0, a1, buf[k], st);
        if (rc != GBD_OK) break;
        const uint64_t base = a0 * n - a0 * (a0 + 1) / 2;
        if ((e = cudaEventRecord(computed[k], st)) == cudaSuccess && (e = cudaStreamWaitEvent(cp, computed[k], 0)) == cudaSuccess &&
            (e = cudaMemcpyAsync(h_tri + base, buf[k], len * sizeof(uint16_t), cudaMemcpyDeviceToHost, cp)) == cudaSuccess)
            e = cudaEventRecord(copied[k], cp);
        if (e != cudaSuccess) rc = cuda_fail(e, "gbd_all_pairs_to_host: band copy");
        a0 = a1;
    }
    // the triangle is in host memory when the call returns
    cudaError_t se = cudaStreamSynchronize(cp);
    cudaError_t se2 = cudaStreamSynchronize(st);
    for (int k = 0; k < 2; ++k) {
        if (buf[k]) cudaFreeAsync(buf[k], st);
        if (computed[k]) cudaEventDestroy(computed[k]);
        if (copied[k]) cudaEventDestroy(copied[k]);
    }
    if (rc != GBD_OK) return rc;
    if (se != cudaSuccess) return cuda_fail(se, "gbd_all_pairs_to_host: copies");
    if (se2 != cudaSuccess) return cuda_fail(se2, "gbd_all_pairs_to_host: bands");
    return GBD_OK;
}

int gbd_tile(gbd_ctx *ctx, const gbd_set *A, uint64_t a0, uint64_t a1, const gbd_set *B,
             uint64_t b0, uint64_t b1, uint16_t *d_out, uint64_t ld, void *stream)
{
    if (!ctx || !A || !B) return fail(GBD_EINVAL, "gbd_tile: NULL context or set");
    if (a0 > a1 || a1 > A->n || b0 > b1 || b1 > B->n)
        return fail(GBD_EINVAL, "gbd_tile: row or column range outside the sets");
    if (ld < b1 - b0) return fail(GBD_EINVAL, "gbd_tile: ld is smaller than the column count");
    if (a0 == a1 || b0 == b1) return GBD_OK;
    if (!d_out) return fail(GBD_EINVAL, "gbd_tile: d_out is NULL");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    return tile_impl(ctx, A, a0, a1, B, b0, b1, d_out, ld, (cudaStream_t)stream);
}

int gbd_tile_hits(gbd_ctx *ctx, const gbd_set *A, uint64_t a0, uint64_t a1, const gbd_set *B,
                  uint64_t b0, uint64_t b1, const gbd_threshold *th, uint16_t *d_out, uint64_t ld,
                  uint32_t *d_hits, uint64_t hit_capacity, uint64_t *d_hit_count,
                  const int32_t *d_ref_labels, int32_t *d_row_labels, void *stream)
{
    if (!ctx || !A || !B) return fail(GBD_EINVAL, "gbd_tile_hits: NULL context or set");
    int rc = check_threshold(th);
    if (rc != GBD_OK) return rc;
    if (a0 > a1 || a1 > A->n || b0 > b1 || b1 > B->n)
        return fail(GBD_EINVAL, "gbd_tile_hits: row or column range outside the sets");
    if (d_out && ld < b1 - b0) return fail(GBD_EINVAL, "gbd_tile_hits: ld is smaller than the column count");
    if (d_hits && !d_hit_count) return fail(GBD_EINVAL, "gbd_tile_hits: a hit list needs d_hit_count");
    if ((d_ref_labels == nullptr) != (d_row_labels == nullptr))
        return fail(GBD_EINVAL, "gbd_tile_hits: annotation needs both d_ref_labels and d_row_labels");
    if (a1 > 0xffffffffull || b1 > 0xffffffffull) return fail(GBD_EINVAL, "gbd_tile_hits: read index beyond 32 bits");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (d_hit_count) GBD_CUDA_TRY(cudaMemsetAsync(d_hit_count, 0, sizeof(uint64_t), st));
    if (d_row_labels && a1 > a0) GBD_CUDA_TRY(cudaMemsetAsync(d_row_labels, 0xff, (a1 - a0) * sizeof(int32_t), st));
    if (a0 == a1 || b0 == b1) return GBD_OK;
    // distances first (into the caller's rectangle or a scratch one), then the epilogue
    // streams over them
    uint16_t *rect = d_out;
    uint64_t rld = ld;
    if (!rect) {
        rld = b1 - b0;
        GBD_CUDA_TRY(cudaMallocAsync((void **)&rect, (a1 - a0) * rld * sizeof(uint16_t), st));
    }
    rc = tile_impl(ctx, A, a0, a1, B, b0, b1, rect, rld, st);
    if (rc == GBD_OK)
        rc = launch_rect_epilogue(rect, rld, A->view(), a0, a1, B->view(), b0, b1, B->max_len,
                                  Threshold{th->num, th->den, th->abs_max},
                                  d_hits, d_hits ? hit_capacity : 0,
                                  reinterpret_cast<unsigned long long *>(d_hit_count), d_ref_labels, d_row_labels,
                                  ctx->sm_count, st);
    if (!d_out) cudaFreeAsync(rect, st);
    return rc;
}

int gbd_threshold_components(gbd_ctx *ctx, const gbd_set *set, const gbd_threshold *th, uint32_t *d_labels,
                             uint64_t *d_edges, uint16_t *d_tri, void *stream)
{
    if (!ctx || !set || !d_labels) return fail(GBD_EINVAL, "gbd_threshold_components: NULL argument");
    int rc = check_threshold(th);
    if (rc != GBD_OK) return rc;
    const uint64_t n = set->n;
    if (n > 0xffffffffull) return fail(GBD_EINVAL, "gbd_threshold_components: more than 2^32 reads");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (d_edges) GBD_CUDA_TRY(cudaMemsetAsync(d_edges, 0, sizeof(uint64_t), st));
    if (n == 0) return GBD_OK;
    const uint64_t m = n * (n - 1) / 2;
    const Threshold t{th->num, th->den, th->abs_max};
    if (d_tri) {
        // the whole triangle, kept for the caller, then one stream over it
        if (m > 0) rc = all_pairs_impl(ctx, set, d_tri, st);
        if (rc == GBD_OK)
            rc = launch_tri_components(d_tri, set->view(), set->max_len, t, d_labels,
                                       reinterpret_cast<unsigned long long *>(d_edges),
                                       ctx->sm_count, st);
        return rc;
    }
    // bands of rows whose distances fit a bounded scratch: each band is computed, its hits
    // joined into the forest, and the scratch reused
    const uint64_t budget = ctx->params.band_entries ? ctx->params.band_entries : kBandEntries;
    // at least one whole row (the longest, n - 1 entries), so every band fits
    const uint64_t scratch = std::max<uint64_t>(n - 1, std::min<uint64_t>(budget, n * (n - 1)));
    uint16_t *rect = nullptr;
    BandForest bf;
    if (m > 0) GBD_CUDA_TRY(cudaMallocAsync((void **)&rect, scratch * sizeof(uint16_t), st));
    rc = band_forest_begin(bf, set->view(), t, d_labels, scratch, ctx->sm_count, st);
    for (uint64_t a0 = 0; rc == GBD_OK && a0 + 1 < n;) {
        const uint64_t ld = n - a0 - 1;              // columns a0 + 1 .. n - 1
        const uint64_t a1 = std::min<uint64_t>(n - 1, a0 + std::max<uint64_t>(1, scratch / ld));
        if ((a1 - a0) * ld > scratch) {
            rc = fail(GBD_EINVAL, "gbd_threshold_components: band larger than its scratch");
            break;
        }
        rc = band_impl(ctx, set, a0, a1, rect, ld, st);
        if (rc == GBD_OK)
            rc = band_forest_add(bf, rect, ld, set->view(), a0, a1, set->max_len, t, d_labels, ctx->sm_count, st);
        a0 = a1;
    }
    const int erc = band_forest_end(bf, d_labels, n, reinterpret_cast<unsigned long long *>(d_edges), ctx->sm_count, st);
    if (rect) cudaFreeAsync(rect, st);
    return rc != GBD_OK ? rc : erc;
}

int gbd_rect_hits(gbd_ctx *ctx, const gbd_set *A, uint64_t a0, uint64_t a1, const gbd_set *B, uint64_t b0,
                  uint64_t b1, const uint16_t *d_rect, uint64_t ld, const gbd_threshold *th, uint32_t *d_hits,
                  uint64_t hit_capacity, uint64_t *d_hit_count, const int32_t *d_ref_labels, int32_t *d_row_labels,
                  void *stream)
{
    if (!ctx || !A || !B) return fail(GBD_EINVAL, "gbd_rect_hits: NULL context or set");
    int rc = check_threshold(th);
    if (rc != GBD_OK) return rc;
    if (a0 > a1 || a1 > A->n || b0 > b1 || b1 > B->n)
        return fail(GBD_EINVAL, "gbd_rect_hits: row or column range outside the sets");
    if (a1 > a0 && b1 > b0 && (!d_rect || ld < b1 - b0 || reinterpret_cast<uintptr_t>(d_rect) % 2 != 0))
        return fail(GBD_EINVAL, "gbd_rect_hits: bad rectangle");
    if (d_hits && !d_hit_count) return fail(GBD_EINVAL, "gbd_rect_hits: a hit list needs d_hit_count");
    if ((d_ref_labels == nullptr) != (d_row_labels == nullptr))
        return fail(GBD_EINVAL, "gbd_rect_hits: annotation needs both d_ref_labels and d_row_labels");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (d_hit_count) GBD_CUDA_TRY(cudaMemsetAsync(d_hit_count, 0, sizeof(uint64_t), st));
    if (d_row_labels && a1 > a0) GBD_CUDA_TRY(cudaMemsetAsync(d_row_labels, 0xff, (a1 - a0) * sizeof(int32_t), st));
    if (a0 == a1 || b0 == b1) return GBD_OK;
    return launch_rect_epilogue(d_rect, ld, A->view(), a0, a1, B->view(), b0, b1, B->max_len,
                                Threshold{th->num, th->den, th->abs_max},
                                d_hits, d_hits ? hit_capacity : 0, reinterpret_cast<unsigned long long *>(d_hit_count),
                                d_ref_labels, d_row_labels, ctx->sm_count, st);
}

int gbd_tri_components(gbd_ctx *ctx, const gbd_set *set, const uint16_t *d_tri, const gbd_threshold *th,
                       uint32_t *d_labels, uint64_t *d_edges, void *stream)
{
    if (!ctx || !set || !d_labels) return fail(GBD_EINVAL, "gbd_tri_components: NULL argument");
    int rc = check_threshold(th);
    if (rc != GBD_OK) return rc;
    const uint64_t n = set->n;
    if (n >= 2 && !d_tri) return fail(GBD_EINVAL, "gbd_tri_components: NULL triangle");
    if (n > 0xffffffffull) return fail(GBD_EINVAL, "gbd_tri_components: more than 2^32 reads");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (d_edges) GBD_CUDA_TRY(cudaMemsetAsync(d_edges, 0, sizeof(uint64_t), st));
    if (n == 0) return GBD_OK;
    return launch_tri_components(d_tri, set->view(), set->max_len, Threshold{th->num, th->den, th->abs_max}, d_labels,
                                 reinterpret_cast<unsigned long long *>(d_edges), ctx->sm_count, st);
}

int gbd_batch(gbd_ctx *ctx, const gbd_set *const *samples, uint64_t ns, uint16_t *const *d_tris,
              void *stream)
{
    if (!ctx || (ns > 0 && (!samples || !d_tris))) return fail(GBD_EINVAL, "gbd_batch: NULL argument");
    for (uint64_t s = 0; s < ns; ++s) {
        if (!samples[s]) return fail(GBD_EINVAL, "gbd_batch: NULL sample " + std::to_string(s));
        if (samples[s]->n >= 2 && !d_tris[s]) return fail(GBD_EINVAL, "gbd_batch: NULL output " + std::to_string(s));
    }
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (!use_systolic(ctx)) {
        for (uint64_t s = 0; s < ns; ++s) {
            const uint64_t n = samples[s]->n;
            if (n < 2) continue;
            GeneralJob job{samples[s]->view(), samples[s]->view(), 0, n, 0, n, 0, OUT_TRI, d_tris[s]};
            job.out_len = out_extent(ctx, n * (n - 1) / 2);
            int rc = run_general(job, scoring_of(ctx), ctx->sm_count, st);
            if (rc != GBD_OK) return rc;
        }
        return GBD_OK;
    }
    // One plan over every sample's entries, largest first; one launch per length bucket.
    // The launch group is captured once as a CUDA graph and replayed while the samples
    // and outputs stay the same.
    for (uint64_t s = 0; s < ns; ++s) {
        int rc = build_tri_schedule(const_cast<gbd_set *>(samples[s]), st);
        if (rc != GBD_OK) return rc;
    }
    int rc = systolic_prepare();
    if (rc != GBD_OK) return rc;
    BatchGraph *bg = static_cast<BatchGraph *>(ctx->batch_cache);
    bool fresh = false;
    if (!(bg && bg->matches(samples, ns, d_tris, ctx->params.conversion, ctx->params.gap_open))) {
        free_batch_cache(ctx);
        bg = new BatchGraph();
        ctx->batch_cache = bg;
        rc = capture_batch(ctx, bg, samples, ns, d_tris);
        if (rc != GBD_OK) {
            free_batch_cache(ctx);
            return rc;
        }
        fresh = true;                        // the capture already counted its kernels
    } else if (bg->trial < kTrials) {
        // autotuning: read the time of the previous candidate's launch, move to the next
        // candidate (or, after the last, to the fastest) and record its graph
        if (bg->timing) {
            GBD_CUDA_TRY(cudaEventSynchronize(bg->t1));
            float ms = 0.f;
            GBD_CUDA_TRY(cudaEventElapsedTime(&ms, bg->t0, bg->t1));
            bg->trial_ms[bg->trial] = ms;
            bg->timing = false;
            ++bg->trial;
            if (bg->trial == 3) {               // the stream-count trials take the best scale
                int bs = 0;
                for (int t = 1; t < 3; ++t)
                    if (bg->trial_ms[t] < bg->trial_ms[bs]) bs = t;
                bg->cands[3].scale = bg->cands[4].scale = bg->cands[bs].scale;
            }
        }
        int next;
        if (bg->trial < kTrials) {
            next = bg->trial;
        } else {
            next = 0;
            for (int t = 1; t < kTrials; ++t)
                if (bg->trial_ms[t] < bg->trial_ms[next]) next = t;
            bg->chosen = next;
        }
        if (next != bg->current || bg->trial < kTrials) {
            rc = record_batch_graph(ctx, bg, samples, ns, d_tris, next);
            if (rc != GBD_OK) {
                free_batch_cache(ctx);
                return rc;
            }
            fresh = true;
        }
    }
    const bool time_it = bg->trial < kTrials;
    if (time_it) GBD_CUDA_TRY(cudaEventRecord(bg->t0, st));
    GBD_CUDA_TRY(cudaGraphLaunch(bg->exec, st));
    if (time_it) {
        GBD_CUDA_TRY(cudaEventRecord(bg->t1, st));
        bg->timing = true;
    }
    if (!fresh) note_launches(bg->kernels);
    return GBD_OK;
}

int gbd_batch_tuning(const gbd_ctx *ctx, uint32_t capacity, double *trial_ms, double *trial_scale,
                     int32_t *trial_streams, uint32_t *ntrials, int32_t *chosen, int *done)
{
    if (!ctx) return fail(GBD_EINVAL, "gbd_batch_tuning: NULL context");
    const BatchGraph *bg = static_cast<const BatchGraph *>(ctx->batch_cache);
    if (!bg) return fail(GBD_ENOTFOUND, "gbd_batch_tuning: no batch has run on this context");
    for (int t = 0; t < kTrials && (uint32_t)t < capacity; ++t) {
        if (trial_ms) trial_ms[t] = bg->trial_ms[t];
        if (trial_scale) trial_scale[t] = bg->cands[t].scale;
        if (trial_streams) trial_streams[t] = 1 + bg->cands[t].naux;
    }
    if (ntrials) *ntrials = kTrials;
    if (chosen) *chosen = bg->chosen;
    if (done) *done = bg->trial >= kTrials ? 1 : 0;
    return GBD_OK;
}

uint64_t gbd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int gbd_bounds_check(uint64_t *violation)
{
    if (!violation) return fail(GBD_EINVAL, "gbd_bounds_check: NULL argument");
    *violation = ~0ull;
    if (!GBD_BOUNDS_CHECK) return fail(GBD_ENOTFOUND, "gbd_bounds_check: the library was built without bounds checks");
    GBD_CUDA_TRY(cudaDeviceSynchronize());        // every launch so far has finished
    *violation = std::min(bounds_take_systolic(), bounds_take_general());
    return GBD_OK;
}

int gbd_debug_output_limit(gbd_ctx *ctx, uint64_t limit)
{
    if (!ctx) return fail(GBD_EINVAL, "gbd_debug_output_limit: NULL context");
    if (!GBD_BOUNDS_CHECK)
        return fail(GBD_ENOTFOUND, "gbd_debug_output_limit: the library was built without bounds checks");
    ctx->debug_out_limit = limit;
    return GBD_OK;
}

int gbd_probe_op_rate(int op, uint32_t iters, double *lane_ops_per_s, void *stream)
{
    int dev = 0, sms = 0;
    GBD_CUDA_TRY(cudaGetDevice(&dev));
    GBD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return probe_op_rate(op, iters, lane_ops_per_s, sms, (cudaStream_t)stream);
}

}  // extern "C"
