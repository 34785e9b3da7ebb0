// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/gbd.h"

namespace gbd {

// ------------------------------------------------------------------ error plumbing
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define GBD_CUDA_TRY(call)                                   \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return ::gbd::cuda_fail(_e, #call); \
    } while (0)

// Count of kernel launches made by the library (see gbd_kernel_launches).
void note_launches(uint64_t k);

// ------------------------------------------------------------------ bounds-checked build
// Compiled with -DGBD_BOUNDS_CHECK=1 (a debug build of the library), every distance store,
// every index into the general kernel's boundary-row scratch and every write into (and the
// read window of) the systolic kernel's shared-memory profile ring checks its index
// against the extent of its buffer.  An index out of range is not used (nothing faults;
// a read window is moved to a harmless in-range place, so results are wrong but no
// access leaves its buffer) and the smallest such index, tagged with its site in the top
// 8 bits, is kept in a device word of the kernel's source file; gbd_bounds_check reads
// and clears it.  Without the flag the checks compile to nothing.
#ifndef GBD_BOUNDS_CHECK
#define GBD_BOUNDS_CHECK 0
#endif
enum BoundsSite : unsigned {
    BOUNDS_SYSTOLIC_OUT = 1,      // a systolic distance store
    BOUNDS_SYSTOLIC_RING = 2,     // the systolic profile ring / table (shared memory)
    BOUNDS_GENERAL_OUT = 3,       // a general-kernel distance store
    BOUNDS_GENERAL_SCRATCH = 4,   // the general kernel's boundary rows
};
#if GBD_BOUNDS_CHECK
static __device__ unsigned long long g_bounds_first = ~0ull;
__device__ __forceinline__ bool bounds_ok(uint64_t idx, uint64_t extent, unsigned site)
{
    if (idx < extent) return true;
    atomicMin(&g_bounds_first, ((unsigned long long)site << 56) | (idx & ((1ull << 56) - 1)));
    return false;
}
#else
__device__ __forceinline__ bool bounds_ok(uint64_t, uint64_t, unsigned) { return true; }
#endif
// Reads and clears the source file's word (UINT64_MAX when nothing was recorded or the
// build has no checks).
uint64_t bounds_take_systolic();
uint64_t bounds_take_general();

// Score-to-distance rule (GBD_CONV_*) applied to the local score S of reads of lengths
// la and lb; the result is stored as uint16.  GBD_CONV_NORM divides in 32 bits: 65535 * x
// with x <= m <= 65535 stays below 2^32.
__device__ __forceinline__ uint16_t score_to_distance(int S, int la, int lb, int conversion)
{
    const int hi = max(la, lb);
    if (conversion == GBD_CONV_NORM) {
        if (hi == 0) return 0;
        const int x = min(max(hi - S, 0), hi);
        return (uint16_t)((65535u * (uint32_t)x) / (uint32_t)hi);
    }
    int d;
    if (conversion == GBD_CONV_SCORE) d = S;
    else if (conversion == GBD_CONV_MIN) d = min(la, lb) - S;
    else d = hi - S;
    d = d < 0 ? 0 : (d > 65535 ? 65535 : d);
    return (uint16_t)d;
}

// ------------------------------------------------------------------ packed read sets
constexpr int kBasesPerWord = 16;

struct DeviceReads {            // plain view passed to kernels
    const uint32_t *words;      // n * stride 2-bit packed words
    const uint16_t *len;        // n lengths
    uint64_t n;
    uint32_t stride;            // words per read
};

// Entries grouped by rows per lane, resident on the device.  Each non-empty bucket is
// one launch of the kernel instantiated for its R.
struct SysPlan {
    struct Bucket {
        int R = 0;
        uint32_t nentries = 0, nunits = 0;
        uint32_t piece = 1024;                  // subjects per work unit
        size_t entry_off = 0, prefix_off = 0;   // offsets into d_buf (bytes)
    };
    std::vector<Bucket> buckets;
    void *d_buf = nullptr;
    bool stream_ordered = false;   // d_buf from cudaMallocAsync (freed on a stream)
    uint32_t piece = 1024;         // subjects per work unit
    uint64_t units() const
    {
        uint64_t u = 0;
        for (const auto &b : buckets) u += b.nunits;
        return u;
    }
};

// Streams over which consecutive bucket launches of the systolic kernel alternate: the
// caller's stream, then aux[0], aux[1], ...; they fork from the caller's stream on `fork`
// and join back into it on join[k].
struct StreamSet {
    static constexpr int kMaxAux = 2;
    cudaStream_t aux[kMaxAux] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxAux] = {};
};

// Device-resident schedule of a read set for the all-pairs triangle: one systolic entry
// per read i short enough to be a systolic query (subjects i+1 .. n-1, in the set's own
// order, so a warp writes a contiguous run of triangle row i), and the list of the
// longer reads, whose rows go to the general kernel.
struct TriSchedule {
    bool built = false;
    SysPlan plan;                     // entries with job index 0
    uint32_t *d_long_rows = nullptr;  // reads longer than the systolic query limit
    uint64_t *d_long_prefix = nullptr;
    uint64_t nlong = 0;
    uint64_t long_units = 0;          // pairs in those rows
};

}  // namespace gbd

struct gbd_ctx {
    int device = 0;
    gbd_params params{};
    int sm_count = 0;
    gbd::StreamSet streams;           // extra streams for overlapping bucket launches
    cudaStream_t capture = nullptr;   // stream that records batch graphs
    void *batch_cache = nullptr;      // last captured batch graph (api.cu)
    // gbd_mds's fp16 square (ld^2 entries, 20 GB at n = 10^5), kept between calls: the
    // stream-ordered pool would unmap it at every synchronisation and map it again (ms)
    void *mds_w = nullptr;
    size_t mds_w_bytes = 0;
    cudaEvent_t mds_w_done = nullptr; // recorded after the last work that used mds_w
    uint64_t debug_out_limit = 0;     // bounds-checked builds: cap on the output extents (0 = none)
};

// The output extent a job of this context checks against: `real`, or the debug cap of a
// bounds-checked build when it is smaller.
inline uint64_t out_extent(const gbd_ctx *ctx, uint64_t real)
{
    return (GBD_BOUNDS_CHECK && ctx->debug_out_limit && ctx->debug_out_limit < real) ? ctx->debug_out_limit : real;
}

struct gbd_set {
    gbd_ctx *ctx = nullptr;
    int device = 0;
    uint64_t id = 0;            // unique per process (keys cached batch graphs)
    uint64_t n = 0;
    uint32_t stride = 0;        // words per read
    uint32_t max_len = 0;
    uint32_t *d_words = nullptr;
    uint16_t *d_len = nullptr;
    std::vector<uint16_t> h_len;
    double pair_cells = 0.0;
    double mean_len = 0.0;
    gbd::TriSchedule sched;
    gbd::DeviceReads view() const { return {d_words, d_len, n, stride}; }
};

namespace gbd {

// ------------------------------------------------------------------ kernels (launchers)
// K0: pack + validate.  seq/offsets are device pointers.  err receives the smallest
// position (relative to offsets[0]) of an invalid byte, or UINT64_MAX.
cudaError_t launch_pack(const uint8_t *seq, const uint64_t *offsets, uint64_t n, uint32_t stride,
                        uint32_t *words, uint16_t *len, unsigned long long *err,
                        cudaStream_t stream);

// Output addressing of a block of pairs.
//  OUT_TRI:      A == B, pairs i < j, out[k(i,j)] (row-major strict upper triangle)
//  OUT_RECT:     out[(i-a0)*ld + (j-b0)]
//  OUT_TRI_ROWS: A == B, the triangle rows listed in rows[]: pairs (rows[x], j) for
//                rows[x] < j < n, units counted by row_prefix (nrows + 1 entries)
enum OutMode : int { OUT_TRI = 0, OUT_RECT = 1, OUT_TRI_ROWS = 2 };

struct Scoring {
    int match, mismatch, gap, conversion;
    int gap_open = 0;           // > 0: affine gaps (Gotoh), gap run of L costs gap_open + L*gap
};

// General kernel: one pair per thread, int32 strip DP, boundary rows in scratch.
struct GeneralJob {
    DeviceReads A, B;
    uint64_t a0, a1, b0, b1, ld;
    int mode;
    uint16_t *out;
    const uint32_t *rows = nullptr;   // OUT_RECT / OUT_TRI_ROWS: explicit list of A rows
    uint64_t nrows = 0;
    const uint64_t *row_prefix = nullptr;   // OUT_TRI_ROWS: pairs before each listed row
    uint64_t units_total = 0;               // OUT_TRI_ROWS: row_prefix[nrows]
    uint64_t out_len = 0;                   // entries of out (checked in bounds-checked builds)
    uint64_t out_base = 0;                  // OUT_TRI_ROWS: out[k(i,j) - out_base] (a band of rows)
};
int run_general(const GeneralJob &job, const Scoring &sc, int sm_count, cudaStream_t stream);
// Same kernel on a rectangle job, with boundary rows in caller-provided scratch
// (scratch_ints ints); allocates nothing.
int run_general_in(const GeneralJob &job, const Scoring &sc, int *scratch, uint64_t scratch_ints,
                   int sm_count, cudaStream_t stream);

// Threshold epilogue (threshold.cu), streaming over distances already computed.
struct Threshold {
    uint32_t num, den, abs_max;
};
// Rectangle D[r][c] = out[(r-a0)*ld + (c-b0)], r in [a0,a1), c in [b0,b1): hits appended
// to hits (3 words each, up to cap; every hit counted in *count), and row annotation
// from col_labels into row_labels (by r - a0) when both are set.
// colmax_len: an upper bound of the column reads' lengths (the set's longest read).
int launch_rect_epilogue(const uint16_t *out, uint64_t ld, const DeviceReads &A, uint64_t a0, uint64_t a1,
                         const DeviceReads &B, uint64_t b0, uint64_t b1, uint32_t colmax_len, const Threshold &th,
                         uint32_t *hits, uint64_t cap, unsigned long long *count, const int32_t *col_labels,
                         int32_t *row_labels, int sm_count, cudaStream_t st);
// Triangle of a set: every hit pair (i, j) is joined in the union-find forest `parent`
// (which starts as parent[i] = i) and counted in *count (if set); then every read is
// pointed at its root, the smallest read of its component.
// max_len: the set's longest read.
int launch_tri_components(const uint16_t *tri, const DeviceReads &S, uint32_t max_len, const Threshold &th,
                          uint32_t *parent, unsigned long long *count, int sm_count, cudaStream_t st);

// Threshold-graph components without the whole triangle: the caller computes the
// distances of one band of rows [a0, a1) at a time into a rectangle whose row a0 + rr
// holds columns j = a0 + 1 + c at rect[rr * ld + c] for c >= rr (that is, j > a0 + rr),
// and hands each band to band_forest_add, which joins its hits into the forest `parent`.
// begin sets every read to its own root; end points every read at its component's
// smallest read, writes the number of hits to *count (if set) and frees the scratch.
struct BandForest {
    uint16_t *T = nullptr;                  // hit bound per read (n + 16 entries)
    uint2 *edges = nullptr;                 // one band's hits
    unsigned long long *cnt = nullptr;      // [0] hits of the band, [1] running total
    uint64_t cap = 0;
    bool first = true;                      // the forest is still fresh
};
int band_forest_begin(BandForest &bf, const DeviceReads &S, const Threshold &th, uint32_t *parent, uint64_t max_entries,
                      int sm_count, cudaStream_t st);
int band_forest_add(BandForest &bf, const uint16_t *rect, uint64_t ld, const DeviceReads &S, uint64_t a0, uint64_t a1,
                    uint32_t max_len, const Threshold &th, uint32_t *parent, int sm_count, cudaStream_t st);
int band_forest_end(BandForest &bf, uint32_t *parent, uint64_t n, unsigned long long *count, int sm_count,
                    cudaStream_t st);

// Frees the context's cached batch graph.
void free_batch_cache(gbd_ctx *ctx);
// Frees the context's cached MDS square (after its last use has finished).
void free_mds_cache(gbd_ctx *ctx);

// Instruction-rate probe.
int probe_op_rate(int op, uint32_t iters, double *rate, int sm_count, cudaStream_t stream);

}  // namespace gbd
