// Host/device interface of the warp-systolic kernel.
#pragma once

#include "gbd_internal.cuh"

namespace gbd {

// Reads up to this length can be the query (row) read of a systolic work unit.
constexpr int kSystolicMaxQuery = 512;
// Default number of subjects per work unit (bounds the tail of every launch).
constexpr uint32_t kSystolicPiece = 1024;

// One output problem: queries of Q against subjects of S.
struct SysJob {
    DeviceReads Q, S;
    const uint32_t *sub_perm;   // subject list (original indices in S); NULL = identity
    uint16_t *out;
    uint64_t n;                 // OUT_TRI: reads in the set
    uint64_t ld, row0, col0;    // OUT_RECT: out[(q-row0)*ld + (s-col0)]
    int mode;                   // OUT_TRI or OUT_RECT
    int conversion;
    int gap_open;               // affine gaps (extend 1) when > 0; launch with affine = true
    uint64_t out_len;           // entries of out (checked in bounds-checked builds)
    uint64_t out_base;          // OUT_TRI: out[k(i,j) - out_base] (a band of rows); 0 otherwise
};

// One query (original index q in Q, length <= 512) against the subjects at list
// positions [sub_begin, sub_begin + nsub); split into units of plan.piece subjects.
struct SysEntry {
    uint32_t job, q, sub_begin, nsub;
};

// Rows per lane of a query of length la (1..16 for la <= 512).
inline int systolic_rows(int la) { return la <= 32 ? 1 : (la + 31) / 32; }

// Groups entries by R (rows[i] = R of entries[i]) and uploads them.  Entries keep their
// order inside a bucket (callers put the largest first).  persistent: cudaMalloc (kept
// with a read set) instead of stream-ordered memory.
// piece_len == 0: each bucket's piece comes from the cost model (tuned_piece) given the
// subjects' mean length.
// piece_scale multiplies the cost model's piece (the batch autotuner's knob).
int build_plan(const std::vector<SysEntry> &entries, const std::vector<uint8_t> &rows,
               SysPlan &plan, bool persistent, cudaStream_t stream, uint32_t piece_len,
               double mean_subject_len, int sm_count, double piece_scale = 1.0);
uint32_t tuned_piece(uint64_t pairs, double mean_len, int warps);
// Number of warps the systolic kernel keeps resident on the whole GPU.
int systolic_resident_warps(int sm_count);
void free_plan(SysPlan &plan, cudaStream_t stream);

// ss, naux: consecutive buckets alternate between `stream` and the first naux streams of
// ss (naux <= StreamSet::kMaxAux; ss == nullptr or naux == 0: one stream).
// affine: the jobs use affine gaps (every job of the launch the same way).
int run_systolic(const SysJob *d_jobs, const SysPlan &plan, int sm_count, cudaStream_t stream,
                 const StreamSet *ss = nullptr, int naux = 0, bool affine = false);
// Streams the plain (non-batched) launches use: the caller's and one more.
constexpr int kDefaultAuxStreams = 1;
// Largest gap opening penalty the systolic kernel takes (its int16 values stay in range).
constexpr int kSystolicMaxGapOpen = 1000;
size_t systolic_smem_bytes();
// Sets kernel attributes and occupancy of every instantiation (once; before any capture).
int systolic_prepare();

}  // namespace gbd
