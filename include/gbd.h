/*
 * gbd -- all-pairs Smith-Waterman read distances on one GB300 (sm_103a).
 *
 * The operation (arxiv 1803.02272, section 2.2, "Scalable pairwise distances
 * computation"): the dissimilarity between two reads is derived from their local
 * alignment score, found by the Smith-Waterman algorithm; the program `disseq` takes
 * two read files of m and n reads and returns the m x n matrix D, and the paper's
 * all-pairs run over 1e5 reads produces ~5e9 values (one per unordered pair).
 *
 * The paper fixes no scores and no score-to-distance rule.  This library's readings,
 * all of them fields of gbd_params:
 *   s(x,y) = +match if x == y else +mismatch (defaults +1 / -1); linear gap penalty
 *   `gap` per gapped base (default 1), optionally affine (`gap_open` per gap run);
 *   H(i,0) = H(0,j) = 0, H(i,j) = max(0, H(i-1,j-1)+s(a_i,b_j), H(i-1,j)-gap,
 *   H(i,j-1)-gap), S = max over all cells of H;
 *   d = max(la, lb) - S (GBD_CONV_MAX, default), stored as uint16.
 *
 * Conventions for every call:
 *   - Reads are bytes over {A,C,G,T} (lower case accepted), concatenated; read r is
 *     seq[offsets[r] .. offsets[r+1]).  Lengths may be 0 .. 65535.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Compute calls are
 *     asynchronous on it; gbd_load_reads synchronises `stream` once to read back its
 *     validation flag.
 *   - Output pointers are DEVICE pointers owned by the caller (for example a torch
 *     tensor's data_ptr()).  The library owns gbd_ctx, gbd_set and gbd_server objects.
 *   - Every int-returning call returns GBD_OK (0) or a GBD_E* code and then sets a
 *     thread-local message readable with gbd_last_error().  No C++ exception crosses
 *     this boundary.
 *   - A context's calls may be issued from one host thread at a time; a server object
 *     is safe to use from several host threads.
 */
#ifndef GBD_H
#define GBD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GBD_OK        0
#define GBD_EINVAL    1   /* bad argument: non-ACGT byte, length > 65535, wrong size, NULL */
#define GBD_ENOMEM    2   /* a device or host allocation failed */
#define GBD_EBUDGET   3   /* a request exceeds the server's HBM budget even when alone */
#define GBD_ETIMEDOUT 4   /* a bounded wait ran out */
#define GBD_ECUDA     5   /* a CUDA runtime call failed (message has the CUDA error) */
#define GBD_ENOTFOUND 6   /* unknown server ticket */

/* score-to-distance rules (gbd_params.conversion).  Section 2.2 derives the dissimilarity
 * from the local score and leaves the rule open; these are the readings offered. */
#define GBD_CONV_MAX   0  /* d = max(la, lb) - S, clamped to [0, 65535]  (default) */
#define GBD_CONV_MIN   1  /* d = min(la, lb) - S, clamped to [0, 65535] */
#define GBD_CONV_SCORE 2  /* the raw local score S, clamped to [0, 65535] */
#define GBD_CONV_NORM  3  /* 1 - S/max(la, lb) in 16-bit fixed point: floor(65535 * x / m) with
                             m = max(la, lb) and x = m - S clamped into [0, m]; 0 when m = 0 */

/* kernel choice (gbd_params.kernel) */
#define GBD_KERNEL_AUTO     0  /* systolic kernel where it applies, else the general one */
#define GBD_KERNEL_GENERAL  1  /* one pair per thread, any length and any scores */
#define GBD_KERNEL_SYSTOLIC 2  /* warp-systolic int16x2 kernel (default scores, reads <= 512) */

typedef struct gbd_ctx gbd_ctx;
typedef struct gbd_set gbd_set;
typedef struct gbd_server gbd_server;

typedef struct {
    int16_t  match;       /* score of a matching base pair (default +1) */
    int16_t  mismatch;    /* score of a mismatching base pair (default -1) */
    int16_t  gap;         /* penalty per gapped base, >= 0 (default 1) */
    int16_t  conversion;  /* GBD_CONV_* (default GBD_CONV_MAX) */
    int32_t  kernel;      /* GBD_KERNEL_* (default GBD_KERNEL_AUTO) */
    uint64_t hbm_budget;  /* server admission budget in bytes; 0 = 90 % of free memory */
    uint32_t timeout_us;  /* bound on any host wait inside the library; 0 = 60 s */
    int16_t  gap_open;    /* affine gaps (Gotoh): a run of L gapped bases costs
                             gap_open + L * gap; 0 = linear (default).  With match +1,
                             mismatch -1, gap 1 and gap_open <= 1000 it runs on the
                             systolic kernel, otherwise on the general kernel. */
    uint64_t band_entries;/* scratch (uint16 entries) of gbd_threshold_components when it
                             holds no triangle; 0 = 2^28 (512 MB); never less than one
                             row (n - 1 entries) */
} gbd_params;

/* Fills *p with the defaults above (library plumbing; the paper fixes none of these values). */
void gbd_default_params(gbd_params *p);

/* sizeof(gbd_params) as compiled into the library (for bindings that mirror the struct;
 * no paper counterpart). */
uint64_t gbd_params_size(void);

/* Creates a context on CUDA device `device` (made current on the calling thread); library
 * plumbing with no paper counterpart.
 * p == NULL selects the defaults.  EINVAL on a negative gap or bad enum values.  The
 * library's scratch is stream-ordered (cudaMallocAsync from the device's default pool);
 * gbd_create raises that pool's release threshold to 4 GiB if it is lower, so scratch is
 * reused across calls instead of being unmapped at every synchronisation. */
int gbd_create(gbd_ctx **out, int device, const gbd_params *p);
void gbd_destroy(gbd_ctx *ctx);

/* (No paper counterpart.)  Frees what the context keeps between calls (the MDS square, the
 * captured batch graph)
 * after waiting for the device to finish its work.  The next call that needs them
 * rebuilds them.  EINVAL on a NULL context. */
int gbd_trim(gbd_ctx *ctx);

/* The input of the distance computation (section 2.2: `disseq` reads the sequences of its
 * read files; the all-pairs run reads the ~1e5 amplicon reads of one sample, section 6.1).
 * Copies (if host pointers) and packs n reads into a device-resident set:
 * 2-bit codes A=0 C=1 G=2 T=3, 16 bases per uint32 (base k of a word in bits 2k..2k+1),
 * a fixed stride of ceil(max_len/16) words per read, and per-read uint16 lengths.
 * `seq` and `offsets` (n+1 entries, offsets[0] may be non-zero) may both be host or both
 * be device pointers.  EINVAL (and no set) if a byte is not A/C/G/T/a/c/g/t, a length
 * exceeds 65535 or offsets decrease.  n == 0 gives an empty set. */
int gbd_load_reads(gbd_ctx *ctx, const uint8_t *seq, const uint64_t *offsets, uint64_t n,
                   gbd_set **out, void *stream);
void gbd_free_set(gbd_set *set);
uint64_t gbd_set_size(const gbd_set *set);           /* number of reads */
uint32_t gbd_set_max_len(const gbd_set *set);        /* longest read */
/* Sum over the pairs i < j of len_i * len_j: the DP cells of gbd_all_pairs. */
double gbd_set_pair_cells(const gbd_set *set);

/* All pairwise distances of one read set (section 2.2: the matrix D of all ~5e9 pairwise
 * values of a ~1e5-read sample, every pair computed independently; one value per unordered
 * pair, the distance being symmetric): d_tri[k(i,j)] = d(read i, read j) for every i < j, with the
 * row-major strict upper triangle index k(i,j) = i*n - i*(i+1)/2 + (j-i-1).
 * tri_len must equal n(n-1)/2 (EINVAL otherwise); d_tri is a device pointer. */
int gbd_all_pairs(gbd_ctx *ctx, const gbd_set *set, uint16_t *d_tri, uint64_t tri_len,
                  void *stream);

/* All pairwise distances into host memory (section 2.2's matrix D of a sample, wanted on
 * the host, or larger than the device memory left for it): the triangle, in the layout of
 * gbd_all_pairs, is computed in bands of consecutive rows (each band a contiguous run of the
 * triangle) into two device staging buffers of at most band_entries entries each (0 = 2^28,
 * two 512 MB buffers; never less than one row, n - 1 entries), and each band is copied to
 * h_tri while the next one is computed.  h_tri is a HOST pointer to tri_len uint16 entries
 * (page-locked memory lets the copies overlap the computation; pageable memory works, with
 * each copy synchronous).  The call synchronises `stream` and returns when the whole
 * triangle is in h_tri.  EINVAL on a wrong tri_len or a NULL h_tri. */
int gbd_all_pairs_to_host(gbd_ctx *ctx, const gbd_set *set, uint16_t *h_tri, uint64_t tri_len,
                          uint64_t band_entries, void *stream);

/* Rectangle (section 2.2: `disseq` on two read files of m and n reads returns the m x n
 * matrix D with d_ij the distance between read i of the first and read j of the second):
 * d_out[(r-a0)*ld + (c-b0)] = d(A[r], B[c])
 * for r in [a0,a1), c in [b0,b1); ld >= b1-b0.  A and B may be the same set. */
int gbd_tile(gbd_ctx *ctx, const gbd_set *A, uint64_t a0, uint64_t a1, const gbd_set *B,
             uint64_t b0, uint64_t b1, uint16_t *d_out, uint64_t ld, void *stream);

/* Batched samples (section 6.1: ten Lake Geneva samples L_1..L_10 of 7e4 to 1.4e5 reads each,
 * whose distances are computed sample by sample, section 2.2): one launch group computes the
 * all-pairs triangle of each of ns sets;
 * d_tris[s] receives sample s's triangle (n_s(n_s-1)/2 entries, device pointers). */
int gbd_batch(gbd_ctx *ctx, const gbd_set *const *samples, uint64_t ns,
              uint16_t *const *d_tris, void *stream);

/* (No paper counterpart: the tuning of this library's batched launch.)  The batched launch
 * tunes itself online.  A candidate fixes the shape of the launch group: the work-unit size
 * (subjects per unit, as a multiple of the cost model's size) and the number of streams the
 * per-length-bucket launches alternate over.  The first five calls with a new list of
 * samples and outputs run one candidate each, timed with events on `stream` (each of these
 * calls first waits for the previous one to finish): scales 1, 0.5 and 2 with two streams,
 * then the fastest scale with one and with three streams; from the sixth call on the
 * fastest candidate is replayed as a CUDA graph.  Results are identical for every
 * candidate.  gbd_batch_tuning reports, for up to `capacity` candidates, the timings (ms,
 * 0 until measured), scales and stream counts (any array may be NULL), the number of
 * candidates, the one chosen (-1 while tuning) and whether tuning has finished;
 * ENOTFOUND before any batch. */
int gbd_batch_tuning(const gbd_ctx *ctx, uint32_t capacity, double *trial_ms, double *trial_scale,
                     int32_t *trial_streams, uint32_t *ntrials, int32_t *chosen, int *done);

/* Query rows against a resident reference set (section 4.3: the distances between every
 * read of a sample and the ~2e3 annotated reads of a reference database, computed as a
 * rectangle by `MPI-disseq`; the rows place new reads against known ones).  A server keeps
 * the reference set resident and answers query batches with distance rows.
 * submit copies the queries (host pointers, nq reads) and returns at once with a
 * ticket; the request is admitted when its memory fits the budget beside the requests
 * in flight, and its work overlaps theirs on the device.  d_rows (device, nq x n_ref,
 * row-major) is complete when poll reports done or wait returns GBD_OK.
 * EBUDGET if the request cannot fit even alone. */
int gbd_server_create(gbd_ctx *ctx, const gbd_set *ref, gbd_server **out);
int gbd_server_submit(gbd_server *srv, const uint8_t *seq, const uint64_t *offsets,
                      uint64_t nq, uint16_t *d_rows, uint64_t *ticket);
int gbd_server_poll(gbd_server *srv, uint64_t ticket, int *done);
int gbd_server_wait(gbd_server *srv, uint64_t ticket);
void gbd_server_destroy(gbd_server *srv);

/* Allocation-free rectangle.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- code whose device memory is owned by another
 * allocator (a framework's caching pool or a pre-reserved arena, where a direct cudaMalloc
 * fails or fragments it) or code paths that must not allocate at all.
 *   d_out[i*ld + j] = d(A[i], B[j]) for i < nA, j < nB, with the context's scores.
 *   Inputs are DEVICE pointers owned by the caller: read bytes and nA+1 / nB+1 offsets as
 *   for gbd_load_reads; every read must be at most max_len (<= 65535) bases long.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch (flags, the
 * 2-bit packed reads, the DP boundary rows) is one static device array of 32 MiB that
 * every GPU loading the library holds until the process exits; inputs whose packed form
 * plus one thread block's boundary rows do not fit return GBD_EINVAL.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) and should come
 * before any stream capture.  All calls share the one array; calls that overlap on the GPU (other
 * streams, other host threads) race on the array and must be serialised by the caller.
 * The offsets are checked (one synchronisation of `stream`) before any kernel reads the
 * bytes, and the bytes are checked (a second synchronisation) before any distance is
 * computed.  Errors: EINVAL for a NULL pointer (d_seqA and d_seqB too, even when every
 * read is empty), a non-ACGT byte, a read longer than max_len, decreasing offsets,
 * ld < nB, or inputs too large for the array. */
int gbd_tile_noalloc(gbd_ctx *ctx, const uint8_t *d_seqA, const uint64_t *d_offA, uint64_t nA,
                     const uint8_t *d_seqB, const uint64_t *d_offB, uint64_t nB,
                     uint32_t max_len, uint16_t *d_out, uint64_t ld, void *stream);

/* ---------------------------------------------------------------- threshold epilogue
 * A distance d between reads of lengths la, lb is a hit when
 *   d <= abs_max  and  d * den <= num * max(la, lb)
 * (integer arithmetic; the paper's 97 % homology gap of section 4.3 is num/den = 3/100
 * with abs_max = 65535, the absolute threshold theta of section 5 is num = den = 1,
 * abs_max = theta).  den must be positive. */
typedef struct {
    uint32_t num, den;
    uint32_t abs_max;
} gbd_threshold;

/* Rectangle with the threshold applied to every distance (section 4.3: sample reads
 * against annotated reference reads): the distances are computed into d_out (or, if it is
 * NULL, a scratch rectangle allocated and freed on `stream`), then one streaming pass
 * applies the rule.  Any of the outputs may be NULL:
 *   d_out         the dense rectangle, as gbd_tile (ld >= b1-b0);
 *   d_hits        up to hit_capacity hits as 3 uint32 each: row read index (in A), column
 *                 read index (in B), d -- in no particular order; needs d_hit_count;
 *   d_hit_count   (device, one uint64) the number of hits, also those past the capacity;
 *                 zeroed by the call;
 *   d_ref_labels  (device, int32 by B read index) species of the reference reads, < 0 for
 *                 an unannotated read; with d_row_labels (device, a1-a0 int32, set by the
 *                 call): the species shared by all hits of a row, -1 for no hit, -2 when
 *                 the hits disagree (the diagno-syst rule of section 4.3).
 * Asynchronous on `stream`.  EINVAL on bad ranges or a NULL d_hit_count with d_hits. */
int gbd_tile_hits(gbd_ctx *ctx, const gbd_set *A, uint64_t a0, uint64_t a1, const gbd_set *B,
                  uint64_t b0, uint64_t b1, const gbd_threshold *th, uint16_t *d_out, uint64_t ld,
                  uint32_t *d_hits, uint64_t hit_capacity, uint64_t *d_hit_count,
                  const int32_t *d_ref_labels, int32_t *d_row_labels, void *stream);

/* The same epilogue over a rectangle already computed (d_rect[(r-a0)*ld + (c-b0)] =
 * d(A[r], B[c]), device): one streaming pass, so several thresholds or label sets can be
 * applied without recomputing distances.  Outputs and errors as for gbd_tile_hits. */
int gbd_rect_hits(gbd_ctx *ctx, const gbd_set *A, uint64_t a0, uint64_t a1, const gbd_set *B, uint64_t b0,
                  uint64_t b1, const uint16_t *d_rect, uint64_t ld, const gbd_threshold *th, uint32_t *d_hits,
                  uint64_t hit_capacity, uint64_t *d_hit_count, const int32_t *d_ref_labels, int32_t *d_row_labels,
                  void *stream);

/* Connected components of the threshold graph of a read set (section 5: vertices are the
 * reads, an edge joins i < j when the pair is a hit).  d_labels (device, n uint32):
 * the smallest read index of each read's component.  d_edges (device, one uint64, may be
 * NULL): the number of edges.  d_tri (may be NULL): when set, the dense triangle as
 * gbd_all_pairs is computed into it and kept, then one streaming pass collects the
 * edges (up to 64 Mi at a time, in 512 MB of scratch) and a lock-free union-find joins
 * them, with direct unions over the triangle for any edges past 64 Mi.  When NULL the
 * triangle is never held: bands of rows are computed in turn into a scratch rectangle
 * of params.band_entries entries (default 512 MB) and each band's hits are joined into the forest before the next band
 * (section 5's graph without the n(n-1)/2 distances in memory).  Asynchronous on
 * `stream`; the scratch is allocated and freed on it. */
int gbd_threshold_components(gbd_ctx *ctx, const gbd_set *set, const gbd_threshold *th, uint32_t *d_labels,
                             uint64_t *d_edges, uint16_t *d_tri, void *stream);

/* The same components from a triangle already computed by gbd_all_pairs for this set
 * (d_tri, n(n-1)/2 entries): one streaming pass, so several thresholds can be explored
 * without recomputing distances. */
int gbd_tri_components(gbd_ctx *ctx, const gbd_set *set, const uint16_t *d_tri, const gbd_threshold *th,
                       uint32_t *d_labels, uint64_t *d_edges, void *stream);

/* ---------------------------------------------------------------- MDS (paper sections 3 and 6.2)
 * Classical multidimensional scaling of the distance triangle: Torgerson's double
 * centering turns the squared distances into the Gram matrix of scalar products
 *   G = -1/2 J (D o D) J,  J = I - 11^T/n            (section 6.2, step 1),
 * whose leading eigenpairs (lambda_a, u_a) give the coordinates X = U Lambda^(1/2)
 * (section 6.2, steps 2-3); the eigenpairs come from a randomized SVD (sections 3.2-3.3, after
 * Halko, Martinsson and Tropp 2011).  Readings: randomized subspace iteration with q
 * rounds (each round multiplies by G twice, G being symmetric, with an
 * orthonormalisation after every product), then B = Q^T G Q and its eigendecomposition;
 * eigenpairs ordered by eigenvalue, largest first; a negative eigenvalue (distances that
 * are not Euclidean) gives zero coordinates.
 *
 * gbd_sqdist_square: W[i*ld + j] = fp16(d_ij^2 * 2^-s) for i, j < n (W[i*ld+i] = 0), and
 *   0 in the padding rows and columns up to ld; d_tri is the device triangle in the layout
 *   of gbd_all_pairs (n(n-1)/2 entries, may be NULL when n < 2); d_w is a device buffer of
 *   ld*ld uint16 (fp16 bit patterns), ld a multiple of 128 and >= n.  s >= 0 is the
 *   smallest shift that keeps the largest squared distance below the fp16 maximum and is
 *   written to *shift (host pointer).  The call synchronises `stream` once to read the
 *   maximum distance.  EINVAL on a NULL pointer or a bad ld.
 * gbd_gram_apply: Y = G X for an n x k float32 row-major X (device), from the W of
 *   gbd_sqdist_square (same n, ld, shift): X is centred and rounded to fp16, W X runs on
 *   the tensor cores with float32 accumulation, the product is centred and scaled by
 *   -2^(s-1).  k is a multiple of 16, 16 <= k <= 256.  Y (device, n x k float32) must not
 *   overlap X.
 * gbd_mds: the whole MDS for an n-read triangle (the paper uses r = 50, section 4.1): r leading eigenvalues into
 *   d_lambda (device, r float32, largest first) and the n x r coordinates into d_coords
 *   (device, float32 row-major).  d_omega is the caller's n x k Gaussian test matrix
 *   (device, float32 row-major; the library draws no random numbers), r <= k, k as above,
 *   k < n, q >= 0 rounds.  Workspace: the fp16 square (ld^2 * 2 bytes with ld = n rounded
 *   up to 128 -- 20 GB at n = 1e5) is kept in the context between calls and reused when
 *   large enough (gbd_trim or gbd_destroy frees it); O(n k) more is allocated on `stream`
 *   and freed before returning; ENOMEM if it does not fit.  The call synchronises `stream`
 *   at its end (it reads back convergence and error flags).  EINVAL on bad sizes. */
int gbd_sqdist_square(gbd_ctx *ctx, const uint16_t *d_tri, uint64_t n, uint16_t *d_w, uint64_t ld,
                      int32_t *shift, void *stream);
int gbd_gram_apply(gbd_ctx *ctx, const uint16_t *d_w, uint64_t n, uint64_t ld, int32_t shift,
                   const float *d_x, uint32_t k, float *d_y, void *stream);
int gbd_mds(gbd_ctx *ctx, const uint16_t *d_tri, uint64_t n, const float *d_omega, uint32_t k,
            uint32_t r, uint32_t q, float *d_lambda, float *d_coords, void *stream);

/* Thread-local text of the last error raised on the calling thread ("" if none; no paper
 * counterpart). */
const char *gbd_last_error(void);

/* Measurement support (no paper counterpart): number of CUDA kernels this library has
 * launched in the process so far (all contexts, all devices). */
uint64_t gbd_kernel_launches(void);

/* Bounds-checked debug build (no paper counterpart).  A library compiled with
 * -DGBD_BOUNDS_CHECK=1 (paper_1803_02272_gb300.build.build(check=True) makes
 * libgbd_check.so beside libgbd.so) checks every distance store, every index into the
 * general kernel's boundary rows and every shared-memory access window of the systolic
 * kernel against the extent of its buffer; an access out of range is skipped, so nothing
 * faults (the results are then wrong, and the violation says where).
 * gbd_bounds_check waits for the device, writes the smallest out-of-range index recorded
 * since its last call, tagged with its site in the top 8 bits (1 systolic store, 2 systolic
 * shared memory, 3 general store, 4 general boundary rows), or UINT64_MAX when there was
 * none, and clears it.  gbd_debug_output_limit caps the output extent that the context's
 * next calls check against (0: the real extent), so a test can make stores run past it.
 * In a build without checks both return ENOTFOUND (*violation = UINT64_MAX). */
int gbd_bounds_check(uint64_t *violation);
int gbd_debug_output_limit(gbd_ctx *ctx, uint64_t limit);

/* Measurement support (no paper counterpart): issue rate of one instruction form of the
 * DP inner loop,
 * in lane operations per second (op codes GBD_PROBE_*), timed with CUDA events
 * on `stream` over `iters` iterations of a saturating kernel. */
#define GBD_PROBE_VIMAX3_S16X2_RELU  0
#define GBD_PROBE_VIADDMAX_S16X2     1
#define GBD_PROBE_VIADDMAX_S16X2_RELU 2
#define GBD_PROBE_VIMAX_S16X2_RELU   3
#define GBD_PROBE_VMAXS2             4
#define GBD_PROBE_PRMT               5
#define GBD_PROBE_IADD3              6
#define GBD_PROBE_LOP3               7
#define GBD_PROBE_IMAX               8
#define GBD_PROBE_HMAX2              9
#define GBD_PROBE_HADD2              10
#define GBD_PROBE_CELL_MIX           11
#define GBD_PROBE_VIMAX3_S16X2       12
#define GBD_PROBE_FMAX               13
#define GBD_PROBE_FMAX3              14
#define GBD_PROBE_FADD               15
#define GBD_PROBE_MIX_DPX_HMAX2      16  /* half the chains DPX, half fp16x2 max */
#define GBD_PROBE_MIX_DPX_FMAX3      17  /* half the chains DPX, half fp32 3-input max */
#define GBD_PROBE_MIX_DPX_IADD3      18  /* half the chains DPX, half 3-input integer add */
#define GBD_PROBE_VIMAX3_U16X2       19  /* unsigned 16x2 3-input max (threshold bounds) */
#define GBD_PROBE_VMINU2             20  /* unsigned 16x2 min, SIMD video form */
#define GBD_PROBE_VSETLEU2           21  /* unsigned 16x2 <= to 0/1 per half, SIMD video form */
#define GBD_PROBE_VIBMIN_U16X2       22  /* unsigned 16x2 min with per-half <= predicates, the
                                            predicate of the high half added back (2 ops) */
#define GBD_PROBE_COUNT              23
int gbd_probe_op_rate(int op, uint32_t iters, double *lane_ops_per_s, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GBD_H */
