// Threshold epilogue (paper sections 4.3 and 5), streamed over distances already in HBM.
//
// A distance d between reads of lengths la, lb is a hit when d <= abs_max and
// d * den <= num * max(la, lb) (integer arithmetic; 97 % homology is num/den = 3/100).
//   * rectangle (section 4.3, sample reads against annotated reference reads): hits are
//     appended to a list (one atomic per warp on its counter), and each row keeps the one species
//     of all its hits, -2 once two species disagree, -1 with no hit (references with a
//     negative label do not vote);
//   * triangle (section 5, the threshold graph): each hit (i, j) joins i and j in a
//     union-find forest.  A root is only ever hooked under a smaller root, so every
//     component ends with its smallest read as the root; a last pass points every read
//     at its root.
// Both streams read each distance once with 16-byte loads and test it against a table of
// per-read bounds (hit_bound), two entries per packed 16-bit instruction instead of a
// multiply-compare per entry.
#include "gbd_internal.cuh"

namespace gbd {
namespace {

__device__ __forceinline__ bool is_hit(uint32_t d, uint32_t la, uint32_t lb, const Threshold &th)
{
    const uint32_t L = la > lb ? la : lb;
    return d <= th.abs_max && (uint64_t)d * th.den <= (uint64_t)th.num * L;
}

__device__ __forceinline__ uint32_t uf_load(const uint32_t *p)
{
    return *reinterpret_cast<const volatile uint32_t *>(p);
}

// Root of x, halving the path on the way.  Links only ever point to smaller indices of
// the same set, and the halving store only rewrites a non-root's link to one of its
// ancestors, so it may race with other halvings (any ancestor is a valid link) and never
// meets a hook (hooks change roots only): a plain store suffices, and unlike an atomic
// it does not serialise the many threads that walk the same hot path.
__device__ __forceinline__ uint32_t uf_find(uint32_t *parent, uint32_t x)
{
    for (;;) {
        const uint32_t p = uf_load(parent + x);
        if (p == x) return x;
        const uint32_t gp = uf_load(parent + p);
        if (gp != p) *reinterpret_cast<volatile uint32_t *>(parent + x) = gp;
        x = p;
    }
}

__device__ __forceinline__ void uf_union(uint32_t *parent, uint32_t a, uint32_t b)
{
    for (;;) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a < b) { const uint32_t t = a; a = b; b = t; }
        if (atomicCAS(parent + a, a, b) == a) return;     // a was still a root
    }
}

// Largest distance that can be a hit when a read of length `len` is the longer of the
// pair: min(abs_max, floor(num * len / den)), at most 65535.  It is non-decreasing in the
// length, so the hit rule for reads of lengths la, lb is d <= max(bound(la), bound(lb)).
__device__ __forceinline__ uint32_t hit_bound(uint32_t len, const Threshold &th)
{
    uint64_t q = th.num <= 0xffffu ? (uint64_t)((th.num * len) / th.den)   // len < 2^16: fits 32 bits
                                   : (uint64_t)th.num * len / th.den;
    if (q > th.abs_max) q = th.abs_max;
    return q > 65535u ? 65535u : (uint32_t)q;
}

// T[j] = hit_bound(len[j]) for j < n, 0 for the padding up to n_pad.
__global__ void hit_bound_kernel(const uint16_t *__restrict__ len, uint64_t n, uint64_t n_pad, Threshold th,
                                 uint16_t *T)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += (uint64_t)gridDim.x * blockDim.x)
        T[j] = j < n ? (uint16_t)hit_bound(len[j], th) : (uint16_t)0;
}

// Hit mask of eight distances of one row (w: two per word, the first in the low half)
// against the row's bound ti and the column bounds T[j .. j+7]: bit e set when entry e
// is a hit.  Two entries per instruction: the column bounds arrive as packed pairs (a
// 16-bit funnel shift when j is odd), the per-pair bound is a packed 3-way max and the
// test a packed min that also yields (d <= bound) per half as predicates (DPX
// instructions on this GPU; the older SIMD video intrinsics are emulated in software).
// T must be 4-byte aligned with T[j + 9] readable.
__device__ __forceinline__ uint32_t hits8(const uint32_t w[4], uint32_t ti, const uint16_t *__restrict__ T, uint64_t j)
{
    const uint32_t *Tw = reinterpret_cast<const uint32_t *>(T) + (j >> 1);
    const uint32_t sh = (uint32_t)(j & 1) * 16u;
    uint32_t W[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) W[k] = __ldg(Tw + k);
    const uint32_t ti2 = ti * 0x10001u;
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t t = __funnelshift_r(W[k], W[k + 1], sh);
        bool hi, lo;
        (void)__vibmin_u16x2(w[k], __vimax3_u16x2(ti2, t, t), &hi, &lo);
        m |= ((uint32_t)lo | ((uint32_t)hi << 1)) << (2 * k);
    }
    return m;
}

// Reserves `cnt` consecutive slots for each lane of a full warp with one atomic: returns
// the lane's first slot.
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long *count, uint32_t cnt)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(count, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (incl - cnt);
}

// Row label lattice: -1 (no vote yet) is neutral, -2 (ambiguous) absorbs, two different
// species give -2.
__device__ __forceinline__ int32_t label_join(int32_t x, int32_t y)
{
    return x == -1 ? y : (y == -1 || y == x) ? x : -2;
}

// Joins v into *p.  Every successful exchange moves *p up the three-level lattice, so the
// loop retries at most twice after a lost race.
__device__ __forceinline__ void label_join_atomic(int32_t *p, int32_t v)
{
    if (v == -1) return;
    int32_t old = *reinterpret_cast<volatile int32_t *>(p);
    for (int it = 0; it < 4; ++it) {
        const int32_t nv = label_join(old, v);
        if (nv == old) return;
        const int32_t prev = atomicCAS(p, old, nv);
        if (prev == old) return;
        old = prev;
    }
}

constexpr uint32_t kSegVec = 1024;         // 8-entry vectors per work unit (8,192 entries)
constexpr int kVecPerLane = 4;             // vectors per lane per iteration

// Where a pass's hits go.
struct RectOut {
    uint32_t *hits;                 // (row, col, d) triples, or
    uint2 *edges;                   // (row, col) pairs (when set)
    uint64_t cap;
    unsigned long long *count;      // every hit counted, also past cap
    const int32_t *col_labels;      // species of column b0 + c (annotation), with
    int32_t *row_labels;            // the label of row a0 + rr (pre-set to -1)
};

// The rows a pass streams over.  Row rr of the pass is read a0 + rr; its entry for column
// b0 + c lies at:
//   SPAN_RECT  out[rr * ld + c], c in [0, nb)
//   SPAN_BAND  out[rr * ld + c], c in [rr, nb) (row a0 + rr of a triangle band: columns
//              after the row's own read)
//   SPAN_TRI   the strict upper triangle of nb reads (a0 = b0 = 0): out[k(rr, c)], c in
//              [rr + 1, nb)
enum SpanKind : int { SPAN_RECT = 0, SPAN_BAND = 1, SPAN_TRI = 2 };

struct Spans {
    const uint16_t *out;
    uint64_t ld, rows, nb, a0, b0;
};

// One row of a pass: entries start at p (column b0 + c_lo); vectors of 8 entries run from
// the row's first 16-byte boundary; head entries come before it, tail entries after the
// last full vector.
struct RowSpan {
    const uint16_t *p;
    uint64_t c_lo, head, nvec, tail0, nbr;
};

template <int KIND>
__device__ __forceinline__ RowSpan row_span(const Spans &S, uint64_t rr)
{
    RowSpan rs;
    if (KIND == SPAN_TRI) {
        rs.c_lo = rr + 1;
        rs.nbr = S.nb - 1 - rr;
        rs.p = S.out + (rr * S.nb - rr * (rr + 1) / 2);
    } else {
        rs.c_lo = KIND == SPAN_BAND ? rr : 0;
        rs.nbr = S.nb > rs.c_lo ? S.nb - rs.c_lo : 0;
        rs.p = S.out + rr * S.ld + rs.c_lo;
    }
    uint64_t head = ((16u - (uint32_t)(reinterpret_cast<uintptr_t>(rs.p) & 15u)) & 15u) / 2u;
    rs.head = head > rs.nbr ? rs.nbr : head;
    rs.nvec = (rs.nbr - rs.head) / 8;
    rs.tail0 = rs.head + 8 * rs.nvec;
    return rs;
}

// Records one hit at `slot` (already reserved).
__device__ __forceinline__ void put_hit(const RectOut &o, unsigned long long slot, uint32_t r, uint32_t col, uint32_t d)
{
    if (slot >= o.cap) return;
    if (o.edges) {
        o.edges[slot] = make_uint2(r, col);
    } else if (o.hits) {
        o.hits[3 * slot] = r;
        o.hits[3 * slot + 1] = col;
        o.hits[3 * slot + 2] = d;
    }
}

// Smallest of the eight distances of a vector, in both halves of the result's pair of
// packed minima (the caller takes the smaller half).
__device__ __forceinline__ uint32_t vmin8(const uint4 &x)
{
    return __vminu2(__vminu2(x.x, x.y), __vminu2(x.z, x.w));
}

__device__ __forceinline__ uint32_t half_min(uint32_t m) { return min(m & 0xffffu, m >> 16); }

// The rows of a pass as (row, segment) work units of kSegVec vectors, each owned by one
// warp (units strided over all warps of the grid, segment-major so that the warps of a
// block work on the same columns and share their bounds in L1; no block-wide
// synchronisation); the warp of a row's segment 0 also takes the row's (fewer than 16)
// head and tail entries.  A hit needs d <= max(row bound, column bound) <= thr =
// max(row bound, tcap), tcap the bound of the longest column read, so a lane takes the
// minimum of each of its four vectors (packed 16-bit mins) and only vectors whose minimum
// is at most thr are candidates.  Candidates are appended to a per-warp queue in shared
// memory (vector and index) and tested against the column bound table 32 at a time, one
// per lane, so the exact test runs with every lane busy however the candidates are
// spread; the queue is drained at the end of each unit (its entries share the unit's
// row).  The four vectors of the next iteration are loaded before the current ones are
// filtered.  Hits are appended with one atomic per warp; for the annotation, a unit's
// species view is combined in the warp and joined into the row's label.  Column bounds:
// TB[toff + c] = hit_bound of column b0 + c (TB 4-byte aligned, toff 0 or 1, readable 10
// entries past the last column).
constexpr int kQueue = 64;                 // candidate queue entries per warp (a power of two)
constexpr int kSpanWarps = 8;              // warps per block

template <int KIND>
__global__ void __launch_bounds__(kSpanWarps * 32)
span_epilogue_kernel(Spans S, const uint16_t *__restrict__ lenA, const uint16_t *__restrict__ TB, uint32_t toff,
                     uint32_t tcap, Threshold th, RectOut o)
{
    __shared__ uint4 qx[kSpanWarps][kQueue];
    __shared__ uint32_t qv[kSpanWarps][kQueue];
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t warp_id = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t maxrow = KIND == SPAN_TRI ? S.nb - 1 : S.nb;      // longest row
    const uint32_t nseg = (uint32_t)(((maxrow + 7) / 8 + kSegVec - 1) / kSegVec);
    const uint64_t units = S.rows * nseg;
    const bool want_hits = o.count != nullptr;
    const bool want_labels = o.row_labels != nullptr;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (uint64_t u = warp_id; u < units; u += nwarps) {
        const uint32_t seg = (uint32_t)(u / S.rows);
        const uint64_t rr = u - (uint64_t)seg * S.rows;
        const RowSpan rs = row_span<KIND>(S, rr);
        const uint32_t v0 = seg * kSegVec;
        if (seg > 0 && v0 >= rs.nvec) continue;                        // warp-uniform
        const uint64_t r = S.a0 + rr;
        const uint32_t ti = hit_bound(lenA[r], th);
        const uint32_t thr = max(ti, tcap);
        const uint64_t cb = S.b0 + rs.c_lo;          // column of the row's entry 0
        const uint64_t tb = toff + rs.c_lo;          // its index in TB
        int32_t mine = -1;
        const uint32_t v1 = (uint32_t)min(rs.nvec, (uint64_t)v0 + kSegVec);
        const uint4 *pv = reinterpret_cast<const uint4 *>(rs.p + rs.head);
        // TB from an even index at or before the bound of the row's vector 0 (so 32-bit
        // loads stay aligned), and that bound's offset from there
        const uint64_t t0 = tb + rs.head;
        const uint16_t *tbv = TB + (t0 & ~1ull);
        const uint32_t par = (uint32_t)(t0 & 1);
        // the hits of one lane's vector v (mask hm, data x); called by the whole warp
        auto take = [&](uint32_t v, const uint4 &x, uint32_t hm) {
            if (!__any_sync(0xffffffffu, hm != 0)) return;
            const uint64_t c = rs.head + 8 * (uint64_t)v;
            unsigned long long slot = want_hits ? warp_reserve(o.count, __popc(hm)) : 0;
            const uint64_t lo = (uint64_t)x.y << 32 | x.x, hi = (uint64_t)x.w << 32 | x.z;
            while (hm) {
                const int e = __ffs(hm) - 1;
                hm &= hm - 1;
                const uint32_t d = (uint32_t)(((e < 4) ? lo : hi) >> (16 * (e & 3))) & 0xffffu;
                const uint64_t col = cb + c + e;
                if (want_hits) put_hit(o, slot++, (uint32_t)r, (uint32_t)col, d);
                if (want_labels) {
                    const int32_t sp = o.col_labels[col];
                    if (sp >= 0) mine = label_join(mine, sp);
                }
            }
        };
        // the queue: entries [qhead, qtail) (indices mod kQueue), fewer than 32 between batches
        uint32_t qhead = 0, qtail = 0;
        auto test_batch = [&](uint32_t cnt) {        // the oldest cnt (<= 32) queued candidates
            uint32_t hm = 0, v = 0;
            uint4 x = make_uint4(0u, 0u, 0u, 0u);
            if (lane < cnt) {
                const uint32_t slot = (qhead + lane) & (kQueue - 1);
                x = qx[wib][slot];
                v = qv[wib][slot];
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
                hm = hits8(w, ti, tbv, 8 * (uint64_t)v + par);
            }
            take(v, x, hm);
            qhead += cnt;
        };
        constexpr uint32_t kStep = 32 * kVecPerLane;
        auto load = [&](uint32_t vb, uint4 (&x)[kVecPerLane]) {
#pragma unroll
            for (int k = 0; k < kVecPerLane; ++k) {
                const uint32_t v = vb + 32 * k + lane;
                x[k] = v < v1 ? __ldg(pv + v) : make_uint4(~0u, ~0u, ~0u, ~0u);
            }
        };
        uint4 nx[kVecPerLane];
        load(v0, nx);
        for (uint32_t vb = v0; vb < v1; vb += kStep) {
            uint4 x[kVecPerLane];
#pragma unroll
            for (int k = 0; k < kVecPerLane; ++k) x[k] = nx[k];
            if (vb + kStep < v1) load(vb + kStep, nx);             // next iteration's loads first
#pragma unroll
            for (int k = 0; k < kVecPerLane; ++k) {
                const uint32_t v = vb + 32 * k + lane;
                const bool cand = v < v1 && half_min(vmin8(x[k])) <= thr;
                const uint32_t cm = __ballot_sync(0xffffffffu, cand);
                if (cm == 0) continue;
                if (cand) {
                    const uint32_t slot = (qtail + __popc(cm & lt_mask)) & (kQueue - 1);
                    qx[wib][slot] = x[k];
                    qv[wib][slot] = v;
                }
                qtail += __popc(cm);
                __syncwarp();
                if (qtail - qhead >= 32) {
                    test_batch(32);
                    __syncwarp();
                }
            }
        }
        if (qtail != qhead) test_batch(qtail - qhead);
        // entries before the first boundary and after the last vector: the warp of segment 0
        if (seg == 0) {
            const uint64_t ntail = rs.nbr - rs.tail0;
            uint32_t hit = 0, d = 0;
            uint64_t c = 0;
            if (lane < rs.head + ntail) {
                c = lane < rs.head ? lane : rs.tail0 + (lane - rs.head);
                d = rs.p[c];
                hit = d <= max(ti, (uint32_t)TB[tb + c]);
            }
            if (__any_sync(0xffffffffu, hit)) {
                const unsigned long long slot = want_hits ? warp_reserve(o.count, hit) : 0;
                if (hit) {
                    if (want_hits) put_hit(o, slot, (uint32_t)r, (uint32_t)(cb + c), d);
                    if (want_labels) {
                        const int32_t sp = o.col_labels[cb + c];
                        if (sp >= 0) mine = label_join(mine, sp);
                    }
                }
            }
        }
        if (want_labels) {
#pragma unroll
            for (int k = 16; k > 0; k >>= 1) mine = label_join(mine, __shfl_xor_sync(0xffffffffu, mine, k));
            if (lane == 0) label_join_atomic(o.row_labels + rr, mine);
        }
        __syncwarp();
    }
}

// Direct unions over a triangle band (layout SPAN_BAND of span_epilogue_kernel),
// one block per row; runs only when the band's edge list overflowed (*count > cap).
__global__ void __launch_bounds__(256)
band_union_rows_kernel(const uint16_t *__restrict__ out, uint64_t ld, const uint16_t *__restrict__ T,
                       uint64_t a0, uint64_t a1, uint64_t b0, uint64_t nb, uint32_t *parent,
                       const unsigned long long *count, uint64_t cap)
{
    if (*count <= cap) return;
    for (uint64_t rr = blockIdx.x; rr < a1 - a0; rr += gridDim.x) {
        const uint64_t r = a0 + rr;
        const uint32_t ti = T[r];
        for (uint64_t c = rr + threadIdx.x; c < nb; c += blockDim.x) {
            const uint64_t col = b0 + c;
            if (out[rr * ld + c] <= max(ti, (uint32_t)T[col])) uf_union(parent, (uint32_t)r, (uint32_t)col);
        }
    }
}

// total += *count; *count = 0 (one thread).
__global__ void band_total_kernel(unsigned long long *count, unsigned long long *total)
{
    *total += *count;
    *count = 0;
}

__global__ void iota_kernel(uint32_t *a, uint64_t n)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        a[i] = (uint32_t)i;
}

// Rows of the triangle strided over the grid (long and short rows interleave), threads
// along the row; every hit joins its two reads.
__global__ void __launch_bounds__(256)
tri_union_kernel(const uint16_t *__restrict__ tri, const uint16_t *__restrict__ len, uint64_t n, Threshold th,
                 uint32_t *parent, unsigned long long *count)
{
    unsigned long long local = 0;
    for (uint64_t i = blockIdx.x; i + 1 < n; i += gridDim.x) {
        const uint64_t base = i * n - i * (i + 1) / 2;       // k(i, i+1)
        const uint32_t li = len[i];
        for (uint64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
            const uint32_t d = tri[base + (j - i - 1)];
            if (!is_hit(d, li, len[j], th)) continue;
            ++local;
            uf_union(parent, (uint32_t)i, (uint32_t)j);
        }
    }
    if (count) {
        for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
        if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
    }
}

// Pre-hooks the larger end y of each edge (x, y), x < y, under x before the unions run.
// On a fresh forest (every read its own root, FRESH) y goes under its smallest neighbour
// (atomicMin): every link is then an edge of the graph, and all edges are unioned next,
// so no connection is lost.  On a forest that earlier unions have built, a link may stand
// for an edge no longer in any list, so only a root is hooked (compare-and-swap from
// itself), which is an ordinary union step.  Either way links point to smaller reads of
// the same component.
template <bool FRESH>
__global__ void min_hook_kernel(const uint2 *__restrict__ edges, uint64_t cap, const unsigned long long *count,
                                uint32_t *parent)
{
    const unsigned long long ne = *count;
    const uint64_t e_end = ne < cap ? ne : cap;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e_end; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 ed = edges[e];            // ed.x < ed.y
        if (FRESH) atomicMin(parent + ed.y, ed.x);
        else atomicCAS(parent + ed.y, ed.y, ed.x);
    }
}

// One edge per thread.
__global__ void union_edges_kernel(const uint2 *__restrict__ edges, uint64_t cap, const unsigned long long *count,
                                   uint32_t *parent)
{
    const unsigned long long ne = *count;
    const uint64_t e_end = ne < cap ? ne : cap;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e_end; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 ed = edges[e];
        uf_union(parent, ed.x, ed.y);
    }
}

// Rows of the triangle, each hit joined directly; with `only_if_over` it runs only when
// the edge list overflowed (*count > cap), as the fallback for the edges it could not hold
// (unions are idempotent, so redoing the others is harmless).
__global__ void __launch_bounds__(256)
tri_union_rows_kernel(const uint16_t *__restrict__ tri, const uint16_t *__restrict__ len, uint64_t n, Threshold th,
                      uint32_t *parent, const unsigned long long *count, uint64_t cap)
{
    if (count && *count <= cap) return;
    for (uint64_t i = blockIdx.x; i + 1 < n; i += gridDim.x) {
        const uint64_t base = i * n - i * (i + 1) / 2;
        const uint32_t li = len[i];
        for (uint64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
            if (is_hit(tri[base + (j - i - 1)], li, len[j], th)) uf_union(parent, (uint32_t)i, (uint32_t)j);
        }
    }
}

__global__ void flatten_kernel(uint32_t *parent, uint64_t n)
{
    // every union has completed (earlier kernel on the stream): roots are final, and a
    // path link only changes to another node of the same path
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        parent[i] = uf_find(parent, (uint32_t)i);
}

constexpr uint64_t kEdgeCap = 64ull << 20;   // edges held between the two phases (512 MB)

int grid_of(uint64_t work, int sm_count, int per_sm)
{
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(work, (uint64_t)std::max(sm_count, 1) * per_sm));
}

// One resident wave of `kernel` (blocks of 256 threads): the streams give every block
// (or warp) an equal share up front, so a partial second wave would double their time.
template <typename K>
int resident_grid(K kernel, int sm_count, uint64_t work)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return grid_of(work, sm_count, per_sm);
}

int check_launch(const char *what)
{
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, what);
}

}  // namespace

// The span kernel counts a row's vectors in 32 bits.
static bool span_units_fit(uint64_t rows, uint64_t maxrow)
{
    (void)rows;
    return maxrow / 8 < (1ull << 32) - kSegVec;
}

// Blocks of 256 threads (8 warps, one work unit each at a time) for a pass.
static uint64_t span_units(uint64_t rows, uint64_t maxrow)
{
    return (rows * (((maxrow + 7) / 8 + kSegVec - 1) / kSegVec) + 7) / 8;
}

// hit_bound on the host: the bound of the longest column read caps every column bound.
static uint32_t host_hit_bound(uint32_t len, const Threshold &th)
{
    uint64_t q = (uint64_t)th.num * len / th.den;
    if (q > th.abs_max) q = th.abs_max;
    return q > 65535u ? 65535u : (uint32_t)q;
}

int launch_rect_epilogue(const uint16_t *out, uint64_t ld, const DeviceReads &A, uint64_t a0, uint64_t a1,
                         const DeviceReads &B, uint64_t b0, uint64_t b1, uint32_t colmax_len, const Threshold &th,
                         uint32_t *hits, uint64_t cap, unsigned long long *count, const int32_t *col_labels,
                         int32_t *row_labels, int sm_count, cudaStream_t st)
{
    if (a1 <= a0 || b1 <= b0) return GBD_OK;
    if (!count && !(row_labels && col_labels)) return GBD_OK;
    if (!span_units_fit(a1 - a0, b1 - b0)) return fail(GBD_EINVAL, "rectangle too large for one epilogue pass");
    // bounds of columns b0 - toff .. b1 - 1 (toff makes the table's first word hold an
    // even column, so its 32-bit loads are aligned), zero padding after
    const uint64_t nb = b1 - b0;
    const uint32_t toff = (uint32_t)(b0 & 1);
    const uint64_t nt = nb + toff, nt_pad = nt + 16;
    uint16_t *TB = nullptr;
    GBD_CUDA_TRY(cudaMallocAsync((void **)&TB, nt_pad * sizeof(uint16_t), st));
    hit_bound_kernel<<<grid_of((nt_pad + 255) / 256, sm_count, 8), 256, 0, st>>>(B.len + (b0 - toff), nt, nt_pad, th,
                                                                                  TB);
    int rc = check_launch("hit_bound_kernel launch");
    if (rc == GBD_OK) {
        const RectOut o{hits, nullptr, cap, count, col_labels, row_labels && col_labels ? row_labels : nullptr};
        const Spans S{out, ld, a1 - a0, nb, a0, b0};
        span_epilogue_kernel<SPAN_RECT>
            <<<resident_grid(span_epilogue_kernel<SPAN_RECT>, sm_count, span_units(a1 - a0, nb)), 256, 0, st>>>(
                S, A.len, TB, toff, host_hit_bound(colmax_len, th), th, o);
        rc = check_launch("span_epilogue_kernel launch");
    }
    cudaFreeAsync(TB, st);
    return rc;
}

int band_forest_begin(BandForest &bf, const DeviceReads &S, const Threshold &th, uint32_t *parent, uint64_t max_entries,
                      int sm_count, cudaStream_t st)
{
    const uint64_t n = S.n;
    bf = BandForest{};
    bf.cap = std::max<uint64_t>(1, std::min<uint64_t>(max_entries, kEdgeCap));
    iota_kernel<<<grid_of((n + 255) / 256, sm_count, 16), 256, 0, st>>>(parent, n);
    int rc = check_launch("iota_kernel launch");
    if (rc != GBD_OK) return rc;
    GBD_CUDA_TRY(cudaMallocAsync((void **)&bf.T, (n + 16) * sizeof(uint16_t), st));
    GBD_CUDA_TRY(cudaMallocAsync((void **)&bf.edges, bf.cap * sizeof(uint2), st));
    GBD_CUDA_TRY(cudaMallocAsync((void **)&bf.cnt, 2 * sizeof(unsigned long long), st));
    GBD_CUDA_TRY(cudaMemsetAsync(bf.cnt, 0, 2 * sizeof(unsigned long long), st));
    hit_bound_kernel<<<grid_of((n + 16 + 255) / 256, sm_count, 8), 256, 0, st>>>(S.len, n, n + 16, th, bf.T);
    return check_launch("hit_bound_kernel launch");
}

int band_forest_add(BandForest &bf, const uint16_t *rect, uint64_t ld, const DeviceReads &S, uint64_t a0, uint64_t a1,
                    uint32_t max_len, const Threshold &th, uint32_t *parent, int sm_count, cudaStream_t st)
{
    const uint64_t n = S.n;
    if (a1 <= a0 || a0 + 1 >= n) return GBD_OK;
    const uint64_t b0 = a0 + 1, nb = n - b0;
    if (!span_units_fit(a1 - a0, nb)) return fail(GBD_EINVAL, "band too large for one epilogue pass");
    const uint32_t toff = (uint32_t)(b0 & 1);
    const RectOut o{nullptr, bf.edges, bf.cap, bf.cnt, nullptr, nullptr};
    const Spans Sp{rect, ld, a1 - a0, nb, a0, b0};
    span_epilogue_kernel<SPAN_BAND>
        <<<resident_grid(span_epilogue_kernel<SPAN_BAND>, sm_count, span_units(a1 - a0, nb)), 256, 0, st>>>(
            Sp, S.len, bf.T + (b0 - toff), toff, host_hit_bound(max_len, th), th, o);
    int rc = check_launch("span_epilogue_kernel launch");
    const int eg = grid_of((bf.cap + 255) / 256, sm_count, 16);
    if (rc == GBD_OK) {
        if (bf.first) min_hook_kernel<true><<<eg, 256, 0, st>>>(bf.edges, bf.cap, bf.cnt, parent);
        else min_hook_kernel<false><<<eg, 256, 0, st>>>(bf.edges, bf.cap, bf.cnt, parent);
        rc = check_launch("min_hook_kernel launch");
    }
    if (rc == GBD_OK) {
        union_edges_kernel<<<eg, 256, 0, st>>>(bf.edges, bf.cap, bf.cnt, parent);
        rc = check_launch("union_edges_kernel launch");
    }
    if (rc == GBD_OK) {
        band_union_rows_kernel<<<grid_of(a1 - a0, sm_count, 8), 256, 0, st>>>(rect, ld, bf.T, a0, a1, b0, nb, parent,
                                                                                bf.cnt, bf.cap);
        rc = check_launch("band_union_rows_kernel launch");
    }
    if (rc == GBD_OK) {
        band_total_kernel<<<1, 1, 0, st>>>(bf.cnt, bf.cnt + 1);
        rc = check_launch("band_total_kernel launch");
    }
    bf.first = false;
    return rc;
}

int band_forest_end(BandForest &bf, uint32_t *parent, uint64_t n, unsigned long long *count, int sm_count,
                    cudaStream_t st)
{
    int rc = GBD_OK;
    if (bf.cnt) {
        flatten_kernel<<<grid_of((n + 255) / 256, sm_count, 16), 256, 0, st>>>(parent, n);
        rc = check_launch("flatten_kernel launch");
        if (rc == GBD_OK && count) {
            const cudaError_t e = cudaMemcpyAsync(count, bf.cnt + 1, sizeof(unsigned long long),
                                                  cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync");
        }
    }
    if (bf.T) cudaFreeAsync(bf.T, st);
    if (bf.edges) cudaFreeAsync(bf.edges, st);
    if (bf.cnt) cudaFreeAsync(bf.cnt, st);
    bf = BandForest{};
    return rc;
}

int launch_tri_components(const uint16_t *tri, const DeviceReads &S, uint32_t max_len, const Threshold &th,
                          uint32_t *parent, unsigned long long *count, int sm_count, cudaStream_t st)
{
    const uint64_t n = S.n;
    iota_kernel<<<grid_of((n + 255) / 256, sm_count, 16), 256, 0, st>>>(parent, n);
    int rc = check_launch("iota_kernel launch");
    if (rc != GBD_OK) return rc;
    if (n >= 2) {
        const uint64_t m = n * (n - 1) / 2;
        if (reinterpret_cast<uintptr_t>(tri) % 2 == 0 && span_units_fit(n - 1, n - 1)) {
            // edge list of up to kEdgeCap hits, then one union per edge; the row kernel
            // takes over only if the list overflowed
            const uint64_t cap = std::min<uint64_t>(m, kEdgeCap);
            uint2 *edges = nullptr;
            unsigned long long *cnt = nullptr;
            GBD_CUDA_TRY(cudaMallocAsync((void **)&edges, cap * sizeof(uint2), st));
            GBD_CUDA_TRY(cudaMallocAsync((void **)&cnt, sizeof(unsigned long long), st));
            GBD_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
            uint16_t *T = nullptr;
            GBD_CUDA_TRY(cudaMallocAsync((void **)&T, (n + 16) * sizeof(uint16_t), st));
            hit_bound_kernel<<<grid_of((n + 16 + 255) / 256, sm_count, 8), 256, 0, st>>>(S.len, n, n + 16, th, T);
            rc = check_launch("hit_bound_kernel launch");
            if (rc == GBD_OK) {
                const RectOut o{nullptr, edges, cap, cnt, nullptr, nullptr};
                const Spans Sp{tri, 0, n - 1, n, 0, 0};
                span_epilogue_kernel<SPAN_TRI>
                    <<<resident_grid(span_epilogue_kernel<SPAN_TRI>, sm_count, span_units(n - 1, n - 1)), 256, 0, st>>>(
                        Sp, S.len, T, 0, host_hit_bound(max_len, th), th, o);
                rc = check_launch("span_epilogue_kernel launch");
            }
            cudaFreeAsync(T, st);
            if (rc == GBD_OK) {
                min_hook_kernel<true><<<grid_of((cap + 255) / 256, sm_count, 16), 256, 0, st>>>(edges, cap, cnt, parent);
                rc = check_launch("min_hook_kernel launch");
            }
            if (rc == GBD_OK) {
                union_edges_kernel<<<grid_of((cap + 255) / 256, sm_count, 16), 256, 0, st>>>(edges, cap, cnt, parent);
                rc = check_launch("union_edges_kernel launch");
            }
            if (rc == GBD_OK) {
                tri_union_rows_kernel<<<grid_of(n - 1, sm_count, 8), 256, 0, st>>>(tri, S.len, n, th, parent, cnt, cap);
                rc = check_launch("tri_union_rows_kernel launch");
            }
            if (rc == GBD_OK && count) {
                cudaError_t e = cudaMemcpyAsync(count, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync");
            }
            cudaFreeAsync(edges, st);
            cudaFreeAsync(cnt, st);
            if (rc != GBD_OK) return rc;
        } else {
            tri_union_kernel<<<grid_of(n - 1, sm_count, 8), 256, 0, st>>>(tri, S.len, n, th, parent, count);
            if ((rc = check_launch("tri_union_kernel launch")) != GBD_OK) return rc;
        }
    }
    flatten_kernel<<<grid_of((n + 255) / 256, sm_count, 16), 256, 0, st>>>(parent, n);
    return check_launch("flatten_kernel launch");
}

}  // namespace gbd
