// Threshold epilogue (paper sections 4.3 and 5), streamed over distances already in HBM.
//
// A distance d between reads of lengths la, lb is a hit when d <= abs_max and
// d * den <= num * max(la, lb) (integer arithmetic; 97 % homology is num/den = 3/100).
//   * rectangle (section 4.3, sample reads against annotated reference reads): hits are
//     appended to a list through one atomic counter, and each row keeps the one species
//     of all its hits, -2 once two species disagree, -1 with no hit (references with a
//     negative label do not vote);
//   * triangle (section 5, the threshold graph): each hit (i, j) joins i and j in a
//     union-find forest.  A root is only ever hooked under a smaller root, so every
//     component ends with its smallest read as the root; a last pass points every read
//     at its root.
// Both kernels read each distance once (2 bytes; the triangle pass with 16-byte loads
// over the flat triangle) plus the column read's length (cache-resident): they are
// HBM-bound streams.
#include "gbd_internal.cuh"

namespace gbd {
namespace {

__device__ __forceinline__ bool is_hit(uint32_t d, uint32_t la, uint32_t lb, const Threshold &th)
{
    const uint32_t L = la > lb ? la : lb;
    return d <= th.abs_max && (uint64_t)d * th.den <= (uint64_t)th.num * L;
}

// The same test in 32-bit arithmetic, exact when num and den are below 2^16 (d and the
// lengths are below 2^16, so both products fit).
__device__ __forceinline__ bool is_hit32(uint32_t d, uint32_t la, uint32_t lb, const Threshold &th)
{
    const uint32_t L = la > lb ? la : lb;
    return d <= th.abs_max && d * th.den <= th.num * L;
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

// One block per row at a time (rows strided over the grid), threads along the row.
__global__ void __launch_bounds__(256)
rect_epilogue_kernel(const uint16_t *__restrict__ out, uint64_t ld, const uint16_t *__restrict__ lenA, uint64_t a0,
                     uint64_t a1, const uint16_t *__restrict__ lenB, uint64_t b0, uint64_t b1, Threshold th,
                     uint32_t *hits, uint64_t cap, unsigned long long *count, const int32_t *__restrict__ col_labels,
                     int32_t *row_labels)
{
    const uint64_t nb = b1 - b0;
    for (uint64_t r = a0 + blockIdx.x; r < a1; r += gridDim.x) {
        const uint32_t la = lenA[r];
        const uint16_t *row = out + (r - a0) * ld;
        int32_t mine = -1;                       // this thread's view of the row's species
        for (uint64_t c = threadIdx.x; c < nb; c += blockDim.x) {
            const uint32_t d = row[c];
            const uint64_t col = b0 + c;
            if (!is_hit(d, la, lenB[col], th)) continue;
            if (count) {
                const unsigned long long slot = atomicAdd(count, 1ull);
                if (hits && slot < cap) {
                    hits[3 * slot] = (uint32_t)r;
                    hits[3 * slot + 1] = (uint32_t)col;
                    hits[3 * slot + 2] = d;
                }
            }
            if (row_labels) {
                const int32_t s = col_labels[col];
                if (s >= 0) mine = (mine == -1 || mine == s) ? s : -2;
            }
        }
        if (row_labels) {
            // combine the threads' views: -1 is neutral, -2 absorbs, two species give -2
            __shared__ int32_t lab[256];
            lab[threadIdx.x] = mine;
            __syncthreads();
            for (int w = blockDim.x / 2; w > 0; w >>= 1) {
                if ((int)threadIdx.x < w) {
                    const int32_t x = lab[threadIdx.x], y = lab[threadIdx.x + w];
                    lab[threadIdx.x] = (x == -1) ? y : (y == -1 || y == x) ? x : -2;
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) row_labels[r - a0] = lab[0];
            __syncthreads();
        }
    }
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

__device__ __forceinline__ uint64_t tri_row_start(uint64_t i, uint64_t n) { return i * n - i * (i + 1) / 2; }

// (i, j) of flat triangle index k (row-major strict upper triangle of n reads).
__device__ __forceinline__ void tri_unindex(uint64_t k, uint64_t n, uint64_t &i, uint64_t &j)
{
    const double b = 2.0 * (double)n - 1.0;
    int64_t r = (int64_t)((b - sqrt(fmax(b * b - 8.0 * (double)k, 0.0))) * 0.5);
    if (r < 0) r = 0;
    if (r > (int64_t)n - 2) r = (int64_t)n - 2;
    while (r + 1 <= (int64_t)n - 2 && tri_row_start((uint64_t)r + 1, n) <= k) ++r;
    while (r > 0 && tri_row_start((uint64_t)r, n) > k) --r;
    i = (uint64_t)r;
    j = k - tri_row_start(i, n) + i + 1;
}

// Moves (i, j) forward by `steps` entries of the triangle.
__device__ __forceinline__ void tri_advance(uint64_t &i, uint64_t &j, uint64_t steps, uint64_t n)
{
    j += steps;
    while (j >= n && i + 2 < n) {
        const uint64_t over = j - n;           // entries past the end of row i
        ++i;
        j = i + 1 + over;
    }
}

// The triangle as one flat stream: each warp owns a contiguous run of 256-entry spans
// and lane l reads entries 8l .. 8l+7 of a span with one 16-byte load (the triangle must
// be 16-byte aligned).  Hits are appended to an edge list (one atomic per warp and entry
// slot, ballot-aggregated): the unions run afterwards one edge per thread, so a warp
// whose rows are full of hits does not serialise the latency of its unions.  Hits are
// rare, so each lane first tests its eight entries into a bit mask and the warp takes the
// append path only when some lane has one.  Every hit is counted; edges past the list's
// capacity are left to tri_union_rows_kernel.
template <bool NARROW>
__global__ void __launch_bounds__(256)
tri_hits_stream_kernel(const uint16_t *__restrict__ tri, const uint16_t *__restrict__ len, uint64_t n,
                       uint64_t m, Threshold th, uint2 *edges, uint64_t cap, unsigned long long *count)
{
    const uint64_t warp_id = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t spans = (m + 255) / 256;
    const uint64_t per = (spans + nwarps - 1) / nwarps;
    const uint64_t s0 = warp_id * per, s1 = min(spans, s0 + per);
    if (s0 >= s1) return;                      // warp-uniform
    uint64_t i = 0, j = 1;
    const uint64_t k_first = s0 * 256 + 8 * lane;
    if (k_first < m) tri_unindex(k_first, n, i, j);
    const uint4 *t4 = reinterpret_cast<const uint4 *>(tri);
    for (uint64_t sp = s0; sp < s1; ++sp) {
        const uint64_t kb = sp * 256 + 8 * lane;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (kb + 8 <= m) {
            const uint4 v = __ldg(t4 + kb / 8);
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
        } else {
            for (uint64_t e = 0; kb + e < m; ++e) w[e >> 1] |= (uint32_t)tri[kb + e] << (16 * (e & 1));
        }
        // bit e of hmask: entry e is a hit
        uint32_t hmask = 0;
        {
            uint64_t ii = i, jj = j;
            uint32_t lii = (kb < m) ? len[i] : 0u;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (kb + e < m) {
                    const uint32_t d = (w[e >> 1] >> (16 * (e & 1))) & 0xffffu;
                    const uint32_t lj = len[jj];
                    if (NARROW ? is_hit32(d, lii, lj, th) : is_hit(d, lii, lj, th)) hmask |= 1u << e;
                    if (++jj == n) { ++ii; jj = ii + 1; lii = len[ii < n ? ii : 0]; }
                }
            }
        }
        if (__any_sync(0xffffffffu, hmask != 0)) {
            uint64_t ii = i, jj = j;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool hit = (hmask >> e) & 1u;
                const uint32_t mask = __ballot_sync(0xffffffffu, hit);
                if (mask) {
                    unsigned long long base = 0;
                    if (lane == (uint32_t)(__ffs(mask) - 1)) base = atomicAdd(count, (unsigned long long)__popc(mask));
                    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
                    if (hit) {
                        const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
                        if (slot < cap) edges[slot] = make_uint2((uint32_t)ii, (uint32_t)jj);
                    }
                }
                if (kb + e < m && ++jj == n) { ++ii; jj = ii + 1; }
            }
        }
        tri_advance(i, j, 256, n);
    }
}

// Hooks every read of an edge's larger end under its smallest neighbour (atomicMin):
// a valid starting forest (links point to smaller reads of the same component) that
// leaves the unions little to do.
__global__ void min_hook_kernel(const uint2 *__restrict__ edges, uint64_t cap, const unsigned long long *count,
                                uint32_t *parent)
{
    const unsigned long long ne = *count;
    const uint64_t e_end = ne < cap ? ne : cap;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e_end; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 ed = edges[e];            // ed.x < ed.y
        atomicMin(parent + ed.y, ed.x);
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

int check_launch(const char *what)
{
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, what);
}

}  // namespace

int launch_rect_epilogue(const uint16_t *out, uint64_t ld, const DeviceReads &A, uint64_t a0, uint64_t a1,
                         const DeviceReads &B, uint64_t b0, uint64_t b1, const Threshold &th, uint32_t *hits,
                         uint64_t cap, unsigned long long *count, const int32_t *col_labels,
                         int32_t *row_labels, int sm_count, cudaStream_t st)
{
    if (a1 <= a0 || b1 <= b0) return GBD_OK;
    if (!count && !(row_labels && col_labels)) return GBD_OK;
    rect_epilogue_kernel<<<grid_of(a1 - a0, sm_count, 8), 256, 0, st>>>(
        out, ld, A.len, a0, a1, B.len, b0, b1, th, hits, cap, count, col_labels, row_labels && col_labels ? row_labels : nullptr);
    return check_launch("rect_epilogue_kernel launch");
}

int launch_tri_components(const uint16_t *tri, const DeviceReads &S, const Threshold &th, uint32_t *parent,
                          unsigned long long *count, int sm_count, cudaStream_t st)
{
    const uint64_t n = S.n;
    iota_kernel<<<grid_of((n + 255) / 256, sm_count, 16), 256, 0, st>>>(parent, n);
    int rc = check_launch("iota_kernel launch");
    if (rc != GBD_OK) return rc;
    if (n >= 2) {
        const uint64_t m = n * (n - 1) / 2;
        if (reinterpret_cast<uintptr_t>(tri) % 16 == 0) {
            // edge list of up to kEdgeCap hits, then one union per edge; the row kernel
            // takes over only if the list overflowed
            const uint64_t cap = std::min<uint64_t>(m, kEdgeCap);
            uint2 *edges = nullptr;
            unsigned long long *cnt = nullptr;
            GBD_CUDA_TRY(cudaMallocAsync((void **)&edges, cap * sizeof(uint2), st));
            GBD_CUDA_TRY(cudaMallocAsync((void **)&cnt, sizeof(unsigned long long), st));
            GBD_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
            const int grid = grid_of((m + 255) / 256, sm_count, 8);
            if (th.num < 65536u && th.den < 65536u)
                tri_hits_stream_kernel<true><<<grid, 256, 0, st>>>(tri, S.len, n, m, th, edges, cap, cnt);
            else
                tri_hits_stream_kernel<false><<<grid, 256, 0, st>>>(tri, S.len, n, m, th, edges, cap, cnt);
            rc = check_launch("tri_hits_stream_kernel launch");
            if (rc == GBD_OK) {
                min_hook_kernel<<<grid_of((cap + 255) / 256, sm_count, 16), 256, 0, st>>>(edges, cap, cnt, parent);
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
