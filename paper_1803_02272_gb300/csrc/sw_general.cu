// General pair kernel: one read pair per thread, any lengths (<= 65535), any scores.
//
// Smith-Waterman local score (paper section 2.2) by the textbook recurrence
//   H(i,j) = max(0, H(i-1,j-1) + s(a_i,b_j), H(i-1,j) - gap, H(i,j-1) - gap)
// (or its affine-gap form, below),
// S = max H, converted to a distance in the epilogue.  The query read is swept in
// strips of R rows held in registers; the strip's last row is handed to the next
// strip through a per-thread boundary row in scratch memory, laid out column-major
// over threads ([column][thread]) so a warp's loads and stores are coalesced.
// This kernel is the path for reads longer than the systolic kernel's limit, for
// non-default scores, and the simple baseline the fast kernel is checked against.
#include <algorithm>

#include "gbd_internal.cuh"

namespace gbd {
namespace {

// Query rows per strip, held in registers.  Each strip passes its last row to the next
// through the boundary rows in scratch (4 bytes read and written per column, twice with
// affine gaps), so a taller strip cuts that traffic per cell.
constexpr int kStrip = 16;

__device__ __forceinline__ uint32_t base_at(const uint32_t *w, uint32_t k)
{
    return (__ldg(w + (k >> 4)) >> ((k & 15u) * 2u)) & 3u;
}

__device__ __forceinline__ uint64_t tri_row_start(uint64_t i, uint64_t n)
{
    return i * n - i * (i + 1) / 2;
}

// Row i of the strict upper triangle holding linear index k.
__device__ __forceinline__ void tri_unindex(uint64_t k, uint64_t n, uint64_t &i, uint64_t &j)
{
    const double b = 2.0 * (double)n - 1.0;
    double disc = b * b - 8.0 * (double)k;
    disc = disc > 0.0 ? disc : 0.0;
    int64_t r = (int64_t)((b - sqrt(disc)) * 0.5);
    if (r < 0) r = 0;
    if (r > (int64_t)n - 2) r = (int64_t)n - 2;
    while (r + 1 <= (int64_t)n - 2 && tri_row_start((uint64_t)r + 1, n) <= k) ++r;
    while (r > 0 && tri_row_start((uint64_t)r, n) > k) --r;
    i = (uint64_t)r;
    j = k - tri_row_start(i, n) + i + 1;
}

// Linear gaps: H = max(0, H_d + s, H_u - gap, H_l - gap).  Affine gaps (Gotoh): E carries
// a horizontal gap run along the strip's rows, F a vertical one down the column (across
// strips through a second boundary row), H = max(0, H_d + s, E, F) with
// E = max(E_l - gap, H_l - gap_open - gap), F = max(F_u - gap, H_u - gap_open - gap).
template <bool AFFINE>
__global__ void __launch_bounds__(128)
sw_general_kernel(GeneralJob job, Scoring sc, int *__restrict__ scratch, uint64_t units, uint64_t scratch_ints)
{
    (void)scratch_ints;                             // checked in bounds-checked builds
    constexpr int NEG = -(1 << 28);
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    int *bnd = scratch + tid;                       // bnd[j * nthr] = H(strip top - 1, j)
    // affine: F(strip top - 1, j) in the second half of the scratch
    const uint64_t foff = (uint64_t)(job.B.stride * kBasesPerWord + 1) * nthr;
    int *bndf = scratch + foff + tid;
    // the boundary-row entry of column j is in the scratch (always, unless the build
    // checks bounds and finds it is not)
    auto in_scratch = [&](uint64_t j, uint64_t off) {
        return bounds_ok(off + j * nthr + tid, scratch_ints, BOUNDS_GENERAL_SCRATCH);
    };
    const uint64_t nb = job.b1 - job.b0;
    const int goe = sc.gap_open + sc.gap;

    for (uint64_t u = tid; u < units; u += nthr) {
        uint64_t ia, jb, o;
        if (job.mode == OUT_TRI) {
            uint64_t ti, tj;
            tri_unindex(u, job.A.n, ti, tj);
            ia = ti; jb = tj; o = u;
        } else if (job.mode == OUT_TRI_ROWS) {
            uint64_t lo = 0, hi = job.nrows;           // row_prefix[lo] <= u < row_prefix[lo+1]
            while (hi - lo > 1) {
                const uint64_t mid = (lo + hi) >> 1;
                if (job.row_prefix[mid] <= u) lo = mid; else hi = mid;
            }
            ia = job.rows[lo];
            jb = ia + 1 + (u - job.row_prefix[lo]);
            o = ia * job.A.n - ia * (ia + 1) / 2 + (jb - ia - 1) - job.out_base;
        } else {
            const uint64_t r = u / nb;
            ia = job.rows ? (uint64_t)job.rows[r] : job.a0 + r;
            jb = job.b0 + (u - r * nb);
            o = (ia - job.a0) * job.ld + (jb - job.b0);
        }
        const uint32_t *a = job.A.words + ia * job.A.stride;
        const uint32_t *b = job.B.words + jb * job.B.stride;
        const int la = job.A.len[ia];
        const int lb = job.B.len[jb];
        int best = 0;
        for (int i0 = 0; i0 < la; i0 += kStrip) {
            uint32_t ac[kStrip];
#pragma unroll
            for (int r = 0; r < kStrip; ++r) ac[r] = (i0 + r < la) ? base_at(a, i0 + r) : 4u;
            int hl[kStrip], el[kStrip];
#pragma unroll
            for (int r = 0; r < kStrip; ++r) { hl[r] = 0; el[r] = NEG; }   // H(i, 0) = 0, E(i, 0) = -inf
            int diag_top = 0;                                // H(i0, 0) = 0
            for (int j = 1; j <= lb; ++j) {
                const uint32_t c = base_at(b, j - 1);
                int up = (i0 == 0 || !in_scratch(j, 0)) ? 0 : bnd[(uint64_t)j * nthr];   // H(i0, j)
                int fup = NEG;                                                          // F(i0, j)
                if (AFFINE && i0 != 0 && in_scratch(j, foff)) fup = bndf[(uint64_t)j * nthr];
                int diag = diag_top;                                  // H(i0, j-1)
                diag_top = up;
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int s = (ac[r] == c) ? sc.match : sc.mismatch;
                    int h = max(0, diag + s);
                    if (AFFINE) {
                        const int e = max(el[r] - sc.gap, hl[r] - goe);
                        const int f = max(fup - sc.gap, up - goe);
                        h = max(h, max(e, f));
                        el[r] = e;
                        fup = f;
                    } else {
                        h = max(h, up - sc.gap);
                        h = max(h, hl[r] - sc.gap);
                    }
                    diag = hl[r];
                    hl[r] = h;
                    up = h;
                    if (i0 + r < la) best = max(best, h);
                }
                if (in_scratch(j, 0)) bnd[(uint64_t)j * nthr] = hl[kStrip - 1];
                if (AFFINE && in_scratch(j, foff)) bndf[(uint64_t)j * nthr] = fup;
            }
        }
        if (bounds_ok(o, job.out_len, BOUNDS_GENERAL_OUT)) job.out[o] = score_to_distance(best, la, lb, sc.conversion);
    }
}

// Blocks of 128 threads resident per SM for the kernel variant (one full wave is launched,
// so the grid-stride loop spreads the pairs evenly).
int resident_blocks(bool affine)
{
    static int cached[2] = {0, 0};
    int &c = cached[affine ? 1 : 0];
    if (c == 0) {
        int b = 0;
        cudaError_t e = affine ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sw_general_kernel<true>, 128, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sw_general_kernel<false>, 128, 0);
        c = (e == cudaSuccess && b > 0) ? b : 4;
    }
    return c;
}

}  // namespace

int run_general(const GeneralJob &job, const Scoring &sc, int sm_count, cudaStream_t stream)
{
    uint64_t units;
    if (job.mode == OUT_TRI) {
        const uint64_t n = job.A.n;
        units = n < 2 ? 0 : n * (n - 1) / 2;
    } else if (job.mode == OUT_TRI_ROWS) {
        units = job.units_total;
    } else {
        units = (job.rows ? job.nrows : (job.a1 - job.a0)) * (job.b1 - job.b0);
    }
    if (units == 0) return GBD_OK;
    const int threads = 128;
    // the boundary row needs (max column count + 1) ints per thread
    const uint32_t maxlb = job.B.stride * kBasesPerWord;
    uint64_t blocks = (uint64_t)std::max(sm_count, 1) * resident_blocks(sc.gap_open > 0);
    const uint64_t per_thread = (uint64_t)(maxlb + 1) * sizeof(int) * (sc.gap_open > 0 ? 2 : 1);
    const uint64_t budget = 1ull << 30;   // at most 1 GiB of boundary rows
    while (blocks > 1 && blocks * threads * per_thread > budget) blocks /= 2;
    const uint64_t need_blocks = (units + threads - 1) / threads;
    if (blocks > need_blocks) blocks = need_blocks;
    int *scratch = nullptr;
    GBD_CUDA_TRY(cudaMallocAsync((void **)&scratch, blocks * threads * per_thread, stream));
    const uint64_t sints = blocks * threads * per_thread / sizeof(int);
    if (sc.gap_open > 0)
        sw_general_kernel<true><<<(unsigned)blocks, threads, 0, stream>>>(job, sc, scratch, units, sints);
    else
        sw_general_kernel<false><<<(unsigned)blocks, threads, 0, stream>>>(job, sc, scratch, units, sints);
    note_launches(1);
    cudaError_t le = cudaGetLastError();
    cudaError_t fe = cudaFreeAsync(scratch, stream);
    if (le != cudaSuccess) return cuda_fail(le, "sw_general_kernel launch");
    if (fe != cudaSuccess) return cuda_fail(fe, "cudaFreeAsync");
    return GBD_OK;
}

int run_general_in(const GeneralJob &job, const Scoring &sc, int *scratch, uint64_t scratch_ints,
                   int sm_count, cudaStream_t stream)
{
    if (job.mode != OUT_RECT || job.rows) return fail(GBD_EINVAL, "internal: rectangle jobs only");
    const uint64_t units = (job.a1 - job.a0) * (job.b1 - job.b0);
    if (units == 0) return GBD_OK;
    const int threads = 128;
    const uint64_t per_thread = ((uint64_t)job.B.stride * kBasesPerWord + 1) * (sc.gap_open > 0 ? 2 : 1);   // ints
    uint64_t blocks = (uint64_t)std::max(sm_count, 1) * resident_blocks(sc.gap_open > 0);
    while (blocks > 0 && blocks * threads * per_thread > scratch_ints) --blocks;
    if (blocks == 0)
        return fail(GBD_EINVAL, "the boundary rows of one thread block do not fit the scratch area");
    const uint64_t need_blocks = (units + threads - 1) / threads;
    if (blocks > need_blocks) blocks = need_blocks;
    if (sc.gap_open > 0)
        sw_general_kernel<true><<<(unsigned)blocks, threads, 0, stream>>>(job, sc, scratch, units, scratch_ints);
    else
        sw_general_kernel<false><<<(unsigned)blocks, threads, 0, stream>>>(job, sc, scratch, units, scratch_ints);
    note_launches(1);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return cuda_fail(le, "sw_general_kernel launch");
    return GBD_OK;
}

uint64_t bounds_take_general()
{
#if GBD_BOUNDS_CHECK
    unsigned long long v = ~0ull, reset = ~0ull;
    if (cudaMemcpyFromSymbol(&v, g_bounds_first, sizeof v) != cudaSuccess) v = ~0ull;
    cudaMemcpyToSymbol(g_bounds_first, &reset, sizeof reset);
    return v;
#else
    return ~0ull;
#endif
}

}  // namespace gbd
