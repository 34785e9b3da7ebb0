// Classical MDS of the distance triangle (paper sections 3 and 6.2): double centering of
// the squared distances into the Gram matrix G = -1/2 J (D o D) J (section 6.2) and its
// leading eigenpairs by randomized SVD (sections 3.2-3.3, after Halko, Martinsson and
// Tropp 2011: randomized subspace iteration, then B = Q^T G Q and its eigenvectors).
//
// Device pipeline:
//   tri_max_kernel        largest distance (sets the fp16 scale 2^-s)
//   sqdist_square_kernel  triangle -> ld x ld fp16 W = d^2 2^-s (both halves, zero padding)
//   G X                   column means of X, centred fp16 X^T, W X^T on the tensor cores
//                         (mds_gemm.cu), slice sum, column means of the product, and
//                         Y = -2^(s-1) (P - 1 mean^T); J W J X = J W (J X) needs no
//                         centred copy of W
//   orthonormalise        Gram S = Y^T Y (float64), Cholesky S = R^T R, Q = Y R^-1
//                         (columns whose pivot falls below a floor dropped); once between
//                         products, twice for the basis that B is formed on
//   eigenpairs of B       B = Q^T (G Q) by the same Gram kernel, threshold Jacobi in
//                         float32, eigenvalues sorted down, coordinates
//                         Q V_r diag(max(lambda, 0)^1/2)
// All reductions run in a fixed order, so results do not depend on scheduling.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "gbd_internal.cuh"
#include "mds_internal.cuh"

namespace gbd {
namespace {

// ------------------------------------------------------------------ triangle maximum
__global__ void tri_max_kernel(const uint16_t *__restrict__ tri, uint64_t m, uint32_t *out)
{
    uint32_t best = 0;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    // scalar head up to a 16-byte boundary, uint4 body, scalar tail
    const uint64_t head = std::min<uint64_t>(m, ((16 - (reinterpret_cast<uintptr_t>(tri) & 15)) & 15) / 2);
    for (uint64_t i = tid; i < head; i += nthr) best = max(best, (uint32_t)tri[i]);
    const uint64_t nvec = (m - head) / 8;
    const uint4 *v = reinterpret_cast<const uint4 *>(tri + head);
    for (uint64_t i = tid; i < nvec; i += nthr) {
        const uint4 w = __ldg(v + i);
        const uint32_t a = __vmaxu2(__vmaxu2(w.x, w.y), __vmaxu2(w.z, w.w));
        best = max(best, max(a & 0xffffu, a >> 16));
    }
    for (uint64_t i = head + nvec * 8 + tid; i < m; i += nthr) best = max(best, (uint32_t)tri[i]);
    best = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// ------------------------------------------------------------------ triangle -> fp16 square
constexpr int ST = 64;   // square tile
constexpr uint64_t SUPER = 16;   // tiles per super-tile side

__device__ __forceinline__ uint64_t tri_index(uint64_t i, uint64_t j, uint64_t n)
{
    return i * n - i * (i + 1) / 2 + (j - i - 1);
}

__device__ __forceinline__ uint16_t sq_half(uint32_t d, float scale)
{
    const float f = (float)d;
    return __half_as_ushort(__float2half_rn(f * f * scale));
}

// Two packed distances (low and high 16 bits) to two packed fp16 values of d^2 * scale.
// float(d) for d < 2^16 comes from the float bit pattern 2^23 + d minus 2^23 (exact),
// which keeps the conversion off the slow integer-to-float path, and the pair is rounded
// to fp16 by one paired conversion.
__device__ __forceinline__ uint32_t sq_half2(uint32_t pair, float scale)
{
    const float lo = __uint_as_float(0x4B000000u | (pair & 0xffffu)) - 8388608.0f;
    const float hi = __uint_as_float(0x4B000000u | (pair >> 16)) - 8388608.0f;
    const __half2 h = __floats2half2_rn(lo * lo * scale, hi * hi * scale);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Tile (I, J), I <= J, of the square: W[I-block][J-block] from the triangle, and its
// transpose W[J-block][I-block] through shared memory.  Off-diagonal tiles whose columns
// all lie below n (all but a thin margin) take the fast path: each warp handles whole
// 64-column row segments, one aligned 32-bit load per lane (the segment's parity fixed up
// with a shuffle), 128-byte stores; the rest go element by element.
__global__ void __launch_bounds__(256)
sqdist_square_kernel(const uint16_t *__restrict__ tri, uint64_t n, uint64_t ld, float scale,
                     uint16_t *__restrict__ W, uint64_t nsuper, int aligned)
{
    __shared__ uint16_t t[ST][ST + 2];
    const uint64_t T = ld / ST;
    // Blocks walk super-tiles of SUPER x SUPER tiles (upper triangle of super-tiles, row by
    // row), and the tiles of a super-tile row by row, so the blocks resident at one time
    // write a compact region of the square in both of its orientations.
    const uint64_t sup = blockIdx.x / (SUPER * SUPER), within = blockIdx.x % (SUPER * SUPER);
    const uint64_t TS = (T + SUPER - 1) / SUPER;
    if (sup >= nsuper) return;
    // row SI of the super-tile triangle holds TS - SI super-tiles (float estimate, exact fix-up)
    const float b = 2.0f * (float)TS + 1.0f;
    int64_t SI = (int64_t)((b - sqrtf(fmaxf(b * b - 8.0f * (float)sup, 0.0f))) * 0.5f);
    auto row_start = [&](int64_t r) { return (uint64_t)r * TS - (uint64_t)r * (uint64_t)(r - 1) / 2; };
    if (SI < 0) SI = 0;
    while (SI > 0 && row_start(SI) > sup) --SI;
    while ((uint64_t)(SI + 1) < TS && row_start(SI + 1) <= sup) ++SI;
    const uint64_t SJ = (uint64_t)SI + (sup - row_start(SI));
    const uint64_t I = (uint64_t)SI * SUPER + within / SUPER, J = SJ * SUPER + within % SUPER;
    if (I > J || J >= T) return;
    const uint64_t i0 = I * ST, j0 = J * ST;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const bool fast = aligned && (uint64_t)I != J && j0 + ST <= n;
    if (fast) {
        // every row i of this tile is below j0 < n, and its 64 columns lie in one
        // triangle row: issue the eight rows' loads of this warp before using any
        const uint32_t *tw = reinterpret_cast<const uint32_t *>(tri);
        uint32_t lo[8], ex[8], odd[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint64_t k0 = tri_index(i0 + warp + 8 * q, j0, n);   // element 0 of the segment
            const uint64_t w0 = k0 >> 1;
            odd[q] = (uint32_t)(k0 & 1);
            lo[q] = __ldg(tw + w0 + lane);
            // for an odd start, lane 31 also needs the word after the segment's 32
            ex[q] = (lane == 31 && odd[q]) ? __ldg(tw + w0 + 32) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = warp + 8 * q;
            uint32_t hi = __shfl_down_sync(0xffffffffu, lo[q], 1);     // the next lane's word
            if (lane == 31) hi = ex[q];
            const uint32_t pair = odd[q] ? __funnelshift_r(lo[q], hi, 16) : lo[q];
            const uint32_t pk = sq_half2(pair, scale);
            t[r][2 * lane] = (uint16_t)(pk & 0xffffu);
            t[r][2 * lane + 1] = (uint16_t)(pk >> 16);
            *reinterpret_cast<uint32_t *>(W + (i0 + r) * ld + j0 + 2 * lane) = pk;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = warp + 8 * q;
            const uint32_t pk = (uint32_t)t[2 * lane][r] | ((uint32_t)t[2 * lane + 1][r] << 16);
            *reinterpret_cast<uint32_t *>(W + (j0 + r) * ld + i0 + 2 * lane) = pk;
        }
        return;
    }

    // general path: each thread 4 consecutive columns of one row, 4 passes of 16 rows
    const int c4 = (threadIdx.x & 15) * 4;
    for (int r = threadIdx.x >> 4; r < ST; r += 16) {
        const uint64_t i = i0 + r;
        uint16_t v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint64_t j = j0 + c4 + e;
            uint16_t h = 0;
            if (i < n && j < n && i != j) {
                const uint32_t d = (i < j) ? tri[tri_index(i, j, n)] : tri[tri_index(j, i, n)];
                h = sq_half(d, scale);
            }
            v[e] = h;
            t[r][c4 + e] = h;
        }
        uint2 pk;
        pk.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
        pk.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
        *reinterpret_cast<uint2 *>(W + i * ld + j0 + c4) = pk;
    }
    if ((uint64_t)I == J) return;
    __syncthreads();
    for (int r = threadIdx.x >> 4; r < ST; r += 16) {
        uint2 pk;
        pk.x = (uint32_t)t[c4][r] | ((uint32_t)t[c4 + 1][r] << 16);
        pk.y = (uint32_t)t[c4 + 2][r] | ((uint32_t)t[c4 + 3][r] << 16);
        *reinterpret_cast<uint2 *>(W + (j0 + r) * ld + i0 + c4) = pk;
    }
}

// ------------------------------------------------------------------ column means
constexpr int kSumBlocks = 256;

// partial[b][c] = sum of X[i][c] over the rows of block b (fixed row ranges).
__global__ void colsum_partial_kernel(const float *__restrict__ X, uint64_t n, uint32_t k, double *partial)
{
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t r0 = blockIdx.x * per, r1 = std::min<uint64_t>(n, r0 + per);
    for (uint32_t c = threadIdx.x; c < k; c += blockDim.x) {
        double s = 0.0;
        for (uint64_t i = r0; i < r1; ++i) s += (double)X[i * k + c];
        partial[(uint64_t)blockIdx.x * k + c] = s;
    }
}

// mean[c] = (sum of the partial sums of column c) / n: one block per column, a strided
// sum per thread and a tree in shared memory (a fixed order, so the result is
// reproducible).
__global__ void __launch_bounds__(256)
colmean_final_kernel(const double *__restrict__ partial, uint32_t nparts, uint32_t k, uint64_t n, double *mean)
{
    __shared__ double red[256];
    const uint32_t c = blockIdx.x;
    double s = 0.0;
    for (uint32_t b = threadIdx.x; b < nparts; b += blockDim.x) s += partial[(uint64_t)b * k + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (uint32_t w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[c] = red[0] / (double)n;
}

// Xt[c][i] = fp16(X[i][c] - mean[c]) for i < n; 0 for n <= i < ld.  32 x 32 tiles.
__global__ void center_transpose_kernel(const float *__restrict__ X, const double *__restrict__ mean, uint64_t n,
                                        uint64_t ld, uint32_t k, uint16_t *__restrict__ Xt)
{
    __shared__ float t[32][33];
    const uint64_t i0 = (uint64_t)blockIdx.x * 32;
    const uint32_t c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const uint64_t i = i0 + r;
        const uint32_t c = c0 + threadIdx.x;
        float v = 0.f;
        if (i < n && c < k) v = (float)((double)X[i * k + c] - mean[c]);
        t[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const uint32_t c = c0 + r;
        const uint64_t i = i0 + threadIdx.x;
        if (c < k && i < ld) Xt[(uint64_t)c * ld + i] = __half_as_ushort(__float2half_rn(t[threadIdx.x][r]));
    }
}

// P[i][c] = sum over slices s (in order) of part[s][i][c], i < n.
__global__ void slice_sum_kernel(const float *__restrict__ part, uint32_t slices, uint64_t n, uint64_t ld,
                                 uint32_t k, float *__restrict__ P)
{
    const uint64_t total = n * k;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (uint32_t q = 0; q < slices; ++q) s += part[(uint64_t)q * ld * k + e];
        P[e] = s;
    }
}

// Y = alpha (P - 1 mean^T)
__global__ void center_scale_kernel(const float *__restrict__ P, const double *__restrict__ mean, uint64_t n,
                                    uint32_t k, double alpha, float *__restrict__ Y)
{
    const uint64_t total = n * k;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x)
        Y[e] = (float)(alpha * ((double)P[e] - mean[e % k]));
}

// ------------------------------------------------------------------ A^T B in float64
constexpr int kGramRows = 32;

// a * b = p + e and s + h = t + f exactly (the product split with a fused multiply-add,
// the sum by Knuth's two-sum); the _rn intrinsics keep the compiler from contracting
// or reassociating these steps.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void two_sum(float s, float h, float &t, float &f)
{
    t = __fadd_rn(s, h);
    const float bp = __fsub_rn(t, s);
    f = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(h, bp));
}

// partial[b] = sum over block b's rows of A[i]^T B[i] (k x k) for float32 A, B.  Each
// product is split exactly into two floats and added to a two-float running sum (the
// high part by an exact two-sum, the low part collecting the rounding terms), which
// carries about 48 bits, close to float64 accumulation, at float32 instruction rates
// (float64 arithmetic runs about 60 times slower on this GPU).  Fixed summation order.
// Rows are staged in shared memory; each thread owns 4 x 4 tiles of the output in
// registers.  With A == B (SYM) only the tiles on or above the diagonal are accumulated
// and each is written to both halves.
template <bool SYM>
__global__ void __launch_bounds__(256)
xty_partial_kernel(const float *__restrict__ A, const float *__restrict__ B, uint64_t n, uint32_t k,
                   double *partial)
{
    extern __shared__ float smf[];
    float *As = smf;                                 // [kGramRows][k]
    float *Bs = SYM ? smf : smf + kGramRows * k;     // [kGramRows][k]
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t r0 = blockIdx.x * per, r1 = std::min<uint64_t>(n, r0 + per);
    const uint32_t kt = k / 4;              // 4 x 4 tiles per side
    const uint32_t ntiles = SYM ? kt * (kt + 1) / 2 : kt * kt;
    double *out = partial + (uint64_t)blockIdx.x * k * k;
    for (uint32_t t0 = 0; t0 < ntiles; t0 += blockDim.x) {
        const uint32_t t = t0 + threadIdx.x;
        const bool active = t < ntiles;
        uint32_t ta = 0, tb = 0;
        if (active) {
            if (SYM) {
                // t-th tile of the upper triangle, row by row: row ta holds tiles ta .. kt-1
                uint32_t rest = t;
                while (rest >= kt - ta) { rest -= kt - ta; ++ta; }
                tb = ta + rest;
            } else {
                ta = t / kt;
                tb = t % kt;
            }
        }
        const uint32_t a0 = ta * 4, b0 = tb * 4;
        float hi[4][4], lo[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) { hi[x][y] = 0.f; lo[x][y] = 0.f; }
        for (uint64_t rb = r0; rb < r1; rb += kGramRows) {
            const uint32_t rows = (uint32_t)std::min<uint64_t>(kGramRows, r1 - rb);
            __syncthreads();
            for (uint32_t e = threadIdx.x; e < rows * k; e += blockDim.x) {
                As[e] = A[rb * k + e];
                if (!SYM) Bs[e] = B[rb * k + e];
            }
            __syncthreads();
            if (active) {
                for (uint32_t r = 0; r < rows; ++r) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(As + r * k + a0);
                    const float4 b4 = *reinterpret_cast<const float4 *>(Bs + r * k + b0);
                    const float av[4] = {a4.x, a4.y, a4.z, a4.w};
                    const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            float p, pe, t2, f;
                            two_prod(av[x], bv[y], p, pe);
                            two_sum(hi[x][y], p, t2, f);
                            hi[x][y] = t2;
                            lo[x][y] = __fadd_rn(lo[x][y], __fadd_rn(f, pe));
                        }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const double v = (double)hi[x][y] + (double)lo[x][y];
                    out[(a0 + x) * k + b0 + y] = v;
                    if (SYM && ta != tb) out[(b0 + y) * k + a0 + x] = v;
                }
        }
    }
}

__global__ void xty_final_kernel(const double *__restrict__ partial, uint32_t nparts, uint32_t kk, double *C)
{
    for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < kk; o += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (uint32_t b = 0; b < nparts; ++b) s += partial[(uint64_t)b * kk + o];
        C[o] = s;
    }
}

// ------------------------------------------------------------------ Cholesky QR step
// S = Y^T Y = R^T R (R upper triangular), float64, one block; T = R^-1 (float32) so that
// Q = Y T has orthonormal columns.  A column whose remaining pivot falls below
// floor_rel * max diag(S) lies (numerically) in the span of the earlier columns: its row
// of R and its column of T are set to 0, so Q gets a zero column there.
__global__ void __launch_bounds__(256)
chol_inverse_kernel(const double *__restrict__ S_in, uint32_t k, double floor_rel, float *__restrict__ T,
                    uint32_t *flags)
{
    extern __shared__ double sc[];
    double *R = sc;                 // k x k, becomes R (upper part)
    double *Ti = sc + k * k;        // k x k, R^-1
    __shared__ double smax;
    __shared__ int keep[128];
    __shared__ double inv_d[128];
    const uint32_t kk = k * k;
    for (uint32_t e = threadIdx.x; e < kk; e += blockDim.x) {
        const uint32_t i = e / k, j = e % k;
        const double a = 0.5 * (S_in[i * k + j] + S_in[j * k + i]);
        R[e] = a;
        Ti[e] = 0.0;
        if (!isfinite(a)) atomicOr(flags, 2u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (uint32_t j = 0; j < k; ++j) m = fmax(m, R[j * k + j]);
        smax = m;
    }
    __syncthreads();
    // right-looking Cholesky on the upper triangle
    for (uint32_t j = 0; j < k; ++j) {
        const double d = R[j * k + j];
        const bool ok = d > floor_rel * smax && d > 0.0;
        const double rjj = ok ? sqrt(d) : 0.0;
        __syncthreads();
        for (uint32_t c = j + threadIdx.x; c < k; c += blockDim.x)
            R[j * k + c] = ok ? (c == j ? rjj : R[j * k + c] / rjj) : 0.0;
        if (threadIdx.x == 0) keep[j] = ok;
        __syncthreads();
        // trailing update A[r][c] -= R[j][r] R[j][c], j < r <= c: warps over rows, lanes
        // over columns
        const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (uint32_t r = j + 1 + warp; r < k; r += nw) {
            const double rjr = R[j * k + r];
            for (uint32_t c = r + lane; c < k; c += 32) R[r * k + c] -= rjr * R[j * k + c];
        }
        __syncthreads();
    }
    // T = R^-1 column by column (back substitution; dropped rows stay 0), with the
    // reciprocals of the diagonal formed once and two partial sums per dot product
    // (float64 division and dependent float64 chains are slow on this GPU)
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) inv_d[i] = keep[i] ? 1.0 / R[i * k + i] : 0.0;
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < k; c += blockDim.x) {
        if (!keep[c]) continue;
        Ti[c * k + c] = inv_d[c];
        for (int i = (int)c - 1; i >= 0; --i) {
            if (!keep[i]) continue;
            double s0 = 0.0, s1 = 0.0;
            uint32_t m2 = (uint32_t)i + 1;
            for (; m2 + 1 <= c; m2 += 2) {
                s0 += R[i * k + m2] * Ti[m2 * k + c];
                s1 += R[i * k + m2 + 1] * Ti[(m2 + 1) * k + c];
            }
            if (m2 <= c) s0 += R[i * k + m2] * Ti[m2 * k + c];
            Ti[i * k + c] = -(s0 + s1) * inv_d[i];
        }
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < kk; e += blockDim.x) T[e] = (float)Ti[e];
}

// ------------------------------------------------------------------ symmetric eigensolver
// Eigenpairs of the small symmetric B = Q^T G Q: cyclic Jacobi with the round-robin
// ordering (k/2 disjoint rotations per round, k-1 rounds per sweep), one block.  The
// matrix, the rotations and their angles live in float32 (this part's output is float32,
// and float64 arithmetic is scarce on this GPU).  A pair is
// rotated only while its off-diagonal entry exceeds 1e-6 of the matrix norm (threshold
// Jacobi); the sweeps stop when one makes no rotation.  Outputs: the r largest eigenvalues in order into lambda, and
// T = V_r diag(max(lambda, 0)^1/2).  flags bit 0: no convergence; bit 1: non-finite input.
constexpr int kMaxJacobiK = 112;
constexpr int kMaxSweeps = 40;
constexpr double kJacobiTol = 1e-6;   // about 17 float32 ulps

__global__ void __launch_bounds__(256)
jacobi_kernel(const double *__restrict__ S_in, uint32_t k, uint32_t r, float *__restrict__ T,
              float *__restrict__ lambda, uint32_t *flags)
{
    extern __shared__ float sf[];
    // rows padded to k + 1 floats: a column walk (fixed p, rows 0..k-1) then falls in
    // different banks instead of one
    const uint32_t la = k + 1;
    float *A = sf;                    // k x la
    float *V = sf + k * la;           // k x la
    __shared__ float cs[kMaxJacobiK / 2], sn[kMaxJacobiK / 2];
    __shared__ int pp[kMaxJacobiK / 2], qq[kMaxJacobiK / 2];
    __shared__ double red[256];
    __shared__ int rotated;
    __shared__ double fro;
    __shared__ int order[kMaxJacobiK];
    const uint32_t kk = k * k;
    double tot = 0.0;
    for (uint32_t e = threadIdx.x; e < kk; e += blockDim.x) {
        const uint32_t i = e / k, j = e % k;
        const double a = 0.5 * (S_in[i * k + j] + S_in[j * k + i]);
        A[i * la + j] = (float)a;
        V[i * la + j] = (i == j) ? 1.f : 0.f;
        tot += a * a;
        if (!isfinite(a)) atomicOr(flags, 2u);
    }
    red[threadIdx.x] = tot;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) fro = sqrt(red[0]);
    __syncthreads();
    const float fro_floor = (float)(kJacobiTol * fro);
    const uint32_t half = k / 2;
    bool converged = false;
    for (int sweep = 0; sweep < kMaxSweeps && !converged; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (uint32_t round = 0; round + 1 < k; ++round) {
            if (threadIdx.x < half) {
                // circle method: position 0 fixed, positions 1..k-1 rotate
                auto at = [&](uint32_t pos) -> uint32_t { return pos == 0 ? 0u : 1u + (pos - 1 + round) % (k - 1); };
                uint32_t p = at(threadIdx.x), q = at(k - 1 - threadIdx.x);
                if (p > q) { const uint32_t t = p; p = q; q = t; }
                const float apq = A[p * la + q], app = A[p * la + p], aqq = A[q * la + q];
                float c = 1.f, s = 0.f;
                // negligible against the matrix norm (float32 cannot resolve less)
                if (fabsf(apq) > fro_floor) {
                    const float theta = (aqq - app) / (2.f * apq);
                    // t = tan of the rotation angle, the root of smaller magnitude; for a
                    // huge theta, t = 1 / (2 theta) without forming theta^2
                    const float at = fabsf(theta);
                    const float t = (theta >= 0.f ? 1.f : -1.f) /
                                    (at + (at < 1e18f ? sqrtf(theta * theta + 1.f) : at));
                    c = rsqrtf(t * t + 1.f);
                    s = t * c;
                    rotated = 1;
                }
                cs[threadIdx.x] = c;
                sn[threadIdx.x] = s;
                pp[threadIdx.x] = (int)p;
                qq[threadIdx.x] = (int)q;
            }
            __syncthreads();
            // columns: A <- A P, V <- V P
            for (uint32_t e = threadIdx.x; e < half * k; e += blockDim.x) {
                const uint32_t pr = e / k, row = e % k;
                const float s = sn[pr];
                if (s == 0.f) continue;
                const int p = pp[pr], q = qq[pr];
                const float c = cs[pr];
                const float ap = A[row * la + p], aq = A[row * la + q];
                A[row * la + p] = c * ap - s * aq;
                A[row * la + q] = s * ap + c * aq;
                const float vp = V[row * la + p], vq = V[row * la + q];
                V[row * la + p] = c * vp - s * vq;
                V[row * la + q] = s * vp + c * vq;
            }
            __syncthreads();
            // rows: A <- P^T A
            for (uint32_t e = threadIdx.x; e < half * k; e += blockDim.x) {
                const uint32_t pr = e / k, col = e % k;
                const float s = sn[pr];
                if (s == 0.f) continue;
                const int p = pp[pr], q = qq[pr];
                const float c = cs[pr];
                const float ap = A[p * la + col], aq = A[q * la + col];
                A[p * la + col] = c * ap - s * aq;
                A[q * la + col] = s * ap + c * aq;
            }
            __syncthreads();
        }
        converged = (rotated == 0);
        __syncthreads();
    }
    if (!converged && threadIdx.x == 0) atomicOr(flags, 1u);
    // eigenvalues on the diagonal; rank them largest first (ties by index)
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
        const float li = A[i * la + i];
        int rank = 0;
        for (uint32_t j = 0; j < k; ++j) {
            const float lj = A[j * la + j];
            if (lj > li || (lj == li && j < i)) ++rank;
        }
        order[rank] = (int)i;
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < k * r; e += blockDim.x) {
        const uint32_t row = e / r, a = e % r;
        const int col = order[a];
        const float lam = A[col * la + col];
        T[e] = V[row * la + col] * sqrtf(fmaxf(lam, 0.f));
    }
    for (uint32_t a = threadIdx.x; a < r; a += blockDim.x) lambda[a] = A[order[a] * la + order[a]];
}

// ------------------------------------------------------------------ Out = A T
// A: n x k (row-major), T: k x m, Out: n x m.  64 rows per block, float32.
__global__ void __launch_bounds__(256)
apply_kernel(const float *__restrict__ A, const float *__restrict__ T, uint64_t n, uint32_t k, uint32_t m,
             float *__restrict__ Out)
{
    extern __shared__ float sa[];
    float *As = sa;                     // [64][k + 1]
    float *Ts = sa + 64 * (k + 1);      // [k][m]
    const uint64_t r0 = (uint64_t)blockIdx.x * 64;
    for (uint32_t e = threadIdx.x; e < 64 * k; e += blockDim.x) {
        const uint32_t r = e / k, c = e % k;
        As[r * (k + 1) + c] = (r0 + r < n) ? A[(r0 + r) * k + c] : 0.f;
    }
    for (uint32_t e = threadIdx.x; e < k * m; e += blockDim.x) Ts[e] = T[e];
    __syncthreads();
    const uint32_t r = threadIdx.x & 63;
    if (r0 + r >= n) return;
    for (uint32_t c = threadIdx.x >> 6; c < m; c += 4) {
        float s = 0.f;
        for (uint32_t j = 0; j < k; ++j) s = fmaf(As[r * (k + 1) + j], Ts[j * m + c], s);
        Out[(r0 + r) * m + c] = s;
    }
}

// ------------------------------------------------------------------ host helpers
int grid_for(uint64_t work, int threads, int sm_count)
{
    const uint64_t want = (work + threads - 1) / threads;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(sm_count, 1) * 8));
}

#define GBD_LAUNCH_CHECK(name)                                   \
    do {                                                         \
        note_launches(1);                                        \
        cudaError_t _le = cudaGetLastError();                    \
        if (_le != cudaSuccess) return cuda_fail(_le, name);     \
    } while (0)

// Workspace of the G X product and of the orthonormalisation.
struct MdsWork {
    uint64_t n = 0, ld = 0;
    uint32_t k = 0, slices = 0;
    uint16_t *xt = nullptr;       // k x ld fp16
    float *part = nullptr;        // slices x ld x k
    float *P = nullptr;           // n x k
    double *sums = nullptr;       // kSumBlocks x k
    double *mean = nullptr;       // k
    double *gram_part = nullptr;  // gram_blocks x k x k
    double *gram = nullptr;       // k x k
    float *T = nullptr;           // k x k
    uint32_t *flags = nullptr;    // [0] product error word, [1] eigensolver flags
    uint32_t gram_blocks = 0;
    cudaStream_t st = nullptr;
    std::vector<void *> owned;

    int alloc(void **p, size_t bytes)
    {
        cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GBD_ENOMEM, std::string("device workspace of ") + std::to_string(bytes) + " bytes: " +
                                        cudaGetErrorString(e));
        }
        owned.push_back(*p);
        return GBD_OK;
    }
    int init(uint64_t n_, uint64_t ld_, uint32_t k_, int sm_count, cudaStream_t s)
    {
        n = n_; ld = ld_; k = k_; st = s;
        slices = w_times_x_slices(ld, sm_count);
        gram_blocks = (uint32_t)std::min<uint64_t>(256, std::max<uint64_t>(1, (n + 255) / 256));
        int rc = alloc((void **)&xt, (size_t)k * ld * 2);
        if (rc == GBD_OK) rc = alloc((void **)&part, (size_t)slices * ld * k * 4);
        if (rc == GBD_OK) rc = alloc((void **)&P, (size_t)n * k * 4);
        if (rc == GBD_OK) rc = alloc((void **)&sums, (size_t)kSumBlocks * k * 8);
        if (rc == GBD_OK) rc = alloc((void **)&mean, (size_t)k * 8);
        if (rc == GBD_OK) rc = alloc((void **)&gram_part, (size_t)gram_blocks * k * k * 8);
        if (rc == GBD_OK) rc = alloc((void **)&gram, (size_t)k * k * 8);
        if (rc == GBD_OK) rc = alloc((void **)&T, (size_t)k * k * 4);
        if (rc == GBD_OK) rc = alloc((void **)&flags, 16);
        if (rc == GBD_OK) {
            cudaError_t e = cudaMemsetAsync(flags, 0, 16, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        }
        return rc;
    }
    void release()
    {
        for (void *p : owned) cudaFreeAsync(p, st);
        owned.clear();
    }
};

int column_means(const float *X, uint64_t n, uint32_t k, MdsWork &w)
{
    colsum_partial_kernel<<<kSumBlocks, 128, 0, w.st>>>(X, n, k, w.sums);
    GBD_LAUNCH_CHECK("colsum_partial_kernel");
    colmean_final_kernel<<<k, 256, 0, w.st>>>(w.sums, kSumBlocks, k, n, w.mean);
    GBD_LAUNCH_CHECK("colmean_final_kernel");
    return GBD_OK;
}

// Y = G X (G = -1/2 J (D o D) J with D o D = 2^s W).
int gram_apply_in(const uint16_t *W, int32_t shift, const float *X, float *Y, MdsWork &w, int sm_count)
{
    int rc = column_means(X, w.n, w.k, w);
    if (rc != GBD_OK) return rc;
    dim3 tg((unsigned)(w.ld / 32), (w.k + 31) / 32);
    center_transpose_kernel<<<tg, dim3(32, 8), 0, w.st>>>(X, w.mean, w.n, w.ld, w.k, w.xt);
    GBD_LAUNCH_CHECK("center_transpose_kernel");
    rc = w_times_x(W, w.ld, w.xt, w.k, w.part, w.slices, w.flags, sm_count, w.st);
    if (rc != GBD_OK) return rc;
    slice_sum_kernel<<<grid_for(w.n * w.k, 256, sm_count), 256, 0, w.st>>>(w.part, w.slices, w.n, w.ld, w.k, w.P);
    GBD_LAUNCH_CHECK("slice_sum_kernel");
    rc = column_means(w.P, w.n, w.k, w);
    if (rc != GBD_OK) return rc;
    const double alpha = -std::ldexp(1.0, shift - 1);
    center_scale_kernel<<<grid_for(w.n * w.k, 256, sm_count), 256, 0, w.st>>>(w.P, w.mean, w.n, w.k, alpha, Y);
    GBD_LAUNCH_CHECK("center_scale_kernel");
    return GBD_OK;
}

int xty(const float *A, const float *B, MdsWork &w)
{
    const size_t smem = 2 * (size_t)kGramRows * w.k * sizeof(float);
    if (A == B) xty_partial_kernel<true><<<w.gram_blocks, 256, smem, w.st>>>(A, B, w.n, w.k, w.gram_part);
    else xty_partial_kernel<false><<<w.gram_blocks, 256, smem, w.st>>>(A, B, w.n, w.k, w.gram_part);
    GBD_LAUNCH_CHECK("xty_partial_kernel");
    xty_final_kernel<<<(w.k * w.k + 255) / 256, 256, 0, w.st>>>(w.gram_part, w.gram_blocks, w.k * w.k, w.gram);
    GBD_LAUNCH_CHECK("xty_final_kernel");
    return GBD_OK;
}

size_t jacobi_smem(uint32_t k) { return 2 * (size_t)k * k * sizeof(double); }
size_t jacobi_smem_f32(uint32_t k) { return 2 * (size_t)k * (k + 1) * sizeof(float); }

int apply(const float *A, const float *T, uint32_t m, float *Out, MdsWork &w)
{
    const size_t smem = (64 * (size_t)(w.k + 1) + (size_t)w.k * m) * sizeof(float);
    apply_kernel<<<(unsigned)((w.n + 63) / 64), 256, smem, w.st>>>(A, T, w.n, w.k, m, Out);
    GBD_LAUNCH_CHECK("apply_kernel");
    return GBD_OK;
}

// Q = basis of the range of Y by Cholesky QR, `passes` times (two give an orthonormal
// basis to working precision; one suffices between the products of the subspace
// iteration, which only need the right span).  Y is overwritten.
constexpr double kOrthFloor = 1e-12;

int orthonormalise(float *Y, float *Q, MdsWork &w, int passes)
{
    float *src = Y, *dst = Q;
    for (int pass = 0; pass < passes; ++pass) {
        int rc = xty(src, src, w);
        if (rc != GBD_OK) return rc;
        chol_inverse_kernel<<<1, 256, jacobi_smem(w.k), w.st>>>(w.gram, w.k, kOrthFloor, w.T, w.flags + 1);
        GBD_LAUNCH_CHECK("chol_inverse_kernel");
        rc = apply(src, w.T, w.k, dst, w);
        if (rc != GBD_OK) return rc;
        std::swap(src, dst);
    }
    // after an even number of passes the result is back in Y
    if (src != Q) {
        cudaError_t e = cudaMemcpyAsync(Q, src, w.n * w.k * sizeof(float), cudaMemcpyDeviceToDevice, w.st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    return GBD_OK;
}

int configure_kernels()
{
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (done) return GBD_OK;
    GBD_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)jacobi_smem_f32(kMaxJacobiK)));
    GBD_CUDA_TRY(cudaFuncSetAttribute(xty_partial_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(2 * kGramRows * kMaxJacobiK * sizeof(float))));
    GBD_CUDA_TRY(cudaFuncSetAttribute(xty_partial_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(2 * kGramRows * kMaxJacobiK * sizeof(float))));
    GBD_CUDA_TRY(cudaFuncSetAttribute(chol_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)jacobi_smem(kMaxJacobiK)));
    GBD_CUDA_TRY(cudaFuncSetAttribute(
        apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)((64 * (kMaxJacobiK + 1) + kMaxJacobiK * kMaxJacobiK) * sizeof(float))));
    done = true;
    return GBD_OK;
}

int sqdist_square_impl(gbd_ctx *ctx, const uint16_t *d_tri, uint64_t n, uint16_t *d_w, uint64_t ld,
                       int32_t *shift, cudaStream_t st)
{
    if (!ctx || !d_w || !shift) return fail(GBD_EINVAL, "NULL argument");
    if (n >= 2 && !d_tri) return fail(GBD_EINVAL, "NULL triangle");
    if (ld == 0 || ld % 128 != 0 || ld < n) return fail(GBD_EINVAL, "ld must be a multiple of 128 and >= n");
    if (n > 0xffffffffull) return fail(GBD_EINVAL, "too many reads");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    const uint64_t m = n < 2 ? 0 : n * (n - 1) / 2;
    uint32_t dmax = 0;
    if (m > 0) {
        uint32_t *d_max = nullptr;
        GBD_CUDA_TRY(cudaMallocAsync((void **)&d_max, sizeof(uint32_t), st));
        GBD_CUDA_TRY(cudaMemsetAsync(d_max, 0, sizeof(uint32_t), st));
        tri_max_kernel<<<grid_for(m / 8 + 1, 256, ctx->sm_count), 256, 0, st>>>(d_tri, m, d_max);
        note_launches(1);
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaMemcpyAsync(&dmax, d_max, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        cudaError_t se = cudaStreamSynchronize(st);
        cudaFreeAsync(d_max, st);
        if (le != cudaSuccess) return cuda_fail(le, "tri_max_kernel launch");
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemcpyAsync");
        if (se != cudaSuccess) return cuda_fail(se, "cudaStreamSynchronize");
    }
    // smallest s >= 0 with dmax^2 * 2^-s <= 65504 (the fp16 maximum)
    int s = 0;
    const double d2 = (double)dmax * (double)dmax;
    while (d2 * std::ldexp(1.0, -s) > 65504.0) ++s;
    *shift = s;
    const uint64_t T = ld / ST;
    const uint64_t TS = (T + SUPER - 1) / SUPER;
    const uint64_t nsuper = TS * (TS + 1) / 2;
    const uint64_t nblocks = nsuper * SUPER * SUPER;
    if (nblocks > 0x7fffffffull) return fail(GBD_EINVAL, "square too large");
    const int aligned = (reinterpret_cast<uintptr_t>(d_tri) % 4) == 0 ? 1 : 0;
    sqdist_square_kernel<<<(unsigned)nblocks, 256, 0, st>>>(d_tri, n, ld, (float)std::ldexp(1.0, -s), d_w, nsuper,
                                                             aligned);
    GBD_LAUNCH_CHECK("sqdist_square_kernel");
    return GBD_OK;
}

// The context's cached square of at least `bytes`, ordered after its previous use on any
// stream.  A larger size replaces it (after the previous use has finished).
int mds_square_buffer(gbd_ctx *ctx, size_t bytes, cudaStream_t st, uint16_t **W)
{
    if (!ctx->mds_w_done) GBD_CUDA_TRY(cudaEventCreateWithFlags(&ctx->mds_w_done, cudaEventDisableTiming));
    if (ctx->mds_w_bytes < bytes) {
        if (ctx->mds_w) {
            GBD_CUDA_TRY(cudaEventSynchronize(ctx->mds_w_done));
            GBD_CUDA_TRY(cudaFree(ctx->mds_w));
            ctx->mds_w = nullptr;
            ctx->mds_w_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&ctx->mds_w, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->mds_w = nullptr;
            return fail(GBD_ENOMEM, std::string("MDS square of ") + std::to_string(bytes) + " bytes: " +
                                        cudaGetErrorString(e));
        }
        ctx->mds_w_bytes = bytes;
    } else {
        GBD_CUDA_TRY(cudaStreamWaitEvent(st, ctx->mds_w_done, 0));
    }
    *W = static_cast<uint16_t *>(ctx->mds_w);
    return GBD_OK;
}

int read_flags(MdsWork &w)
{
    uint32_t h[2] = {0, 0};
    GBD_CUDA_TRY(cudaMemcpyAsync(h, w.flags, sizeof(h), cudaMemcpyDeviceToHost, w.st));
    GBD_CUDA_TRY(cudaStreamSynchronize(w.st));
    if (h[0] != 0)
        return fail(GBD_ETIMEDOUT, "tensor-core product: a bounded wait ran out (code " + std::to_string(h[0]) + ")");
    if (h[1] & 2u) return fail(GBD_EINVAL, "eigensolver: non-finite input");
    if (h[1] & 1u) return fail(GBD_ECUDA, "eigensolver: Jacobi sweeps did not converge");
    return GBD_OK;
}

}  // namespace
}  // namespace gbd

using namespace gbd;

namespace gbd {
void free_mds_cache(gbd_ctx *ctx)
{
    if (ctx->mds_w) {
        if (ctx->mds_w_done) cudaEventSynchronize(ctx->mds_w_done);
        cudaFree(ctx->mds_w);
        ctx->mds_w = nullptr;
        ctx->mds_w_bytes = 0;
    }
    if (ctx->mds_w_done) {
        cudaEventDestroy(ctx->mds_w_done);
        ctx->mds_w_done = nullptr;
    }
    cudaGetLastError();
}
}  // namespace gbd

extern "C" int gbd_sqdist_square(gbd_ctx *ctx, const uint16_t *d_tri, uint64_t n, uint16_t *d_w, uint64_t ld,
                                 int32_t *shift, void *stream)
{
    return sqdist_square_impl(ctx, d_tri, n, d_w, ld, shift, static_cast<cudaStream_t>(stream));
}

extern "C" int gbd_gram_apply(gbd_ctx *ctx, const uint16_t *d_w, uint64_t n, uint64_t ld, int32_t shift,
                              const float *d_x, uint32_t k, float *d_y, void *stream)
{
    if (!ctx || !d_w || !d_x || !d_y) return fail(GBD_EINVAL, "NULL argument");
    if (ld == 0 || ld % 128 != 0 || ld < n || n == 0) return fail(GBD_EINVAL, "need 0 < n <= ld, ld a multiple of 128");
    if (k < 16 || k > 256 || k % 16 != 0) return fail(GBD_EINVAL, "k must be a multiple of 16 in [16, 256]");
    if (shift < 0 || shift > 64) return fail(GBD_EINVAL, "bad shift");
    const size_t xb = n * k * sizeof(float);
    const uintptr_t x0 = reinterpret_cast<uintptr_t>(d_x), y0 = reinterpret_cast<uintptr_t>(d_y);
    if (x0 < y0 + xb && y0 < x0 + xb) return fail(GBD_EINVAL, "X and Y overlap");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MdsWork w;
    int rc = w.init(n, ld, k, ctx->sm_count, st);
    if (rc == GBD_OK) rc = gram_apply_in(d_w, shift, d_x, d_y, w, ctx->sm_count);
    int frc = (rc == GBD_OK) ? read_flags(w) : rc;
    w.release();
    return frc;
}

extern "C" int gbd_mds(gbd_ctx *ctx, const uint16_t *d_tri, uint64_t n, const float *d_omega, uint32_t k,
                       uint32_t r, uint32_t q, float *d_lambda, float *d_coords, void *stream)
{
    if (!ctx || !d_tri || !d_omega || !d_lambda || !d_coords) return fail(GBD_EINVAL, "NULL argument");
    if (k < 16 || k > (uint32_t)kMaxJacobiK || k % 16 != 0)
        return fail(GBD_EINVAL, "k must be a multiple of 16 in [16, 112]");
    if (r == 0 || r > k) return fail(GBD_EINVAL, "need 0 < r <= k");
    if (n <= k) return fail(GBD_EINVAL, "need n > k");
    if (q > 16) return fail(GBD_EINVAL, "at most 16 rounds");
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    int rc = configure_kernels();
    if (rc != GBD_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t ld = (n + 127) / 128 * 128;
    MdsWork w;
    uint16_t *W = nullptr;
    float *Y = nullptr, *Q = nullptr;
    int32_t shift = 0;
    rc = w.init(n, ld, k, ctx->sm_count, st);
    if (rc == GBD_OK) rc = mds_square_buffer(ctx, (size_t)ld * ld * 2, st, &W);
    if (rc == GBD_OK) rc = w.alloc((void **)&Y, (size_t)n * k * 4);
    if (rc == GBD_OK) rc = w.alloc((void **)&Q, (size_t)n * k * 4);
    if (rc == GBD_OK) rc = sqdist_square_impl(ctx, d_tri, n, W, ld, &shift, st);
    // range finder: Q = orth(G Omega), then q rounds of two products (G is symmetric)
    if (rc == GBD_OK) rc = gram_apply_in(W, shift, d_omega, Y, w, ctx->sm_count);
    if (rc == GBD_OK) rc = orthonormalise(Y, Q, w, q == 0 ? 2 : 1);
    for (uint32_t t = 0; rc == GBD_OK && t < 2 * q; ++t) {
        rc = gram_apply_in(W, shift, Q, Y, w, ctx->sm_count);
        if (rc == GBD_OK) rc = orthonormalise(Y, Q, w, t + 1 == 2 * q ? 2 : 1);
    }
    // B = Q^T G Q, eigenpairs, coordinates Q V_r diag(sqrt(max(lambda, 0)))
    if (rc == GBD_OK) rc = gram_apply_in(W, shift, Q, Y, w, ctx->sm_count);
    if (rc == GBD_OK) rc = xty(Q, Y, w);
    if (rc == GBD_OK) {
        jacobi_kernel<<<1, 256, jacobi_smem_f32(k), st>>>(w.gram, k, r, w.T, d_lambda, w.flags + 1);
        note_launches(1);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) rc = cuda_fail(le, "jacobi_kernel launch");
    }
    if (rc == GBD_OK) rc = apply(Q, w.T, r, d_coords, w);
    if (W) cudaEventRecord(ctx->mds_w_done, st);
    int frc = (rc == GBD_OK) ? read_flags(w) : rc;
    w.release();
    return frc;
}
