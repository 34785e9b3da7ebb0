// Instruction-rate probe: how many lane operations per second one GB300 issues for
// each instruction form the DP inner loops use.  The integer DP is bound by the
// issue rate of these operations (no tensor-core or HBM bound applies), so the
// measured rates are the denominators of its roofline.
//
// Each thread runs 8 interleaved dependency chains (enough independent work to hide
// latency at full occupancy); every operation's result feeds the next one, and the
// chains are folded into one store so nothing can be removed as dead code.
#include <cuda_fp16.h>

#include "gbd_internal.cuh"

namespace gbd {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <int OP>
__device__ __forceinline__ uint32_t apply(uint32_t x, uint32_t y, uint32_t k)
{
    if constexpr (OP == GBD_PROBE_VIMAX3_S16X2_RELU) return __vimax3_s16x2_relu(x, y, k);
    else if constexpr (OP == GBD_PROBE_VIADDMAX_S16X2) return __viaddmax_s16x2(x, k, y);
    else if constexpr (OP == GBD_PROBE_VIADDMAX_S16X2_RELU) return __viaddmax_s16x2_relu(x, k, y);
    else if constexpr (OP == GBD_PROBE_VIMAX_S16X2_RELU) return __vimax_s16x2_relu(x, y);
    else if constexpr (OP == GBD_PROBE_VMAXS2) return __vmaxs2(x, y);
    else if constexpr (OP == GBD_PROBE_PRMT) return __byte_perm(x, y, x);
    else if constexpr (OP == GBD_PROBE_IADD3) return x + y + k;
    else if constexpr (OP == GBD_PROBE_LOP3) {
        uint32_t r;
        asm("lop3.b32 %0, %1, %2, %3, 0x6a;" : "=r"(r) : "r"(x), "r"(y), "r"(k));
        return r;
    }
    else if constexpr (OP == GBD_PROBE_IMAX) return (uint32_t)max((int)x, (int)y);
    else if constexpr (OP == GBD_PROBE_HMAX2) {
        __half2 a = *reinterpret_cast<__half2 *>(&x), b = *reinterpret_cast<__half2 *>(&y);
        __half2 r = __hmax2(a, b);
        return *reinterpret_cast<uint32_t *>(&r);
    } else if constexpr (OP == GBD_PROBE_HADD2) {
        __half2 a = *reinterpret_cast<__half2 *>(&x), b = *reinterpret_cast<__half2 *>(&y);
        __half2 r = __hadd2(a, b);
        return *reinterpret_cast<uint32_t *>(&r);
    } else if constexpr (OP == GBD_PROBE_VIMAX3_S16X2) return __vimax3_s16x2(x, y, k);
    else if constexpr (OP == GBD_PROBE_FMAX) {
        return __float_as_uint(fmaxf(__uint_as_float(x), __uint_as_float(y)));
    } else if constexpr (OP == GBD_PROBE_FMAX3) {
        float d;
        asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(__uint_as_float(x)), "f"(__uint_as_float(y)),
            "f"(__uint_as_float(k)));
        return __float_as_uint(d);
    } else if constexpr (OP == GBD_PROBE_FADD) {
        return __float_as_uint(__fadd_rn(__uint_as_float(x), __uint_as_float(y)));
    } else if constexpr (OP == GBD_PROBE_VIMAX3_U16X2) return __vimax3_u16x2(x, y, k);
    else if constexpr (OP == GBD_PROBE_VMINU2) return __vminu2(x, y);
    else if constexpr (OP == GBD_PROBE_VSETLEU2) return __vsetleu2(x, y) ^ k;
    else if constexpr (OP == GBD_PROBE_VIBMIN_U16X2) {
        bool hi, lo;
        const uint32_t m = __vibmin_u16x2(x, y, &hi, &lo);
        return m + (uint32_t)hi;
    } else return x ^ y;
}

// Two instruction forms on interleaved chains: even chains run A, odd chains run B.
template <int OP>
__device__ __forceinline__ uint32_t apply_mix(int c, uint32_t x, uint32_t y, uint32_t k)
{
    if (c & 1) {
        if constexpr (OP == GBD_PROBE_MIX_DPX_HMAX2) return apply<GBD_PROBE_HMAX2>(x, y, k);
        else if constexpr (OP == GBD_PROBE_MIX_DPX_FMAX3) return apply<GBD_PROBE_FMAX3>(x, y, k);
        else return apply<GBD_PROBE_IADD3>(x, y, k);
    }
    return apply<GBD_PROBE_VIMAX3_S16X2>(x, y, k);
}

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(uint32_t iters, uint32_t seed,
                                                    uint32_t *sink)
{
    uint32_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (threadIdx.x * 2654435761u) ^ (seed + 77u * c);
    const uint32_t k = seed | 0x00010001u;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (OP >= GBD_PROBE_MIX_DPX_HMAX2)
                    x[c] = apply_mix<OP>(c, x[c], x[(c + 2) % kChains], k);
                else
                    x[c] = apply<OP>(x[c], x[(c + 1) % kChains], k);
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= x[c];
    if (acc == seed) sink[blockIdx.x] = acc;   // practically never taken, never provable
}

// One DP cell of the anti-diagonal int16x2 form: score by byte permute, diagonal plus
// score against the floor, then the 3-way max.  Counted as 3 lane operations.
__global__ void __launch_bounds__(256) probe_cell_kernel(uint32_t iters, uint32_t seed,
                                                         uint32_t *sink)
{
    uint32_t v[kChains], d[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        v[c] = (threadIdx.x * 2654435761u) ^ (seed + 77u * c);
        d[c] = v[c] ^ 0x5a5a5a5au;
    }
    const uint32_t prof = 0x01030101u ^ (seed & 0x0202u);
    uint32_t f = seed & 0x00ff00ffu;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                const uint32_t s = __byte_perm(prof, 0x80018001u, v[c]);
                const uint32_t e = __viaddmax_s16x2(d[c], s, f);
                d[c] = v[c];
                v[c] = __vimax3_s16x2(v[c], v[(c + 1) % kChains], e);
            }
            f += 0x00010001u;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= v[c] ^ d[c];
    if (acc == seed) sink[blockIdx.x] = acc;
}

template <int OP>
void launch_probe(unsigned blocks, uint32_t iters, uint32_t *sink, cudaStream_t st)
{
    probe_kernel<OP><<<blocks, 256, 0, st>>>(iters, 0x9e3779b9u, sink);
}

}  // namespace

int probe_op_rate(int op, uint32_t iters, double *rate, int sm_count, cudaStream_t stream)
{
    if (op < 0 || op >= GBD_PROBE_COUNT || rate == nullptr || iters == 0)
        return fail(GBD_EINVAL, "probe_op_rate: bad op, iters or output pointer");
    const unsigned blocks = (unsigned)std::max(sm_count, 1) * 8u;
    uint32_t *sink = nullptr;
    GBD_CUDA_TRY(cudaMallocAsync((void **)&sink, blocks * sizeof(uint32_t), stream));
    cudaEvent_t e0, e1;
    GBD_CUDA_TRY(cudaEventCreate(&e0));
    GBD_CUDA_TRY(cudaEventCreate(&e1));
    auto run = [&](uint32_t it) {
        switch (op) {
            case GBD_PROBE_VIMAX3_S16X2_RELU: launch_probe<GBD_PROBE_VIMAX3_S16X2_RELU>(blocks, it, sink, stream); break;
            case GBD_PROBE_VIADDMAX_S16X2: launch_probe<GBD_PROBE_VIADDMAX_S16X2>(blocks, it, sink, stream); break;
            case GBD_PROBE_VIADDMAX_S16X2_RELU: launch_probe<GBD_PROBE_VIADDMAX_S16X2_RELU>(blocks, it, sink, stream); break;
            case GBD_PROBE_VIMAX_S16X2_RELU: launch_probe<GBD_PROBE_VIMAX_S16X2_RELU>(blocks, it, sink, stream); break;
            case GBD_PROBE_VMAXS2: launch_probe<GBD_PROBE_VMAXS2>(blocks, it, sink, stream); break;
            case GBD_PROBE_PRMT: launch_probe<GBD_PROBE_PRMT>(blocks, it, sink, stream); break;
            case GBD_PROBE_IADD3: launch_probe<GBD_PROBE_IADD3>(blocks, it, sink, stream); break;
            case GBD_PROBE_LOP3: launch_probe<GBD_PROBE_LOP3>(blocks, it, sink, stream); break;
            case GBD_PROBE_IMAX: launch_probe<GBD_PROBE_IMAX>(blocks, it, sink, stream); break;
            case GBD_PROBE_HMAX2: launch_probe<GBD_PROBE_HMAX2>(blocks, it, sink, stream); break;
            case GBD_PROBE_HADD2: launch_probe<GBD_PROBE_HADD2>(blocks, it, sink, stream); break;
            case GBD_PROBE_VIMAX3_S16X2: launch_probe<GBD_PROBE_VIMAX3_S16X2>(blocks, it, sink, stream); break;
            case GBD_PROBE_FMAX: launch_probe<GBD_PROBE_FMAX>(blocks, it, sink, stream); break;
            case GBD_PROBE_FMAX3: launch_probe<GBD_PROBE_FMAX3>(blocks, it, sink, stream); break;
            case GBD_PROBE_FADD: launch_probe<GBD_PROBE_FADD>(blocks, it, sink, stream); break;
            case GBD_PROBE_MIX_DPX_HMAX2: launch_probe<GBD_PROBE_MIX_DPX_HMAX2>(blocks, it, sink, stream); break;
            case GBD_PROBE_MIX_DPX_FMAX3: launch_probe<GBD_PROBE_MIX_DPX_FMAX3>(blocks, it, sink, stream); break;
            case GBD_PROBE_MIX_DPX_IADD3: launch_probe<GBD_PROBE_MIX_DPX_IADD3>(blocks, it, sink, stream); break;
            case GBD_PROBE_VIMAX3_U16X2: launch_probe<GBD_PROBE_VIMAX3_U16X2>(blocks, it, sink, stream); break;
            case GBD_PROBE_VMINU2: launch_probe<GBD_PROBE_VMINU2>(blocks, it, sink, stream); break;
            case GBD_PROBE_VSETLEU2: launch_probe<GBD_PROBE_VSETLEU2>(blocks, it, sink, stream); break;
            case GBD_PROBE_VIBMIN_U16X2: launch_probe<GBD_PROBE_VIBMIN_U16X2>(blocks, it, sink, stream); break;
            case GBD_PROBE_CELL_MIX: probe_cell_kernel<<<blocks, 256, 0, stream>>>(it, 0x9e3779b9u, sink); break;
        }
    };
    note_launches(2);
    run(std::max(1u, iters / 16));          // warm-up
    cudaEventRecord(e0, stream);
    run(iters);
    cudaEventRecord(e1, stream);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, stream);
    if (err != cudaSuccess) return cuda_fail(err, "probe kernel");
    const double per_iter = (op == GBD_PROBE_CELL_MIX) ? 3.0 * kUnroll * kChains
                                                        : (double)kUnroll * kChains;
    const double lane_ops = (double)blocks * 256.0 * (double)iters * per_iter;
    *rate = lane_ops / (ms * 1e-3);
    return GBD_OK;
}

}  // namespace gbd
