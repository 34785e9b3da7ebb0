// Allocation-free rectangle of distances (gbd_tile_noalloc).
//
// Some callers cannot call cudaMalloc: their device memory belongs to another
// allocator (a framework's caching pool or a pre-reserved arena, where a direct
// cudaMalloc fails or fragments it), or they run code paths that must not allocate at
// all.  This entry point serves them: it takes the reads and the output buffer from the
// caller, and everything else it needs -- validation flags, the 2-bit packed copies of
// both read sets and the DP boundary rows -- lives in one fixed array in device memory,
// g_noalloc_scratch, of kNoAllocScratchBytes bytes.  The array is part of the library
// image: every GPU that loads the library holds it until the process exits.
//
// The work is the general pair kernel (one pair per thread, boundary rows in scratch),
// run on a rectangle with its boundary rows placed in the array.
#include <mutex>

#include "gbd_internal.cuh"

namespace gbd {
namespace {

constexpr uint64_t kNoAllocScratchBytes = 32ull << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host-side names of the array are host stand-ins, not device addresses: kernels get
// the address obtained from cudaGetSymbolAddress for the current device.
std::mutex g_setup_mu;
bool g_ready[kMaxDevices];
unsigned char *g_dev_ptr[kMaxDevices];

int scratch_for_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(GBD_EINVAL, "gbd_tile_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_ready[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
        g_ready[dev] = true;
    }
    *out = g_dev_ptr[dev];
    return GBD_OK;
}

// flag <- smallest read index whose offsets decrease or whose length exceeds max_len
__global__ void check_offsets_kernel(const uint64_t *__restrict__ off, uint64_t n, uint32_t max_len,
                                     unsigned long long *flag)
{
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = off[r], b = off[r + 1];
        if (b < a || b - a > max_len) atomicMin(flag, (unsigned long long)r);
    }
}

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

}  // namespace
}  // namespace gbd

using namespace gbd;

extern "C" int gbd_tile_noalloc(gbd_ctx *ctx, const uint8_t *d_seqA, const uint64_t *d_offA,
                                uint64_t nA, const uint8_t *d_seqB, const uint64_t *d_offB,
                                uint64_t nB, uint32_t max_len, uint16_t *d_out, uint64_t ld,
                                void *stream)
{
    if (!ctx) return fail(GBD_EINVAL, "gbd_tile_noalloc: NULL context");
    if (nA == 0 || nB == 0) return GBD_OK;
    if (!d_seqA || !d_seqB || !d_offA || !d_offB || !d_out)
        return fail(GBD_EINVAL, "gbd_tile_noalloc: NULL pointer");
    if (ld < nB) return fail(GBD_EINVAL, "gbd_tile_noalloc: ld is smaller than nB");
    if (max_len > 65535) return fail(GBD_EINVAL, "gbd_tile_noalloc: max_len above 65535");
    // layout: 4 flags | A words | A lengths | B words | B lengths | boundary rows
    const uint32_t stride = max_len == 0 ? 1u : (max_len + kBasesPerWord - 1) / kBasesPerWord;
    // every read set alone must fit the array: this keeps the products below from wrapping
    const uint64_t max_reads = kNoAllocScratchBytes / (4ull * stride);
    if (nA > max_reads || nB > max_reads)
        return fail(GBD_EINVAL, "gbd_tile_noalloc: more reads than the " + std::to_string(kNoAllocScratchBytes) +
                                    "-byte scratch array of the allocation-free entry point holds");
    cudaStream_t st = (cudaStream_t)stream;
    GBD_CUDA_TRY(cudaSetDevice(ctx->device));
    unsigned char *base = nullptr;
    int rc = scratch_for_device(ctx->device, &base);
    if (rc != GBD_OK) return rc;

    const uint64_t off_wA = 256;
    const uint64_t off_lA = align256(off_wA + nA * stride * 4);
    const uint64_t off_wB = align256(off_lA + nA * 2);
    const uint64_t off_lB = align256(off_wB + nB * stride * 4);
    const uint64_t off_bd = align256(off_lB + nB * 2);
    if (off_bd >= kNoAllocScratchBytes)
        return fail(GBD_EINVAL, "gbd_tile_noalloc: the packed reads need " + std::to_string(off_bd) +
                                    " bytes of scratch; the allocation-free entry point has " +
                                    std::to_string(kNoAllocScratchBytes));
    unsigned long long *flags = reinterpret_cast<unsigned long long *>(base);
    uint32_t *wA = reinterpret_cast<uint32_t *>(base + off_wA);
    uint16_t *lA = reinterpret_cast<uint16_t *>(base + off_lA);
    uint32_t *wB = reinterpret_cast<uint32_t *>(base + off_wB);
    uint16_t *lB = reinterpret_cast<uint16_t *>(base + off_lB);
    int *bnd = reinterpret_cast<int *>(base + off_bd);
    const uint64_t bnd_ints = (kNoAllocScratchBytes - off_bd) / sizeof(int);

    // the array keeps the previous call's contents: reset the flags (all ones = no error)
    GBD_CUDA_TRY(cudaMemsetAsync(flags, 0xff, 4 * sizeof(unsigned long long), st));
    check_offsets_kernel<<<64, 256, 0, st>>>(d_offA, nA, max_len, flags + 0);
    check_offsets_kernel<<<64, 256, 0, st>>>(d_offB, nB, max_len, flags + 1);
    note_launches(2);
    GBD_CUDA_TRY(cudaGetLastError());
    // the offsets are read back and checked before the pack kernels index the bytes with them
    unsigned long long h_flags[4];
    GBD_CUDA_TRY(cudaMemcpyAsync(h_flags, flags, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    GBD_CUDA_TRY(cudaStreamSynchronize(st));
    for (int s = 0; s < 2; ++s)
        if (h_flags[s] != ~0ull)
            return fail(GBD_EINVAL, std::string("gbd_tile_noalloc: read ") + std::to_string(h_flags[s]) +
                                        " of " + (s ? "B" : "A") +
                                        " is longer than max_len or its offsets decrease");
    GBD_CUDA_TRY(launch_pack(d_seqA, d_offA, nA, stride, wA, lA, flags + 2, st));
    GBD_CUDA_TRY(launch_pack(d_seqB, d_offB, nB, stride, wB, lB, flags + 3, st));
    GBD_CUDA_TRY(cudaMemcpyAsync(h_flags + 2, flags + 2, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    GBD_CUDA_TRY(cudaStreamSynchronize(st));
    for (int s = 0; s < 2; ++s)
        if (h_flags[2 + s] != ~0ull)
            return fail(GBD_EINVAL, std::string("gbd_tile_noalloc: byte at position ") +
                                        std::to_string(h_flags[2 + s]) + " of " + (s ? "B" : "A") +
                                        " is not one of A, C, G, T");
    GeneralJob job{{wA, lA, nA, stride}, {wB, lB, nB, stride}, 0, nA, 0, nB, ld, OUT_RECT, d_out};
    job.out_len = out_extent(ctx, (nA - 1) * ld + nB);
    const Scoring sc{ctx->params.match, ctx->params.mismatch, ctx->params.gap, ctx->params.conversion,
                     ctx->params.gap_open};
    return run_general_in(job, sc, bnd, bnd_ints, ctx->sm_count, st);
}
