// Tensor-core product P = W X for classical MDS (paper sections 3.2 and 6.2).
//
// W is the ld x ld fp16 matrix of scaled squared distances (row-major, K contiguous)
// and X^T the k x ld fp16 matrix of the centred test vectors (also K contiguous); P
// (ld x k, float32) is written as S partial products, one per slice of K, which a
// second kernel sums in a fixed order (deterministic results).
//
// One persistent CTA per SM runs a static round-robin list of work units
// (128-row block of W, K slice).  Warp roles:
//   warp 0      TMA producer: 128 x 64 tile of W and k x 64 tile of X^T per stage,
//               128-byte swizzled, completion counted on the stage's mbarrier;
//   warp 1      allocates TMEM (two k-column fp32 accumulators) and issues
//               tcgen05.mma (M = 128, N = k, K = 16; four per stage), committing
//               each stage back to the producer and each finished unit to the epilogue;
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (each warp its 32 TMEM lanes),
//               float4 stores of the partial rows, then release of the accumulator.
// Every mbarrier wait is bounded in time; a wait that runs out sets the error word,
// makes the other roles leave their loops, waits for its own copies and MMAs in flight
// and frees TMEM before the kernel returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "gbd_internal.cuh"
#include "mds_internal.cuh"

namespace gbd {
namespace {

constexpr int BM = 128;              // rows of W per unit (MMA M)
constexpr int BK = 64;               // K elements per stage (128 bytes of fp16)
constexpr int THREADS = 192;         // 6 warps
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s bound on any wait
constexpr uint64_t kDrainNs = 200000000ull;   // 0.2 s bound on the drain after an abort

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `parity` to complete.  Gives up (false) when the abort flag is
// raised or after `limit_ns`; a timeout raises the flag and records `code` in *err.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                         uint32_t *err, uint32_t code, uint64_t limit_ns,
                                         bool watch_abort = true)
{
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u) {
            if (watch_abort && *abort_flag) return false;
            if (globaltimer() - t0 > limit_ns) {
                *abort_flag = 1;
                if (err) atomicOr(err, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart.  Fields: start address >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29, unused for this layout), stride byte offset >> 4 (32-45),
// descriptor version 1 (46-47), base offset 0 (49-51), layout 2 = 128-byte swizzle (61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), A and B fp16
// (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct GemmShape {
    uint32_t k;           // columns of X (MMA N)
    uint32_t ld;          // rows and columns of W (multiple of 128)
    uint32_t nblk_m;      // ld / 128
    uint32_t nblk_k;      // ld / 64
    uint32_t slices;      // K slices
    uint32_t kb_per;      // K blocks per slice (the last slice may have fewer)
    uint32_t stages;
    uint32_t units;       // nblk_m * slices
};

__global__ void __launch_bounds__(THREADS, 1)
w_times_x_kernel(const __grid_constant__ CUtensorMap map_w, const __grid_constant__ CUtensorMap map_x,
                 GemmShape sh, float *__restrict__ part, uint32_t *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t a_bytes = BM * BK * 2;
    const uint32_t b_bytes = sh.k * BK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint8_t *tiles = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + sh.stages * stage_bytes);
    uint64_t *full = bars;                       // [stages]
    uint64_t *empty = bars + sh.stages;          // [stages]
    uint64_t *tfull = bars + 2 * sh.stages;      // [2]
    uint64_t *tempty = tfull + 2;                // [2]
    uint64_t *drain = tempty + 2;                // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t tmem_cols = sh.k * 2 <= 32 ? 32 : (sh.k * 2 <= 64 ? 64 : (sh.k * 2 <= 128 ? 128 : (sh.k * 2 <= 256 ? 256 : 512)));

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < sh.stages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), 4);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------------- producer
            uint32_t stage = 0, phase = 0;
            uint32_t issued_total = 0;
            bool ok = true;
            for (uint32_t u = blockIdx.x; ok && u < sh.units; u += gridDim.x) {
                const uint32_t mb = u / sh.slices, ks = u % sh.slices;
                const uint32_t kb0 = ks * sh.kb_per;
                const uint32_t kb1 = min(kb0 + sh.kb_per, sh.nblk_k);
                for (uint32_t kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, abort_flag, err, 1u, kWaitNs)) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = tiles + stage * stage_bytes;
                    const uint32_t fb = smem_u32(&full[stage]);
                    mbar_expect_tx(fb, stage_bytes);
                    tma_load_2d(smem_u32(st), &map_w, (int)(kb * BK), (int)(mb * BM), fb);
                    tma_load_2d(smem_u32(st + a_bytes), &map_x, (int)(kb * BK), 0, fb);
                    ++issued_total;
                    if (++stage == sh.stages) { stage = 0; phase ^= 1u; }
                }
            }
            // The last load issued into each stage completes phase (loads - 1) of its full
            // barrier: wait for those, so no copy lands after the block exits (immediate
            // when the MMA warp consumed them all).
            (void)ok;
            for (uint32_t s = 0; s < sh.stages; ++s) {
                const uint32_t loads = issued_total / sh.stages + (s < issued_total % sh.stages ? 1u : 0u);
                if (loads == 0) continue;
                mbar_wait(smem_u32(&full[s]), (loads - 1) & 1u, abort_flag, nullptr, 0, kDrainNs, false);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------------------- MMA issuer
            const uint32_t idesc = instr_desc(BM, (int)sh.k);
            uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
            bool ok = true;
            bool issued_any = false;
            for (uint32_t u = blockIdx.x; ok && u < sh.units; u += gridDim.x) {
                const uint32_t ks = u % sh.slices;
                const uint32_t kb0 = ks * sh.kb_per;
                const uint32_t kb1 = min(kb0 + sh.kb_per, sh.nblk_k);
                if (!mbar_wait(smem_u32(&tempty[acc]), acc_phase ^ 1u, abort_flag, err, 2u, kWaitNs)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + acc * sh.k;
                for (uint32_t kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(smem_u32(&full[stage]), phase, abort_flag, err, 4u, kWaitNs)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(tiles + stage * stage_bytes);
                    const uint64_t adesc = smem_desc(a_addr);
                    const uint64_t bdesc = smem_desc(a_addr + a_bytes);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        // +32 bytes along K inside the 128-byte swizzled row
                        mma_f16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc,
                                (kb > kb0 || kk > 0) ? 1u : 0u);
                    }
                    issued_any = true;
                    mma_commit(smem_u32(&empty[stage]));      // frees the stage once read
                    if (++stage == sh.stages) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(smem_u32(&tfull[acc]));            // accumulator complete
                if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
            }
            if (issued_any) {
                // every MMA issued so far has completed once this commit arrives
                mma_commit(smem_u32(drain));
                mbar_wait(smem_u32(drain), 0, abort_flag, nullptr, 0, kDrainNs, false);
            }
        }
    } else {
        // -------------------------------------------------------------------- epilogue
        const uint32_t quarter = (uint32_t)(warp & 3);       // TMEM lanes 32*quarter ...
        uint32_t acc = 0, acc_phase = 0;
        for (uint32_t u = blockIdx.x; u < sh.units; u += gridDim.x) {
            const uint32_t mb = u / sh.slices, ks = u % sh.slices;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(smem_u32(&tfull[acc]), acc_phase, abort_flag, err, 8u, kWaitNs);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            const uint32_t row = mb * BM + quarter * 32 + (uint32_t)lane;
            float *dst = part + ((uint64_t)ks * sh.ld + row) * sh.k;
            const uint32_t taddr = tmem_base + ((quarter * 32u) << 16) + acc * sh.k;
            for (uint32_t c = 0; c < sh.k; c += 16) {
                uint32_t v[16];
                tmem_ld16(taddr + c, v);
                float4 *d4 = reinterpret_cast<float4 *>(dst + c);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    d4[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                        __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
            if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encoder()
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (g_encode) return GBD_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr)
        return fail(GBD_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return GBD_OK;
}

// 2-D fp16 tensor map over a row-major rows x cols matrix (cols contiguous), tile box
// of box_rows x 64 elements, 128-byte swizzle.
int make_map(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint32_t box_rows)
{
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GBD_ECUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    return GBD_OK;
}

}  // namespace

uint32_t w_times_x_slices_used(uint64_t ld, uint32_t requested)
{
    const uint64_t nblk_k = ld / BK;
    const uint64_t req = std::max<uint64_t>(1, requested);
    const uint64_t per = (nblk_k + req - 1) / req;
    return (uint32_t)((nblk_k + per - 1) / per);
}

uint32_t w_times_x_slices(uint64_t ld, int sm_count)
{
    const uint64_t nblk_m = ld / BM, nblk_k = ld / BK;
    // enough units for ~16 per SM, slices of at least 8 K blocks
    uint64_t s = 1;
    while (s < 64 && nblk_m * s < (uint64_t)std::max(sm_count, 1) * 16 && nblk_k / (s * 2) >= 8) s *= 2;
    return w_times_x_slices_used(ld, (uint32_t)s);
}

int w_times_x(const uint16_t *d_w, uint64_t ld, const uint16_t *d_xt, uint32_t k, float *d_part,
              uint32_t slices, uint32_t *d_err, int sm_count, cudaStream_t stream)
{
    if (slices == 0 || slices != w_times_x_slices_used(ld, slices))
        return fail(GBD_EINVAL, "internal: slice count must come from w_times_x_slices");
    if (ld == 0 || ld % BM != 0 || k < 16 || k > 256 || k % 16 != 0)
        return fail(GBD_EINVAL, "internal: bad tensor-core product shape");
    if (reinterpret_cast<uintptr_t>(d_w) % 16 != 0 || reinterpret_cast<uintptr_t>(d_xt) % 16 != 0)
        return fail(GBD_EINVAL, "internal: tensor-core operands must be 16-byte aligned");
    int rc = get_encoder();
    if (rc != GBD_OK) return rc;
    CUtensorMap map_w, map_x;
    rc = make_map(&map_w, d_w, ld, ld, BM);
    if (rc == GBD_OK) rc = make_map(&map_x, d_xt, ld, k, k);
    if (rc != GBD_OK) return rc;

    GemmShape sh;
    sh.k = k;
    sh.ld = (uint32_t)ld;
    sh.nblk_m = (uint32_t)(ld / BM);
    sh.nblk_k = (uint32_t)(ld / BK);
    // every slice gets at least one K block
    sh.kb_per = (sh.nblk_k + std::max(1u, slices) - 1) / std::max(1u, slices);
    sh.slices = (sh.nblk_k + sh.kb_per - 1) / sh.kb_per;
    const uint32_t stage_bytes = BM * BK * 2 + k * BK * 2;
    sh.stages = std::min(8u, (uint32_t)((196u * 1024u) / stage_bytes));
    sh.units = sh.nblk_m * sh.slices;
    const size_t smem = 1024 + (size_t)sh.stages * stage_bytes + (2 * sh.stages + 5) * 8 + 16;
    static std::once_flag attr_once;
    cudaError_t ae = cudaSuccess;
    std::call_once(attr_once, [&] {
        ae = cudaFuncSetAttribute(w_times_x_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (ae != cudaSuccess) return cuda_fail(ae, "cudaFuncSetAttribute(w_times_x_kernel)");
    const uint32_t grid = std::min<uint32_t>(sh.units, (uint32_t)std::max(sm_count, 1));
    w_times_x_kernel<<<grid, THREADS, smem, stream>>>(map_w, map_x, sh, d_part, d_err);
    note_launches(1);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return cuda_fail(le, "w_times_x_kernel launch");
    return GBD_OK;
}

}  // namespace gbd
