// K0: validate ACGT bytes and pack reads into 2-bit words (ingest step of the path).
//
// Each thread produces one 32-bit word: 16 consecutive bases of one read, base k of
// the word in bits 2k..2k+1 with A=0, C=1, G=2, T=3.  Positions past the read's end
// are zero.  An invalid byte records its position (relative to offsets[0]) with an
// atomicMin, so the host reports the first one.
#include "gbd_internal.cuh"

namespace gbd {
namespace {

__global__ void pack_kernel(const uint8_t *__restrict__ seq, const uint64_t *__restrict__ off,
                            uint64_t n, uint32_t stride, uint32_t *__restrict__ words,
                            uint16_t *__restrict__ len, unsigned long long *err)
{
    const uint64_t total = n * (uint64_t)stride;
    const uint64_t origin = off[0];
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = t / stride;
        const uint32_t w = (uint32_t)(t - r * stride);
        const uint64_t s = off[r];
        // callers validate the offsets first; a read whose offsets decrease or whose
        // length exceeds the stride is packed as empty, so the bytes are never indexed
        // past it
        const uint64_t e = off[r + 1];
        const uint64_t L = (e < s || e - s > (uint64_t)stride * kBasesPerWord) ? 0 : e - s;
        if (w == 0) len[r] = (uint16_t)L;
        uint32_t word = 0;
        const uint64_t k0 = (uint64_t)w * kBasesPerWord;
#pragma unroll
        for (int k = 0; k < kBasesPerWord; ++k) {
            const uint64_t pos = k0 + k;
            if (pos < L) {
                const uint8_t c = seq[s + pos] | 0x20;   // 'A'/'a' -> 'a', ...
                uint32_t code = 0;
                bool ok = true;
                switch (c) {
                    case 'a': code = 0; break;
                    case 'c': code = 1; break;
                    case 'g': code = 2; break;
                    case 't': code = 3; break;
                    default: ok = false; break;
                }
                if (!ok) atomicMin(err, (unsigned long long)(s + pos - origin));
                word |= code << (2 * k);
            }
        }
        words[t] = word;
    }
}

}  // namespace

cudaError_t launch_pack(const uint8_t *seq, const uint64_t *offsets, uint64_t n, uint32_t stride,
                        uint32_t *words, uint16_t *len, unsigned long long *err,
                        cudaStream_t stream)
{
    const uint64_t total = n * (uint64_t)stride;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    uint64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    pack_kernel<<<(unsigned)blocks, threads, 0, stream>>>(seq, offsets, n, stride, words, len, err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace gbd
