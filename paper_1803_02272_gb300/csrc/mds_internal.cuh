// Internal declarations of the classical-MDS kernels (paper sections 3 and 6.2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbd {

// K slices of the tensor-core product for an ld x ld W (each slice non-empty), and the
// slice count that a requested count turns into.
uint32_t w_times_x_slices(uint64_t ld, int sm_count);
uint32_t w_times_x_slices_used(uint64_t ld, uint32_t requested);

// part[s][i][c] = sum over the K blocks of slice s of W[i][j] * Xt[c][j]  (fp16 inputs,
// fp32 accumulation on tcgen05), for i < ld, c < k.  part holds slices * ld * k floats.
// *d_err receives a non-zero code if a bounded wait inside the kernel ran out.
int w_times_x(const uint16_t *d_w, uint64_t ld, const uint16_t *d_xt, uint32_t k, float *d_part,
              uint32_t slices, uint32_t *d_err, int sm_count, cudaStream_t stream);

}  // namespace gbd
