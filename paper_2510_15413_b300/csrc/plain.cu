// plain.cu -- scan outputs that need no bootstrap.
//
// With plaintext query constants (the variant of §4.2 where an operand of
// the comparison is a plaintext) some outputs of a row are not gate outputs:
// the match bit can be a column bit or its negation (EQ of width 1, LT whose
// constant has one set bit), and when the match is a known bit every masked
// payload bit is the payload bit itself or a known 0.  This kernel writes
// them: a copy, a negation (every word negated mod 2^32: the phase changes
// sign, so the bit flips and the noise is kept) or the trivial ciphertext
// (0, .., 0, +-q/8) of a known bit.  HBM bound and tiny next to the gates.
#include <cuda_runtime.h>

#include "engine.h"

namespace fsql {
namespace {

constexpr int kLitThreads = 128;

__global__ void __launch_bounds__(kLitThreads) literal_kernel(const OutDesc* __restrict__ lits, size_t count, int n) {
  const uint32_t E = 1u << 29;  // q/8
  for (size_t i = blockIdx.x; i < count; i += gridDim.x) {
    const OutDesc d = lits[i];
    for (int x = threadIdx.x; x <= n; x += kLitThreads) {
      uint32_t v;
      if (d.mode == kOutCopy) v = d.src[x];
      else if (d.mode == kOutNegate) v = 0u - d.src[x];
      else v = x < n ? 0u : (d.mode == kOutTrue ? E : 0u - E);
      d.dst[x] = v;
    }
  }
}

}  // namespace

int launch_literals(const OutDesc* d_lits, size_t count, int n, void* stream) {
  if (count == 0) return FSQL_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t grid = count < static_cast<size_t>(16 * sms) ? count : static_cast<size_t>(16 * sms);
  literal_kernel<<<static_cast<unsigned>(grid), kLitThreads, 0, static_cast<cudaStream_t>(stream)>>>(d_lits, count,
                                                                                                       n);
  if (cudaGetLastError() != cudaSuccess) {
    set_error("literal output kernel launch failed");
    return FSQL_ERR_CUDA;
  }
  return FSQL_OK;
}

}  // namespace fsql
