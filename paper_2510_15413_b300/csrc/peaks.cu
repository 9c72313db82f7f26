// peaks.cu -- in-register microkernels that measure the integer-ALU rates
// the blind rotation is bound by, so that its roofline fraction divides by a
// measured peak rather than an assumed unit count:
//   - 32-bit multiply-add (IMAD), high-half multiply (IMAD.HI) and widening
//     multiply-add into 64 bits (IMAD.WIDE): raw pipe rates;
//   - one forward butterfly of the two-prime engine (a Shoup product by a
//     twiddle and its add / subtract, exactly the code the NTT runs);
//   - one butterfly mod the 64-bit prime p = 2^64 - 2^32 + 1 (Goldilocks).
// Every kernel keeps kChains independent chains per thread so that
// dependency latency is hidden, loops a fixed number of times and writes one
// word per thread (so nothing is optimised away); the grid is a whole number
// of waves (4 CTAs of 256 threads per SM).  Nothing waits on anything but
// kernel completion.
#include <cuda_runtime.h>

#include <string>

#include "engine.h"
#include "ntt.cuh"

namespace fsql {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;

__global__ void __launch_bounds__(kPeakThreads) imad_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + threadIdx.x * 7u + c;
  const uint32_t m = seed | 1u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(m), "r"(x[(c + 1) % kChains]));
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) imadhi_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + threadIdx.x * 7u + c;
  const uint32_t m = seed | 0x80000001u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(m), "r"(x[(c + 1) % kChains]));
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) imadwide_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint64_t x[kChains];
  uint32_t y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = seed + threadIdx.x * 7ull + c;
    y[c] = seed ^ (threadIdx.x + 3u * c);
  }
  const uint32_t m = seed | 1u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(x[c]) : "r"(y[c]), "r"(m));
  }
  uint64_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = static_cast<uint32_t>(s ^ (s >> 32));
}

// Forward butterflies of the two-prime engine on one prime's residues:
// the lazy Cooley-Tukey step of the transform (Shoup product by a twiddle,
// then x + t and x - t + 2p), run as the transform runs them: 10 radix-2
// stages over 8 registers (distances 4, 2, 1, repeated), two independent
// polynomials per thread.  After the 10 stages every value is masked below
// 2^26 (one logic op per value, 16 per 80 butterflies) so that the next
// round starts inside the transform's input range again.
template <int D>
__device__ __forceinline__ void dp_stage(uint32_t (&x)[8], const uint32_t (&w)[4], const uint32_t (&ws)[4]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & D) continue;
    x[k] = dev::DualPrime::ct1(x[k], x[k + D], w[k & 3], ws[k & 3], dev::kP1);
  }
}

__global__ void __launch_bounds__(kPeakThreads) shoup_bfly_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint32_t x[8], y[8], w[4], ws[4];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = (seed + threadIdx.x * 13u + k) & 0x3FFFFFFu;
    y[k] = (seed ^ (threadIdx.x * 29u + 5u * k)) & 0x3FFFFFFu;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[k] = (seed * 2654435761u + 977u * k) % dev::kP1;
    ws[k] = static_cast<uint32_t>((static_cast<uint64_t>(w[k]) << 32) / dev::kP1);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dp_stage<4>(x, w, ws);
      dp_stage<4>(y, w, ws);
      dp_stage<2>(x, w, ws);
      dp_stage<2>(y, w, ws);
      dp_stage<1>(x, w, ws);
      dp_stage<1>(y, w, ws);
    }
    dp_stage<1>(x, w, ws);
    dp_stage<1>(y, w, ws);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x[k] &= 0x3FFFFFFu;
      y[k] &= 0x3FFFFFFu;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= x[k] ^ y[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same butterflies with the Shoup quotient taken from the high word of
// a widening 32 x 32 -> 64-bit multiply (mode 1) or multiply-add with a
// zero addend that is only known at run time (mode 2), instead of the
// high-half multiply: the three ways the engine can form floor(a w' / 2^32).
template <int kMode>
__device__ __forceinline__ uint32_t quot(uint32_t a, uint32_t ws, uint64_t zero) {
  if (kMode == 0) return __umulhi(a, ws);
  uint64_t r;
  if (kMode == 1) asm("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(a), "r"(ws));
  else asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(ws), "l"(zero));
  return static_cast<uint32_t>(r >> 32);
}
template <int kMode, int D>
__device__ __forceinline__ void dpw_stage(uint32_t (&x)[8], const uint32_t (&w)[4], const uint32_t (&ws)[4],
                                          uint64_t zero) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & D) continue;
    const uint32_t hi = x[k + D];
    const uint32_t t = hi * w[k & 3] - quot<kMode>(hi, ws[k & 3], zero) * dev::kP1;
    x[k + D] = x[k] - t + 2 * dev::kP1;
    x[k] = x[k] + t;
  }
}
template <int kMode>
__global__ void __launch_bounds__(kPeakThreads) shoup_mode_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint32_t x[8], y[8], w[4], ws[4];
  const uint64_t zero = seed >> 31;  // 0 for the seeds used here, unknown to the compiler
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = (seed + threadIdx.x * 13u + k) & 0x3FFFFFFu;
    y[k] = (seed ^ (threadIdx.x * 29u + 5u * k)) & 0x3FFFFFFu;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[k] = (seed * 2654435761u + 977u * k) % dev::kP1;
    ws[k] = static_cast<uint32_t>((static_cast<uint64_t>(w[k]) << 32) / dev::kP1);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dpw_stage<kMode, 4>(x, w, ws, zero);
      dpw_stage<kMode, 4>(y, w, ws, zero);
      dpw_stage<kMode, 2>(x, w, ws, zero);
      dpw_stage<kMode, 2>(y, w, ws, zero);
      dpw_stage<kMode, 1>(x, w, ws, zero);
      dpw_stage<kMode, 1>(y, w, ws, zero);
    }
    dpw_stage<kMode, 1>(x, w, ws, zero);
    dpw_stage<kMode, 1>(y, w, ws, zero);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x[k] &= 0x3FFFFFFu;
      y[k] &= 0x3FFFFFFu;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= x[k] ^ y[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Butterflies mod the 64-bit prime (the Goldilocks engine's forward step:
// one modular product, a modular add and subtract; canonical residues, so
// no masking), the same 10-stage pattern over 8 registers.
template <int D>
__device__ __forceinline__ void gl_stage(uint64_t (&x)[8], const uint64_t (&w)[4]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & D) continue;
    dev::Goldilocks::ct(x[k], x[k + D], w[k & 3]);
  }
}

__global__ void __launch_bounds__(kPeakThreads) goldilocks_bfly_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint64_t x[8], w[4];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (seed + threadIdx.x * 0x9E3779B97F4A7C15ull + k) % kP;
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = (seed * 0x94D049BB133111EBull + 31ull * k) % kP;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      gl_stage<4>(x, w);
      gl_stage<2>(x, w);
      gl_stage<1>(x, w);
    }
    gl_stage<1>(x, w);
  }
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = static_cast<uint32_t>(s ^ (s >> 32));
}

template <class K>
cudaError_t time_kernel(K kernel, int grid, uint32_t* d_out, int iters, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  kernel<<<grid, kPeakThreads>>>(d_out, iters / 4 + 1, 12345u);  // warm-up
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) kernel<<<grid, kPeakThreads>>>(d_out, iters, 12345u);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  return e;
}

}  // namespace
}  // namespace fsql

extern "C" int fsql_measure_alu_peaks(int device, fsql_alu_peaks* out) {
  using namespace fsql;
  if (!out) {
    set_error("null output");
    return FSQL_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    set_error("cudaSetDevice failed");
    return FSQL_ERR_ARG;
  }
  int sms = 0, clock_khz = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
    set_error("cannot read the SM count");
    return FSQL_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, device);
  const int grid = sms * kPeakCtasPerSm;
  uint32_t* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&d_out, static_cast<size_t>(grid) * kPeakThreads * 4);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const double threads = static_cast<double>(grid) * kPeakThreads;
  const double per_iter = 8.0 * kChains;  // operations per thread per loop iteration
  float ms = 0.f;
  // iteration counts sized for tens of milliseconds per kernel
  const int it_mul = 50000, it_bfly = 10000, it_gl = 2500;
  if (e == cudaSuccess) e = time_kernel(imad_kernel, grid, d_out, it_mul, e0, e1, &ms);
  if (e == cudaSuccess) out->imad_per_s = threads * per_iter * it_mul / (ms * 1e-3);
  if (e == cudaSuccess) e = time_kernel(imadhi_kernel, grid, d_out, it_mul, e0, e1, &ms);
  if (e == cudaSuccess) out->imad_hi_per_s = threads * per_iter * it_mul / (ms * 1e-3);
  if (e == cudaSuccess) e = time_kernel(imadwide_kernel, grid, d_out, it_mul, e0, e1, &ms);
  if (e == cudaSuccess) out->imad_wide_per_s = threads * per_iter * it_mul / (ms * 1e-3);
  if (e == cudaSuccess) e = time_kernel(shoup_bfly_kernel, grid, d_out, it_bfly, e0, e1, &ms);
  if (e == cudaSuccess) out->dual_prime_bfly_per_s = threads * 80.0 * it_bfly / (ms * 1e-3);
  if (e == cudaSuccess) e = time_kernel(shoup_mode_kernel<1>, grid, d_out, it_bfly, e0, e1, &ms);
  if (e == cudaSuccess) out->dual_prime_bfly_wide_per_s = threads * 80.0 * it_bfly / (ms * 1e-3);
  if (e == cudaSuccess) e = time_kernel(shoup_mode_kernel<2>, grid, d_out, it_bfly, e0, e1, &ms);
  if (e == cudaSuccess) out->dual_prime_bfly_madwide_per_s = threads * 80.0 * it_bfly / (ms * 1e-3);
  if (e == cudaSuccess) e = time_kernel(goldilocks_bfly_kernel, grid, d_out, it_gl, e0, e1, &ms);
  if (e == cudaSuccess) out->goldilocks_bfly_per_s = threads * 40.0 * it_gl / (ms * 1e-3);
  out->sm_count = sms;
  out->clock_mhz = clock_khz / 1000.0;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_out);
  if (e != cudaSuccess) {
    set_error(std::string("ALU peak microkernels: ") + cudaGetErrorString(e));
    return FSQL_ERR_CUDA;
  }
  return FSQL_OK;
}
