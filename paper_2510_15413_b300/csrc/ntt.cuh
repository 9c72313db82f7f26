// ntt.cuh -- exact arithmetic mod the Goldilocks prime p = 2^64 - 2^32 + 1 and
// a warp-resident 1024-point negacyclic NTT.
//
// Why this transform is exact for the blind rotation: the external product
// multiplies digit polynomials with coefficients in [-2^(bg-1), 2^(bg-1)) by
// key polynomials with coefficients in [0, 2^32) and sums 2l such products, so
// every coefficient of the integer result is below 2l * N * 2^(bg-1) * 2^32
// = 2^51.6 in magnitude for N = 1024, bg = 7, l = 3, far inside (-p/2, p/2).
// The product computed mod p therefore lifts back to the exact integer, and
// reducing that mod 2^32 gives the Torus32 result with no rounding.
//
// Register layout.  A warp holds one polynomial of 1024 coefficients, 32 per
// lane.  Layout A: lane L, register j holds element L + 32 j.  Layout B: lane
// L, register j holds element 32 L + j.  A butterfly whose distance is a
// multiple of 32 pairs registers of one lane in layout A; one with distance
// below 32 pairs registers of one lane in layout B.  Each transform runs its
// five long-distance stages in one layout, transposes once through a
// swizzled 8 KB shared-memory tile, and runs the five short-distance stages
// in the other layout, so butterflies never cross lanes.
//
// Forward: Cooley-Tukey, natural order in, bit-reversed order out, with the
// negacyclic twist folded into the twiddles psi^bitrev(k), psi a primitive
// 2048-th root of unity (Longa & Naehrig, CANS 2016).  Inverse: Gentleman-
// Sande with psi^-bitrev(k), bit-reversed in, natural out, without the final
// 1/N (the caller folds 1/N into one operand).  Forward input is layout A,
// forward output and inverse input are layout B, inverse output is layout A.
#pragma once

#include <cstdint>

#include "engine.h"

namespace fsql {
namespace dev {

constexpr uint64_t kEps = 0xFFFFFFFFull;  // 2^64 mod p

// a, b in [0, p): a + b mod p.  On carry out of 64 bits the dropped 2^64 is
// worth kEps; a + b < 2p keeps the corrected sum below p.
__device__ __forceinline__ uint64_t gl_add(uint64_t a, uint64_t b) {
  uint64_t s = a + b;
  if (s < a) return s + kEps;
  return s >= kP ? s - kP : s;
}

// a, b in [0, p): a - b mod p.  On borrow the wrapped value is 2^64 too big,
// i.e. kEps too big modulo p.
__device__ __forceinline__ uint64_t gl_sub(uint64_t a, uint64_t b) {
  uint64_t d = a - b;
  return a < b ? d - kEps : d;
}

// 128-bit value hi*2^64 + lo reduced mod p, using 2^64 = 2^32 - 1 and
// 2^96 = -1 (mod p): with hi = h1*2^32 + h0, value = lo - h1 + h0*(2^32 - 1).
__device__ __forceinline__ uint64_t gl_reduce(uint64_t lo, uint64_t hi) {
  const uint64_t h1 = hi >> 32;
  const uint64_t h0 = hi & kEps;
  uint64_t t = lo - h1;
  if (lo < h1) t -= kEps;
  const uint64_t m = (h0 << 32) - h0;
  uint64_t r = t + m;
  if (r < m) r += kEps;
  return r >= kP ? r - kP : r;
}

__device__ __forceinline__ uint64_t gl_mul(uint64_t a, uint64_t b) { return gl_reduce(a * b, __umul64hi(a, b)); }

// Signed integer v (|v| < p/2) as an element of Z_p.
__device__ __forceinline__ uint64_t gl_from_int(int32_t v) {
  return v < 0 ? kP - static_cast<uint64_t>(-static_cast<int64_t>(v)) : static_cast<uint64_t>(v);
}

// Centered lift of x in [0, p) to (-p/2, p/2), reduced mod 2^32.  Since
// p = 1 mod 2^32, x - p = x - 1 mod 2^32.
__device__ __forceinline__ uint32_t gl_lift32(uint64_t x) {
  return static_cast<uint32_t>(x) - (x > (kP >> 1) ? 1u : 0u);
}

// Swizzled slot of element (row r, column c) of a 32 x 32 tile of u64:
// row-wise and column-wise warp accesses both touch 16 distinct 8-byte bank
// pairs per half warp.
__device__ __forceinline__ int tile_slot(int r, int c) { return r * 32 + (c ^ r); }

// Forward negacyclic NTT of one polynomial held by the warp (layout A in,
// layout B out).  tile: this warp's 1024-u64 shared-memory tile.
__device__ __forceinline__ void ntt_forward(uint64_t (&x)[32], uint64_t* tile, const NttTables& T, int lane) {
  // distances 512 .. 32 (m = 1 .. 16 groups): partner register j + 16>>s
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int d = 16 >> s;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j & d) continue;
      const uint64_t w = T.fwd_uniform[(1 << s) + j / (2 * d)];
      const uint64_t v = gl_mul(x[j + d], w);
      const uint64_t u = x[j];
      x[j] = gl_add(u, v);
      x[j + d] = gl_sub(u, v);
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) tile[tile_slot(j, lane)] = x[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) x[j] = tile[tile_slot(lane, j)];
  // distances 16 .. 1: partner register j + 16>>s, per-lane twiddles
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int d = 16 >> s;
    const int off = (1 << s) - 1;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j & d) continue;
      const uint64_t w = T.fwd_lane[(off + j / (2 * d)) * 32 + lane];
      const uint64_t v = gl_mul(x[j + d], w);
      const uint64_t u = x[j];
      x[j] = gl_add(u, v);
      x[j + d] = gl_sub(u, v);
    }
  }
}

// Inverse negacyclic NTT without the 1/N factor (layout B in, layout A out).
__device__ __forceinline__ void ntt_inverse(uint64_t (&x)[32], uint64_t* tile, const NttTables& T, int lane) {
  // distances 1 .. 16: partner register j + (1<<s), per-lane twiddles
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int d = 1 << s;
    const int off = 32 - (32 >> s);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j & d) continue;
      const uint64_t w = T.inv_lane[(off + j / (2 * d)) * 32 + lane];
      const uint64_t u = x[j], v = x[j + d];
      x[j] = gl_add(u, v);
      x[j + d] = gl_mul(gl_sub(u, v), w);
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) tile[tile_slot(lane, j)] = x[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) x[j] = tile[tile_slot(j, lane)];
  // distances 32 .. 512: partner register j + (1<<s), uniform twiddles
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int d = 1 << s;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j & d) continue;
      const uint64_t w = T.inv_uniform[(16 >> s) + j / (2 * d)];
      const uint64_t u = x[j], v = x[j + d];
      x[j] = gl_add(u, v);
      x[j + d] = gl_mul(gl_sub(u, v), w);
    }
  }
}

}  // namespace dev
}  // namespace fsql
