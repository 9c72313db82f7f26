// ntt.cuh -- exact arithmetic mod the Goldilocks prime p = 2^64 - 2^32 + 1 and
// a 1024-point negacyclic NTT computed by 128 threads holding 8 coefficients
// each.
//
// Why this transform is exact for the blind rotation: the external product
// multiplies digit polynomials with coefficients in [-2^(bg-1), 2^(bg-1)) by
// key polynomials with coefficients in [0, 2^32) and sums 2l such products, so
// every coefficient of the integer result is below 2l * N * 2^(bg-1) * 2^32
// = 2^51.6 in magnitude for N = 1024, bg = 7, l = 3, far inside (-p/2, p/2).
// The product computed mod p therefore lifts back to the exact integer, and
// reducing that mod 2^32 gives the Torus32 result with no rounding.
//
// Transform.  Forward: Cooley-Tukey, natural order in, bit-reversed order out,
// negacyclic twist folded into the twiddles psi^bitrev(k) (psi a primitive
// 2048-th root of unity; Longa & Naehrig, CANS 2016).  Inverse: Gentleman-Sande
// with psi^-bitrev(k), bit-reversed in, natural out, without the final 1/N
// (the caller folds 1/N into one operand).
//
// Work split.  The 10 radix-2 stages run as four passes over registers:
// 3 + 3 + 3 + 1 stages forward, 3 + 3 + 3 + 1 inverse.  Within a pass every
// butterfly pairs two registers of one thread; between passes the 1024
// values go through an 8 KB shared-memory buffer (one named barrier of the
// 128 threads).  Thread t, register k holds element
//   F1: t + 128k         F2: 128(t>>4) + 16k + (t&15)     F3: 16(t>>1) + 2k + (t&1)
//   F4 = I1: 8t + k      I2: 64(t>>3) + 8k + (t&7)         I3: 512(t>>6) + 64k + (t&63)
//   I4 = F1.
// The forward output layout (F4) is the inverse input layout (I1), so the
// pointwise products need no exchange.  The buffer index of element e is
// swizzled, e ^ ((e >> 3) & 15) on its low four bits, which makes every one
// of these patterns hit 16 distinct 8-byte bank pairs per half warp.
#pragma once

#include <cstdint>

#include "engine.h"

namespace fsql {
namespace dev {

constexpr uint64_t kEps = 0xFFFFFFFFull;  // 2^64 mod p

// a, b in [0, p): a + b mod p.  On carry out of 64 bits the dropped 2^64 is
// worth kEps; a + b < 2p keeps the corrected sum below p.
__device__ __forceinline__ uint64_t gl_add(uint64_t a, uint64_t b) {
  const uint64_t s = a + b;
  if (s < a) return s + kEps;
  return s >= kP ? s - kP : s;
}

// a, b in [0, p): a - b mod p.  On borrow the wrapped value is 2^64 too big,
// i.e. kEps too big modulo p.
__device__ __forceinline__ uint64_t gl_sub(uint64_t a, uint64_t b) {
  const uint64_t d = a - b;
  return a < b ? d - kEps : d;
}

// a * b mod p for a, b < 2^64.  The 128-bit product is formed from four
// 32 x 32 -> 64-bit products (r3:r2:r1:r0 in 32-bit words) and reduced with
// 2^64 = 2^32 - 1 and 2^96 = -1 (mod p):
//   value = (r1:r0) + r2 * (2^32 - 1) - r3.
__device__ __forceinline__ uint64_t gl_mul(uint64_t a, uint64_t b) {
  const uint32_t a0 = static_cast<uint32_t>(a), a1 = static_cast<uint32_t>(a >> 32);
  const uint32_t b0 = static_cast<uint32_t>(b), b1 = static_cast<uint32_t>(b >> 32);
  const uint64_t p00 = static_cast<uint64_t>(a0) * b0;
  const uint64_t p01 = static_cast<uint64_t>(a0) * b1 + (p00 >> 32);
  const uint64_t p10 = static_cast<uint64_t>(a1) * b0 + static_cast<uint32_t>(p01);
  const uint64_t p11 = static_cast<uint64_t>(a1) * b1 + (p01 >> 32) + (p10 >> 32);
  const uint64_t lo = (p10 << 32) | static_cast<uint32_t>(p00);
  const uint64_t r2 = p11 & kEps, r3 = p11 >> 32;
  uint64_t t = lo - r3;
  if (lo < r3) t -= kEps;
  const uint64_t m = (r2 << 32) - r2;
  uint64_t r = t + m;
  if (r < m) r += kEps;
  return r >= kP ? r - kP : r;
}

// Signed integer v (|v| < p/2) as an element of Z_p.
__device__ __forceinline__ uint64_t gl_from_int(int32_t v) {
  return v < 0 ? kP - static_cast<uint64_t>(-static_cast<int64_t>(v)) : static_cast<uint64_t>(v);
}

// Centered lift of x in [0, p) to (-p/2, p/2), reduced mod 2^32.  Since
// p = 1 mod 2^32, x - p = x - 1 mod 2^32.
__device__ __forceinline__ uint32_t gl_lift32(uint64_t x) {
  return static_cast<uint32_t>(x) - (x > (kP >> 1) ? 1u : 0u);
}

__device__ __forceinline__ void named_sync(int id) {
  asm volatile("bar.sync %0, 128;\n" ::"r"(id) : "memory");
}

__device__ __forceinline__ int swz(int e) { return (e & ~15) | ((e ^ (e >> 3)) & 15); }

// element index held by thread t in register k, per layout
struct LF1 { static __device__ __forceinline__ int at(int t, int k) { return t + 128 * k; } };
struct LF2 { static __device__ __forceinline__ int at(int t, int k) { return 128 * (t >> 4) + 16 * k + (t & 15); } };
struct LF3 { static __device__ __forceinline__ int at(int t, int k) { return 16 * (t >> 1) + 2 * k + (t & 1); } };
struct LF4 { static __device__ __forceinline__ int at(int t, int k) { return 8 * t + k; } };
struct LI2 { static __device__ __forceinline__ int at(int t, int k) { return 64 * (t >> 3) + 8 * k + (t & 7); } };
struct LI3 { static __device__ __forceinline__ int at(int t, int k) { return 512 * (t >> 6) + 64 * k + (t & 63); } };

// Move the 1024 values from layout S to layout D through one of the group's
// two exchange buffers.  Consecutive exchanges alternate buffers, so the
// barrier of exchange j also guarantees that every thread has finished
// reading the buffer of exchange j-1 before exchange j+1 overwrites it.
template <class S, class D>
__device__ __forceinline__ void exchange(uint64_t (&x)[8], uint64_t* bufs, int& parity, int t, int bar) {
  uint64_t* buf = bufs + (parity << 10);
  parity ^= 1;
#pragma unroll
  for (int k = 0; k < 8; ++k) buf[swz(S::at(t, k))] = x[k];
  named_sync(bar);
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = buf[swz(D::at(t, k))];
}

// Cooley-Tukey butterfly on registers (k, k+d) with twiddle w.
__device__ __forceinline__ void ct(uint64_t& lo, uint64_t& hi, uint64_t w) {
  const uint64_t v = gl_mul(hi, w);
  const uint64_t u = lo;
  lo = gl_add(u, v);
  hi = gl_sub(u, v);
}
// Gentleman-Sande butterfly.
__device__ __forceinline__ void gs(uint64_t& lo, uint64_t& hi, uint64_t w) {
  const uint64_t u = lo, v = hi;
  lo = gl_add(u, v);
  hi = gl_mul(gl_sub(u, v), w);
}

// Forward transform: x in layout F1 -> layout F4.  bufs: this group's two
// 1024-u64 exchange buffers; parity: which one the next exchange uses.
__device__ __forceinline__ void ntt_forward(uint64_t (&x)[8], uint64_t* bufs, int& parity, const NttTables& T,
                                            int t, int bar) {
  // F1: distances 512, 256, 128 (register bits 2, 1, 0), twiddles uniform
#pragma unroll
  for (int k = 0; k < 4; ++k) ct(x[k], x[k + 4], T.f_small[1]);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & 2)) ct(x[k], x[k + 2], T.f_small[2 + (k >> 2)]);
#pragma unroll
  for (int k = 0; k < 8; k += 2) ct(x[k], x[k + 1], T.f_small[4 + (k >> 1)]);
  exchange<LF1, LF2>(x, bufs, parity, t, bar);
  // F2: distances 64, 32, 16
  const int h3 = t >> 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) ct(x[k], x[k + 4], T.f_small[8 + h3]);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & 2)) ct(x[k], x[k + 2], T.f_small[16 + 2 * h3 + (k >> 2)]);
#pragma unroll
  for (int k = 0; k < 8; k += 2) ct(x[k], x[k + 1], T.f_small[32 + 4 * h3 + (k >> 1)]);
  exchange<LF2, LF3>(x, bufs, parity, t, bar);
  // F3: distances 8, 4, 2 (per-thread twiddles)
#pragma unroll
  for (int k = 0; k < 4; ++k) ct(x[k], x[k + 4], T.f3[0][t]);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & 2)) ct(x[k], x[k + 2], T.f3[1 + (k >> 2)][t]);
#pragma unroll
  for (int k = 0; k < 8; k += 2) ct(x[k], x[k + 1], T.f3[3 + (k >> 1)][t]);
  exchange<LF3, LF4>(x, bufs, parity, t, bar);
  // F4: distance 1
#pragma unroll
  for (int k = 0; k < 8; k += 2) ct(x[k], x[k + 1], T.f4[k >> 1][t]);
}

// Inverse transform (no 1/N): x in layout F4 -> layout F1 (natural order).
__device__ __forceinline__ void ntt_inverse(uint64_t (&x)[8], uint64_t* bufs, int& parity, const NttTables& T,
                                            int t, int bar) {
  // I1: distances 1, 2, 4 (per-thread twiddles)
#pragma unroll
  for (int k = 0; k < 8; k += 2) gs(x[k], x[k + 1], T.i1[k >> 1][t]);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & 2)) gs(x[k], x[k + 2], T.i1[4 + (k >> 2)][t]);
#pragma unroll
  for (int k = 0; k < 4; ++k) gs(x[k], x[k + 4], T.i1[6][t]);
  exchange<LF4, LI2>(x, bufs, parity, t, bar);
  // I2: distances 8, 16, 32
  const int h4 = t >> 3;
#pragma unroll
  for (int k = 0; k < 8; k += 2) gs(x[k], x[k + 1], T.g_small[64 + 4 * h4 + (k >> 1)]);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & 2)) gs(x[k], x[k + 2], T.g_small[32 + 2 * h4 + (k >> 2)]);
#pragma unroll
  for (int k = 0; k < 4; ++k) gs(x[k], x[k + 4], T.g_small[16 + h4]);
  exchange<LI2, LI3>(x, bufs, parity, t, bar);
  // I3: distances 64, 128, 256
  const int b9 = t >> 6;
#pragma unroll
  for (int k = 0; k < 8; k += 2) gs(x[k], x[k + 1], T.g_small[8 + 4 * b9 + (k >> 1)]);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & 2)) gs(x[k], x[k + 2], T.g_small[4 + 2 * b9 + (k >> 2)]);
#pragma unroll
  for (int k = 0; k < 4; ++k) gs(x[k], x[k + 4], T.g_small[2 + b9]);
  exchange<LI3, LF1>(x, bufs, parity, t, bar);
  // I4: distance 512
#pragma unroll
  for (int k = 0; k < 4; ++k) gs(x[k], x[k + 4], T.g_small[1]);
}

}  // namespace dev
}  // namespace fsql
