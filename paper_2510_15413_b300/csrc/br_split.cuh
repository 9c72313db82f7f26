// br_split.cuh -- blind rotation of the two-prime engine with the two primes
// on separate warps ("prime-split").
//
// The two-prime engine computes every external product exactly by CRT from
// two 1024-point negacyclic NTTs mod p1 and mod p2 (ntt.cuh).  In
// blind_rotate_kernel one 128-thread group holds both residues of 8
// coefficients per thread (packed in 64 bits), so each thread carries two
// transforms' worth of registers (158 per thread for 3 gates per CTA, 12
// warps per SM).  Here a gate is 256 threads: half 0 (warps 0-3 of the gate)
// runs every transform mod p1, half 1 mod p2, each on 32-bit residues, with
// the half's own exchange buffers and twiddle table.  Per thread the
// registers of one transform suffice, so more gates (warps) are resident and
// the dependency chains of the butterflies are hidden by other warps.
//
// Per CMux i, for each step of P gadget rows (both halves):
//   - digits of X^a ACC_u - ACC_u (from the shared ACC) for the step's rows,
//     lifted to [0, 2p) of the half's prime;
//   - forward NTT of the P digit polynomials (lazy Shoup butterflies);
//   - multiply-accumulate with the half's words of the staged key rows into
//     64-bit sums (two output polynomials per slot).
// After the last step: one Montgomery reduction per sum, the inverse NTT of
// the two output polynomials, then the CRT: half h lifts output polynomial h
// and needs the other prime's residues of it, exchanged through a small
// shared buffer (one 256-thread named barrier), and adds the exact integer
// mod 2^32 into ACC.  Same arithmetic as the packed kernel (same reductions,
// same bounds), so the output words are the same.
//
// Key layout (bks): [i][row][prime][k][t][c] u32, slot 8t + k of the forward
// transform of BK[i][row][c] scaled like the packed key; a row is 16 KB and
// the P rows of a step are contiguous.  Twiddles: one NttTablesT<uint2>
// ({w, floor(w 2^32 / p)}) per prime.
#pragma once

#include <cstdint>

#include "engine.h"
#include "ntt.cuh"

namespace fsql {
namespace dev {

using SplitTables = NttTablesT<uint2>;

// Bank swizzle for 32-bit elements of a 1024-element polynomial: the low
// five address bits are XORed with a fixed linear function of bits 5-7
// (bit 5 -> bit 1, bit 6 -> bits 2, 3, bit 7 -> bits 0, 3, 4).  For every
// thread layout of ntt.cuh (F1..F4, I2, I3) the 32 lanes of a warp then hit
// 32 distinct banks for every register index, and the map keeps each
// 256-element block (a warp's region in the warp-local layouts) in place.
__device__ __forceinline__ int swz32(int e) {
  const int b = e >> 5;
  return e ^ (((b & 1) << 1) ^ (((b >> 1) & 1) * 12) ^ (((b >> 2) & 1) * 25));
}

// Lazy forward butterfly on residues below 22p (inputs), outputs grow by
// less than 2p (the packed engine's ct1 with a runtime prime).
__device__ __forceinline__ void ct32(uint32_t& lo, uint32_t& hi, uint2 w, uint32_t p, uint32_t p2) {
  const uint32_t q = __umulhi(hi, w.y);
  const uint32_t t = hi * w.x - q * p;
  hi = lo - t + p2;
  lo = lo + t;
}
// Inverse (Gentleman-Sande) butterfly, residues in [0, 2p) in and out.
__device__ __forceinline__ void gs32(uint32_t& lo, uint32_t& hi, uint2 w, uint32_t p, uint32_t p2) {
  const uint32_t y = hi;
  const uint32_t d = lo - y + p2;
  hi = d * w.x - __umulhi(d, w.y) * p;
  lo = fold(lo + y, p2);
}

template <int P, int B, int NB, class S, class D, bool kWarpLocal>
__device__ __forceinline__ void xch32(uint32_t (&x)[P][8], uint32_t* bufs, int& parity, int t, int bar) {
  static_assert(P <= B, "exchange buffer too small");
  uint32_t* buf = bufs + (NB == 2 ? parity : 0) * (B * 1024);
  parity ^= 1;
  if (NB == 1) __syncwarp();
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int k = 0; k < 8; ++k) buf[p * 1024 + swz32(S::at(t, k))] = x[p][k];
  if (kWarpLocal) __syncwarp();
  else named_sync(bar);
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[p][k] = buf[p * 1024 + swz32(D::at(t, k))];
}

template <int P, int D, class TwOf>
__device__ __forceinline__ void ct32_stage(uint32_t (&x)[P][8], TwOf tw, uint32_t p, uint32_t p2) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & D) continue;
    const uint2 w = tw(k);
#pragma unroll
    for (int q = 0; q < P; ++q) ct32(x[q][k], x[q][k + D], w, p, p2);
  }
}
template <int P, int D, class TwOf>
__device__ __forceinline__ void gs32_stage(uint32_t (&x)[P][8], TwOf tw, uint32_t p, uint32_t p2) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & D) continue;
    const uint2 w = tw(k);
#pragma unroll
    for (int q = 0; q < P; ++q) gs32(x[q][k], x[q][k + D], w, p, p2);
  }
}

// First two forward stages of a digit polynomial by table lookup, one prime
// (the 32-bit form of digit_stages12 in ntt.cuh): tab[m][u] = (u - half) m
// mod p, canonical, for m = w1, w2a, w2a w1, w2b, w2b w1.
__device__ __forceinline__ void digit_stages12_32(const uint32_t (&u)[8], uint32_t (&z)[8], uint32_t half,
                                                  const uint32_t* __restrict__ tab, uint32_t p, uint32_t p2) {
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const uint32_t d0 = u[a] + p - half;
    const uint32_t A = tab[0 * kDigitTabSize + u[a + 4]];
    const uint32_t Bv = tab[1 * kDigitTabSize + u[a + 2]];
    const uint32_t C = tab[2 * kDigitTabSize + u[a + 6]];
    const uint32_t D = tab[3 * kDigitTabSize + u[a + 2]];
    const uint32_t E = tab[4 * kDigitTabSize + u[a + 6]];
    z[a] = d0 + A + Bv + C;
    z[a + 2] = d0 + A + p2 - Bv - C;
    z[a + 4] = d0 + p2 - A + D - E + p2;
    z[a + 6] = d0 + p2 - A - D + E + p2;
  }
}
// The tables of digit_stages12_32 for prime p from its twiddle table.
__device__ __forceinline__ void build_digit_tables32(uint32_t* tab, const SplitTables& T, uint32_t half, uint32_t p,
                                                     int tid, int nthreads) {
  for (int e = tid; e < kDigitTabs * kDigitTabSize; e += nthreads) {
    const int m = e / kDigitTabSize, u = e % kDigitTabSize;
    const uint64_t w1 = T.f_small[1].x, w2a = T.f_small[2].x, w2b = T.f_small[3].x;
    const uint64_t mult = m == 0 ? w1 : m == 1 ? w2a : m == 2 ? w2a * w1 % p : m == 3 ? w2b : w2b * w1 % p;
    const uint64_t d = (static_cast<uint64_t>(u) + p - half) % p;
    tab[e] = static_cast<uint32_t>(d * mult % p);
  }
}

// Forward transform of P polynomials mod p (layout F1 -> F4), the passes of
// ntt_forward on 32-bit residues.  kFrom3: the first two stages were done by
// digit_stages12_32.
template <int P, int B, int NB, bool kFrom3 = false>
__device__ __forceinline__ void ntt_forward32(uint32_t (&x)[P][8], uint32_t* bufs, int& parity, const SplitTables& T,
                                              int t, int bar, uint32_t p, uint32_t p2) {
  if (!kFrom3) {
    ct32_stage<P, 4>(x, [&](int) { return T.f_small[1]; }, p, p2);
    ct32_stage<P, 2>(x, [&](int k) { return T.f_small[2 + (k >> 2)]; }, p, p2);
  }
  ct32_stage<P, 1>(x, [&](int k) { return T.f_small[4 + (k >> 1)]; }, p, p2);
  xch32<P, B, NB, LF1, LF2, false>(x, bufs, parity, t, bar);
  const int h3 = t >> 4;
  ct32_stage<P, 4>(x, [&](int) { return T.f_small[8 + h3]; }, p, p2);
  ct32_stage<P, 2>(x, [&](int k) { return T.f_small[16 + 2 * h3 + (k >> 2)]; }, p, p2);
  ct32_stage<P, 1>(x, [&](int k) { return T.f_small[32 + 4 * h3 + (k >> 1)]; }, p, p2);
  xch32<P, B, NB, LF2, LF3, true>(x, bufs, parity, t, bar);
  ct32_stage<P, 4>(x, [&](int) { return T.f3[0][t]; }, p, p2);
  ct32_stage<P, 2>(x, [&](int k) { return T.f3[1 + (k >> 2)][t]; }, p, p2);
  ct32_stage<P, 1>(x, [&](int k) { return T.f3[3 + (k >> 1)][t]; }, p, p2);
  xch32<P, B, NB, LF3, LF4, true>(x, bufs, parity, t, bar);
  ct32_stage<P, 1>(x, [&](int k) { return T.f4[k >> 1][t]; }, p, p2);
}

// Inverse transform of P polynomials mod p (no 1/N): layout F4 -> F1.
template <int P, int B, int NB>
__device__ __forceinline__ void ntt_inverse32(uint32_t (&x)[P][8], uint32_t* bufs, int& parity, const SplitTables& T,
                                              int t, int bar, uint32_t p, uint32_t p2) {
  gs32_stage<P, 1>(x, [&](int k) { return T.i1[k >> 1][t]; }, p, p2);
  gs32_stage<P, 2>(x, [&](int k) { return T.i1[4 + (k >> 2)][t]; }, p, p2);
  gs32_stage<P, 4>(x, [&](int) { return T.i1[6][t]; }, p, p2);
  xch32<P, B, NB, LF4, LI2, true>(x, bufs, parity, t, bar);
  const int h4 = t >> 3;
  gs32_stage<P, 1>(x, [&](int k) { return T.g_small[64 + 4 * h4 + (k >> 1)]; }, p, p2);
  gs32_stage<P, 2>(x, [&](int k) { return T.g_small[32 + 2 * h4 + (k >> 2)]; }, p, p2);
  gs32_stage<P, 4>(x, [&](int) { return T.g_small[16 + h4]; }, p, p2);
  xch32<P, B, NB, LI2, LI3, false>(x, bufs, parity, t, bar);
  const int b9 = t >> 6;
  gs32_stage<P, 1>(x, [&](int k) { return T.g_small[8 + 4 * b9 + (k >> 1)]; }, p, p2);
  gs32_stage<P, 2>(x, [&](int k) { return T.g_small[4 + 2 * b9 + (k >> 2)]; }, p, p2);
  gs32_stage<P, 4>(x, [&](int) { return T.g_small[2 + b9]; }, p, p2);
  if (NB == 1) named_sync(bar);  // every thread's I2 -> I3 reads are over (spread write next)
  xch32<P, B, NB, LI3, LF1, false>(x, bufs, parity, t, bar);
  gs32_stage<P, 4>(x, [&](int) { return T.g_small[1]; }, p, p2);
}

__device__ __forceinline__ void named_sync_n(int id, int threads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(threads) : "memory");
}

// residues x1 (mod p1) and x2 (mod p2), each in [0, 2p) -> the integer in
// (-p1 p2 / 2, p1 p2 / 2) they represent, mod 2^32 (DualPrime::to_torus on
// separate words)
__device__ __forceinline__ uint32_t crt_torus(uint32_t x1, uint32_t x2) {
  return DualPrime::to_torus(pack(x1, x2));
}

}  // namespace dev
}  // namespace fsql
