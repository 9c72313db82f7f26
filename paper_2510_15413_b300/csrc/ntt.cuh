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

// ---------------------------------------------------------------------------
// Engine 1: one 64-bit prime, p = 2^64 - 2^32 + 1 (Goldilocks).  Elements are
// canonical in [0, p).
// ---------------------------------------------------------------------------
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

struct Goldilocks {
  static constexpr int kEngine = FSQL_ENGINE_GOLDILOCKS;
  using Tw = uint64_t;
  using Tables = NttTablesT<Tw>;
  // signed integer v (|v| < p/2)
  static __device__ __forceinline__ uint64_t from_int(int32_t v) {
    return v < 0 ? kP - static_cast<uint64_t>(-static_cast<int64_t>(v)) : static_cast<uint64_t>(v);
  }
  static __device__ __forceinline__ uint64_t from_digit(uint32_t u, uint32_t half) {
    return from_int(static_cast<int32_t>(u) - static_cast<int32_t>(half));
  }
  static __device__ __forceinline__ uint64_t from_u32(uint32_t v) { return v; }
  static __device__ __forceinline__ void ct(uint64_t& lo, uint64_t& hi, uint64_t w) {
    const uint64_t v = gl_mul(hi, w);
    const uint64_t u = lo;
    lo = gl_add(u, v);
    hi = gl_sub(u, v);
  }
  static __device__ __forceinline__ void gs(uint64_t& lo, uint64_t& hi, uint64_t w) {
    const uint64_t u = lo, v = hi;
    lo = gl_add(u, v);
    hi = gl_mul(gl_sub(u, v), w);
  }
  // key conversion: canonical x times the stored constant (1/N)
  static __device__ __forceinline__ uint64_t scale_key(uint64_t x, uint64_t k) { return gl_mul(x, k); }
  // multiply-accumulate of one gadget row into the two output polynomials
  struct Acc {
    uint64_t c0, c1;
  };
  static __device__ __forceinline__ void mac(Acc& a, uint64_t x, ulonglong2 w, bool first) {
    const uint64_t p0 = gl_mul(x, w.x), p1 = gl_mul(x, w.y);
    a.c0 = first ? p0 : gl_add(a.c0, p0);
    a.c1 = first ? p1 : gl_add(a.c1, p1);
  }
  static __device__ __forceinline__ uint64_t acc0(const Acc& a) { return a.c0; }
  static __device__ __forceinline__ uint64_t acc1(const Acc& a) { return a.c1; }
  // centered lift to (-p/2, p/2), reduced mod 2^32 (p = 1 mod 2^32, so x - p = x - 1 there)
  static __device__ __forceinline__ uint32_t to_torus(uint64_t x) {
    return static_cast<uint32_t>(x) - (x > (kP >> 1) ? 1u : 0u);
  }
};

// ---------------------------------------------------------------------------
// Engine 2: two primes p1, p2 < 2^32/24 with 2048 | p - 1, the integer
// result recovered by CRT (p1 p2 ~ 2^54.8 > 2^52.6).  An element packs the
// two residues (low word mod p1, high word mod p2).  Residues are kept lazily
// (not reduced below p) in the manner of Harvey ("Faster arithmetic for
// number-theoretic transforms", 2014), with bounds chosen for these primes:
//   forward: no reduction at all; a butterfly adds at most 2p to the bound,
//     so from digits below 2p the 10 stages stay below 22p < 2^32;
//   multiply-accumulate: six products of forward outputs (below 22p) and
//     canonical key values summed in 64 bits (below 132 p^2), reduced once;
//   inverse: residues in [0, 2p), one fold per butterfly.
// Products by a twiddle w use Shoup's precomputed quotient
// w' = floor(w 2^32 / p): q = hi(a w'), r = a w - q p in [0, 2p) for any
// a < 2^32 (three integer multiply-adds, no compare).  Sums of products and
// the CRT use signed Montgomery reduction with R = 2^32 (Seiler, 2018):
// m = (T mod R) p^-1 mod R, r = hi(T) - hi(m p) + p in (0, 2p) for T < p R.
// ---------------------------------------------------------------------------
constexpr uint32_t kP1 = 178956289u, kP2 = 178948097u;         // 87381 * 2^11 + 1, 87377 * 2^11 + 1
constexpr uint32_t kP1inv = 2207602689u, kP2inv = 3717560321u;  // p^-1 mod 2^32
constexpr uint32_t kCrtC = 524288u;                             // (p1^-1 mod p2) * R mod p2
constexpr uint64_t kCrtM = static_cast<uint64_t>(kP1) * kP2;
static_assert(22ull * kP1 < (1ull << 32) && 22ull * kP2 < (1ull << 32), "forward bound 22 p < 2^32");
static_assert(24ull * kP1 <= (1ull << 32) && 24ull * kP2 <= (1ull << 32), "multiply-accumulate bound 24 p < 2^32");

__device__ __forceinline__ uint32_t mont(uint32_t a, uint32_t w, uint32_t p, uint32_t pinv) {
  const uint32_t lo = a * w;
  const uint32_t hi = __umulhi(a, w);
  return hi - __umulhi(lo * pinv, p) + p;
}
// 64-bit T reduced to T R^-1 mod p: hi(T) - hi(m p) + p, in (0, hi(T) + p]
// (in (0, 2p) when T < p R)
__device__ __forceinline__ uint32_t mont64(uint64_t T, uint32_t p, uint32_t pinv) {
  const uint32_t lo = static_cast<uint32_t>(T), hi = static_cast<uint32_t>(T >> 32);
  return hi - __umulhi(lo * pinv, p) + p;
}
__device__ __forceinline__ uint32_t lo32(uint64_t x) { return static_cast<uint32_t>(x); }
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return static_cast<uint32_t>(x >> 32); }
__device__ __forceinline__ uint64_t pack(uint32_t a, uint32_t b) { return (static_cast<uint64_t>(b) << 32) | a; }
// x in [0, 2m) -> [0, m): unsigned min with the wrapped difference
__device__ __forceinline__ uint32_t fold(uint32_t x, uint32_t m) { return min(x, x - m); }

__device__ __forceinline__ uint32_t shoup(uint32_t a, uint32_t w, uint32_t ws, uint32_t p) {
  const uint32_t q = __umulhi(a, ws);
  return a * w - q * p;
}

struct DualPrime {
  static constexpr int kEngine = FSQL_ENGINE_DUAL_PRIME;
  using Tw = uint4;  // {w mod p1, w' for p1, w mod p2, w' for p2}
  using Tables = NttTablesT<Tw>;
  static __device__ __forceinline__ uint64_t from_int(int32_t v) {
    return v < 0 ? pack(kP1 + v, kP2 + v) : pack(v, v);
  }
  // digit u - half (u in [0, 2^bg)) as u + p - half, below 2p
  static __device__ __forceinline__ uint64_t from_digit(uint32_t u, uint32_t half) {
    return pack(u + (kP1 - half), u + (kP2 - half));
  }
  static __device__ __forceinline__ uint64_t from_u32(uint32_t v) { return pack(v % kP1, v % kP2); }
  // forward butterfly, no reduction: both outputs grow by less than 2p
  static __device__ __forceinline__ uint32_t ct1(uint32_t x, uint32_t& hi, uint32_t w, uint32_t ws, uint32_t p) {
    const uint32_t t = shoup(hi, w, ws, p);
    hi = x - t + 2 * p;
    return x + t;
  }
  static __device__ __forceinline__ void ct(uint64_t& lo, uint64_t& hi, const uint4& w) {
    uint32_t h1 = lo32(hi), h2 = hi32(hi);
    const uint32_t l1 = ct1(lo32(lo), h1, w.x, w.y, kP1);
    const uint32_t l2 = ct1(hi32(lo), h2, w.z, w.w, kP2);
    lo = pack(l1, l2);
    hi = pack(h1, h2);
  }
  // residues in [0, 2p) in and out
  static __device__ __forceinline__ uint32_t gs1(uint32_t x, uint32_t& hi, uint32_t w, uint32_t ws, uint32_t p) {
    const uint32_t y = hi;
    hi = shoup(x - y + 2 * p, w, ws, p);
    return fold(x + y, 2 * p);
  }
  static __device__ __forceinline__ void gs(uint64_t& lo, uint64_t& hi, const uint4& w) {
    uint32_t h1 = lo32(hi), h2 = hi32(hi);
    const uint32_t l1 = gs1(lo32(lo), h1, w.x, w.y, kP1);
    const uint32_t l2 = gs1(hi32(lo), h2, w.z, w.w, kP2);
    lo = pack(l1, l2);
    hi = pack(h1, h2);
  }
  // key conversion: forward output (below 22p) times k = N^-1 R^2, canonical
  static __device__ __forceinline__ uint64_t scale_key(uint64_t x, uint64_t k) {
    const uint32_t a = fold(mont(lo32(x), lo32(k), kP1, kP1inv), kP1);
    const uint32_t b = fold(mont(hi32(x), hi32(k), kP2, kP2inv), kP2);
    return pack(a, b);
  }
  // Multiply-accumulate: 64-bit sums of six products x w (x a forward
  // output below 22p, w a canonical key value in Montgomery form), so
  // T < 132 p^2 < 2^64.  Signed Montgomery reduction of any 64-bit T gives
  // hi(T) - hi(m p) in (-p, hi(T)], here (-p, 5.5p); adding p and two folds
  // bring it into [0, 2p), the input range of the inverse transform.
  struct Acc {
    uint64_t s10, s20, s11, s21;  // (prime, output polynomial)
  };
  static __device__ __forceinline__ void mac(Acc& a, uint64_t x, ulonglong2 w, bool first) {
    const uint32_t x1 = lo32(x), x2 = hi32(x);
    a.s10 = static_cast<uint64_t>(x1) * lo32(w.x) + (first ? 0ull : a.s10);
    a.s20 = static_cast<uint64_t>(x2) * hi32(w.x) + (first ? 0ull : a.s20);
    a.s11 = static_cast<uint64_t>(x1) * lo32(w.y) + (first ? 0ull : a.s11);
    a.s21 = static_cast<uint64_t>(x2) * hi32(w.y) + (first ? 0ull : a.s21);
  }
  static __device__ __forceinline__ uint32_t settle(uint64_t T, uint32_t p, uint32_t pinv) {
    return fold(fold(mont64(T, p, pinv), 4 * p), 2 * p);
  }
  static __device__ __forceinline__ uint64_t acc0(const Acc& a) {
    return pack(settle(a.s10, kP1, kP1inv), settle(a.s20, kP2, kP2inv));
  }
  static __device__ __forceinline__ uint64_t acc1(const Acc& a) {
    return pack(settle(a.s11, kP1, kP1inv), settle(a.s21, kP2, kP2inv));
  }
  // residues in [0, 2p) -> the integer V in (-M/2, M/2) by CRT
  // (V = x1 + p1 ((x2 - x1) p1^-1 mod p2)), reduced mod 2^32
  static __device__ __forceinline__ uint32_t to_torus(uint64_t x) {
    const uint32_t x1 = fold(lo32(x), kP1), x2 = fold(hi32(x), kP2);
    const uint32_t h = fold(mont(x2 + 2 * kP2 - x1, kCrtC, kP2, kP2inv), kP2);
    const uint64_t v = static_cast<uint64_t>(kP1) * h + x1;
    return static_cast<uint32_t>(v) - (v > (kCrtM >> 1) ? static_cast<uint32_t>(kCrtM) : 0u);
  }
};

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

// Move the P x 1024 values of P polynomials from layout S to layout D
// through the group's exchange buffers: NB = 2 buffers used alternately, or
// NB = 1 buffer (less shared memory, one more barrier per inverse).  Each
// buffer holds B >= P polynomials (B is the same for every exchange of a
// kernel, so two buffers never overlap).
//
// Warp-local exchanges.  In layouts F2, F3, F4 (= I1) and I2 the 32 threads
// of warp w hold exactly the elements [256 w, 256 w + 256); F1 and I3 spread
// a warp over the whole polynomial.  An exchange whose source and
// destination are both warp-local (F2->F3, F3->F4, F4->I2) only moves data
// inside each warp and synchronises the warp alone; the others (F1->F2,
// I2->I3, I3->F1) use the group's named barrier.  Reuse of a buffer is safe:
// a warp-local exchange writes only its warp's region, which no other warp
// reads in the previous exchange on that buffer (its destination was warp
// local, or a named barrier came in between); a spread exchange is always
// preceded by a group-wide barrier since the last reads of its buffer (the
// CTA barrier at the start of each step, or the named barrier of I2->I3).
template <int P, int B, int NB, class S, class D, bool kWarpLocal>
__device__ __forceinline__ void exchange(uint64_t (&x)[P][8], uint64_t* bufs, int& parity, int t, int bar) {
  static_assert(P <= B, "exchange buffer too small");
  uint64_t* buf = bufs + (NB == 2 ? parity : 0) * (B * 1024);
  parity ^= 1;
  // with one buffer, the previous exchange's reads must be over before these
  // writes: within the warp for warp-local writes; a spread write follows a
  // spread read only in the inverse (I3 -> F1), whose caller adds the barrier
  if (NB == 1) __syncwarp();
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int k = 0; k < 8; ++k) buf[p * 1024 + swz(S::at(t, k))] = x[p][k];
  if (kWarpLocal) __syncwarp();
  else named_sync(bar);
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[p][k] = buf[p * 1024 + swz(D::at(t, k))];
}

// One radix-2 stage on registers (k, k + d) of P polynomials, twiddle by
// the lower register index.
template <class F, int P, int D, class TwOf>
__device__ __forceinline__ void ct_stage(uint64_t (&x)[P][8], TwOf tw) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & D) continue;
    const typename F::Tw w = tw(k);
#pragma unroll
    for (int p = 0; p < P; ++p) F::ct(x[p][k], x[p][k + D], w);
  }
}
template <class F, int P, int D, class TwOf>
__device__ __forceinline__ void gs_stage(uint64_t (&x)[P][8], TwOf tw) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & D) continue;
    const typename F::Tw w = tw(k);
#pragma unroll
    for (int p = 0; p < P; ++p) F::gs(x[p][k], x[p][k + D], w);
  }
}

// First two forward stages of a digit polynomial by table lookup (two-prime
// engine).  A thread's registers 0..7 hold elements t + 128k; stages 1 and 2
// (distances 512 and 256, twiddles w1 = f[1], w2a = f[2] for registers 0-3,
// w2b = f[3] for 4-7) combine the four digits d0..d3 of registers
// (a, a+2, a+4, a+6), a = 0, 1, into
//   z_a   = d0 + w1 d2 + w2a d1 + w2a w1 d3     z_a+2 = d0 + w1 d2 - w2a d1 - w2a w1 d3
//   z_a+4 = d0 - w1 d2 + w2b d1 - w2b w1 d3     z_a+6 = d0 - w1 d2 - w2b d1 + w2b w1 d3
// (mod each prime).  A digit takes 2^bg <= 128 values, so each product is
// read from a table of (u - 2^(bg-1)) m mod p for the five multipliers m
// (tab[m][u], both residues packed, canonical), built once per CTA by
// build_digit_tables: five lookups and adds replace eight Shoup products per
// group.  Outputs stay below 6p, the bound the lazy transform has after two
// stages from digits below 2p, so the remaining stages are unchanged.
constexpr int kDigitTabs = 5;
constexpr int kDigitTabSize = 128;
__device__ __forceinline__ void digit_stages12(const uint32_t (&u)[8], uint64_t (&z)[8], uint32_t half,
                                               const uint64_t* __restrict__ tab) {
  const uint64_t off2 = pack(2 * kP1, 2 * kP2);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const uint64_t d0 = DualPrime::from_digit(u[a], half);
    const uint64_t A = tab[0 * kDigitTabSize + u[a + 4]];
    const uint64_t Bv = tab[1 * kDigitTabSize + u[a + 2]];
    const uint64_t C = tab[2 * kDigitTabSize + u[a + 6]];
    const uint64_t D = tab[3 * kDigitTabSize + u[a + 2]];
    const uint64_t E = tab[4 * kDigitTabSize + u[a + 6]];
    // every lane stays in [0, 2^32): the packed 64-bit sums carry nothing across lanes
    z[a] = d0 + A + Bv + C;
    z[a + 2] = d0 + A + off2 - Bv - C;
    z[a + 4] = d0 + off2 - A + D - E + off2;
    z[a + 6] = d0 + off2 - A - D + E + off2;
  }
}
// tab[m][u] = (u - half) * m mod p for m = w1, w2a, w2a w1, w2b, w2b w1
// (the residues of the stage twiddles f[1], f[2], f[3]), both primes packed.
template <class Tab>
__device__ __forceinline__ void build_digit_tables(uint64_t* tab, const Tab& T, uint32_t half, int tid,
                                                   int nthreads) {
  for (int e = tid; e < kDigitTabs * kDigitTabSize; e += nthreads) {
    const int m = e / kDigitTabSize, u = e % kDigitTabSize;
    uint32_t r[2];
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      const uint64_t p = pr ? kP2 : kP1;
      const uint64_t w1 = pr ? T.f_small[1].z : T.f_small[1].x;
      const uint64_t w2a = pr ? T.f_small[2].z : T.f_small[2].x;
      const uint64_t w2b = pr ? T.f_small[3].z : T.f_small[3].x;
      const uint64_t mult = m == 0 ? w1 : m == 1 ? w2a : m == 2 ? w2a * w1 % p : m == 3 ? w2b : w2b * w1 % p;
      const uint64_t d = (static_cast<uint64_t>(u) + p - half) % p;
      r[pr] = static_cast<uint32_t>(d * mult % p);
    }
    tab[e] = pack(r[0], r[1]);
  }
}

// Forward transform of P polynomials: layout F1 -> layout F4.  bufs: this
// group's two exchange buffers of B polynomials each; parity: which one the
// next exchange uses.  Its first exchange writes across warps, so the caller
// separates it from the exchanges of an earlier transform by a group-wide
// barrier.  kFrom3: the first two stages were done already (digit_stages12).
template <class F, int P, int B, int NB = 2, bool kFrom3 = false>
__device__ __forceinline__ void ntt_forward(uint64_t (&x)[P][8], uint64_t* bufs, int& parity,
                                            const typename F::Tables& T, int t, int bar) {
  // F1: distances 512, 256, 128 (register bits 2, 1, 0), twiddles uniform
  if (!kFrom3) {
    ct_stage<F, P, 4>(x, [&](int) { return T.f_small[1]; });
    ct_stage<F, P, 2>(x, [&](int k) { return T.f_small[2 + (k >> 2)]; });
  }
  ct_stage<F, P, 1>(x, [&](int k) { return T.f_small[4 + (k >> 1)]; });
  exchange<P, B, NB, LF1, LF2, false>(x, bufs, parity, t, bar);
  // F2: distances 64, 32, 16
  const int h3 = t >> 4;
  ct_stage<F, P, 4>(x, [&](int) { return T.f_small[8 + h3]; });
  ct_stage<F, P, 2>(x, [&](int k) { return T.f_small[16 + 2 * h3 + (k >> 2)]; });
  ct_stage<F, P, 1>(x, [&](int k) { return T.f_small[32 + 4 * h3 + (k >> 1)]; });
  exchange<P, B, NB, LF2, LF3, true>(x, bufs, parity, t, bar);
  // F3: distances 8, 4, 2 (per-thread twiddles)
  ct_stage<F, P, 4>(x, [&](int) { return T.f3[0][t]; });
  ct_stage<F, P, 2>(x, [&](int k) { return T.f3[1 + (k >> 2)][t]; });
  ct_stage<F, P, 1>(x, [&](int k) { return T.f3[3 + (k >> 1)][t]; });
  exchange<P, B, NB, LF3, LF4, true>(x, bufs, parity, t, bar);
  // F4: distance 1
  ct_stage<F, P, 1>(x, [&](int k) { return T.f4[k >> 1][t]; });
}

// Inverse transform of P polynomials (no 1/N): layout F4 -> layout F1 (natural order).
template <class F, int P, int B, int NB = 2>
__device__ __forceinline__ void ntt_inverse(uint64_t (&x)[P][8], uint64_t* bufs, int& parity,
                                            const typename F::Tables& T, int t, int bar) {
  // I1: distances 1, 2, 4 (per-thread twiddles)
  gs_stage<F, P, 1>(x, [&](int k) { return T.i1[k >> 1][t]; });
  gs_stage<F, P, 2>(x, [&](int k) { return T.i1[4 + (k >> 2)][t]; });
  gs_stage<F, P, 4>(x, [&](int) { return T.i1[6][t]; });
  exchange<P, B, NB, LF4, LI2, true>(x, bufs, parity, t, bar);
  // I2: distances 8, 16, 32
  const int h4 = t >> 3;
  gs_stage<F, P, 1>(x, [&](int k) { return T.g_small[64 + 4 * h4 + (k >> 1)]; });
  gs_stage<F, P, 2>(x, [&](int k) { return T.g_small[32 + 2 * h4 + (k >> 2)]; });
  gs_stage<F, P, 4>(x, [&](int) { return T.g_small[16 + h4]; });
  exchange<P, B, NB, LI2, LI3, false>(x, bufs, parity, t, bar);
  // I3: distances 64, 128, 256
  const int b9 = t >> 6;
  gs_stage<F, P, 1>(x, [&](int k) { return T.g_small[8 + 4 * b9 + (k >> 1)]; });
  gs_stage<F, P, 2>(x, [&](int k) { return T.g_small[4 + 2 * b9 + (k >> 2)]; });
  gs_stage<F, P, 4>(x, [&](int) { return T.g_small[2 + b9]; });
  if (NB == 1) named_sync(bar);  // every thread's I2 -> I3 reads are over (spread write next)
  exchange<P, B, NB, LI3, LF1, false>(x, bufs, parity, t, bar);
  // I4: distance 512
  gs_stage<F, P, 4>(x, [&](int) { return T.g_small[1]; });
}

}  // namespace dev
}  // namespace fsql
