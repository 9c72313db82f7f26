// kernels.cu -- device half of the library: the gate-bootstrap engine
// (linear combination, modulus switch, blind rotation, sample extraction,
// keyswitch) and the scan driver that runs the predicate circuit level by
// level over all rows (Alg. 2 ProcessQuery; §4.2 mask generation and
// application).
//
// Blind rotation kernel.  A group of 128 threads owns one gate for all n CMux
// steps; each thread holds 8 of the 1024 coefficients of every polynomial it
// transforms (ntt.cuh).  A CTA runs G gates.  The bootstrapping-key slice
// of each step (P gadget rows, 16 KB each in the NTT domain) is staged into
// shared memory by cp.async either once per CTA into a 2-slot ring read by
// all G groups in lockstep, or (the own-slot form, the default shape) by
// each group into a slot of its own, so the groups synchronise only
// themselves and drift apart (one group's exchanges overlap another's
// butterflies); each group then reads the key from L2.  Key copies carry an
// L2 evict-last hint, gate inputs and extracted outputs the streaming hint,
// so the key stays in L2 while gate I/O streams through.  Per CMux a group:
//   for each of the 2l = 6 rows (u, j), P rows per step: forms digit j of
//     X^a*ACC_u - ACC_u, runs the forward NTT, and multiply-accumulates with
//     the staged key row into two NTT-domain accumulators (one per output
//     polynomial) held in registers;
//   runs the two inverse NTTs, lifts the exact integers mod 2^32 and adds
//   them into its accumulator polynomials in shared memory.
// Keyswitch kernel.  A CTA takes 16 gates and one tile of 128 output
// columns; each thread owns one column of the tile, walks the (i, j) digit
// positions once and reads the three nonzero-digit key words of its column,
// so each key row read from L2 serves 16 gates.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "br_split.cuh"
#include "engine.h"
#include "ntt.cuh"

namespace fsql {

namespace {

constexpr int kGroup = 128;                      // threads per gate
constexpr int kChunkU64 = 8 * kGroup * 2;        // one key row: 1024 slots x 2 output polys
constexpr int kStages = 2;                       // cp.async ring of steps
constexpr int kGateAcc = 2 * kN * 4;             // accumulator polynomials (u32)
constexpr int kGateAbar = kMaxN * 2;             // switched mask, u16
// Polynomials per exchange buffer of the blind rotation: a step transforms
// P gadget rows at once, the inverse transforms the two output polynomials.
template <int P>
__host__ __device__ constexpr int xbuf_polys() {
  return P > 2 ? P : 2;
}
// Per gate: NB exchange buffers, the accumulator, the switched mask.
template <int P, int NB = 2>
__host__ __device__ constexpr int gate_bytes() {
  return NB * xbuf_polys<P>() * kN * 8 + kGateAcc + kGateAbar + 16;
}
template <class F>
__host__ __device__ constexpr int tab_bytes() {
  return (sizeof(typename F::Tables) + 127) / 128 * 128;
}
// Exchange buffers per gate: two (one barrier per exchange) when they fit,
// one for 3 or more gates per CTA.
template <int G>
__host__ __device__ constexpr int xbufs_for() {
  return G >= 3 ? 1 : 2;
}
// digit tables of the first two forward stages (two-prime engine)
template <class F>
__host__ __device__ constexpr int digit_tab_bytes() {
  return F::kEngine == FSQL_ENGINE_DUAL_PRIME ? dev::kDigitTabs * dev::kDigitTabSize * 8 : 0;
}
// kOwn: every gate group stages its own key rows (one slot per group, no
// CTA-wide barrier per step, so the groups drift apart and their butterfly
// and exchange phases overlap); else one ring of kStages slots shared by all
// groups of the CTA.
template <class F, int G, int P, bool kOwn = false>
__host__ __device__ constexpr int br_smem() {
  return tab_bytes<F>() + digit_tab_bytes<F>() + (kOwn ? G : kStages) * P * kChunkU64 * 8 +
         G * gate_bytes<P, xbufs_for<G>()>();
}

constexpr int kKsGates = 16;                     // gates per keyswitch CTA
constexpr int kKsCols = 128;                     // output columns per keyswitch CTA
constexpr int kKsTiles = kKsRowWords / kKsCols;  // 5 column tiles cover n + 1 <= 640

#define CK(call)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
      return FSQL_ERR_CUDA;                                                      \
    }                                                                            \
  } while (0)

// ------------------------------------------------------------------ host math
uint64_t mulmod_host(uint64_t a, uint64_t b) {
  return static_cast<uint64_t>((static_cast<unsigned __int128>(a) * b) % kP);
}
uint64_t powmod_host(uint64_t a, uint64_t e) {
  uint64_t r = 1;
  while (e) {
    if (e & 1) r = mulmod_host(r, a);
    a = mulmod_host(a, a);
    e >>= 1;
  }
  return r;
}
uint32_t bitrev10(uint32_t k) {
  uint32_t r = 0;
  for (int b = 0; b < 10; ++b) r |= ((k >> b) & 1u) << (9 - b);
  return r;
}

uint64_t powmod_u32(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1;
  a %= m;
  while (e) {
    if (e & 1) r = r * a % m;
    a = a * a % m;
    e >>= 1;
  }
  return r;
}

// Fill the twiddle tables from f[k], g[k] (forward / inverse, bit-reversed
// powers, already in the engine's twiddle form) in the thread layouts of ntt.cuh.
template <class Tw>
void fill_tables(NttTablesT<Tw>* T, const std::vector<Tw>& f, const std::vector<Tw>& g, uint64_t key_scale) {
  for (int k = 0; k < 64; ++k) T->f_small[k] = f[k];
  for (int k = 0; k < 128; ++k) T->g_small[k] = g[k];
  for (int t = 0; t < kGroup; ++t) {
    const int h = t >> 1;
    T->f3[0][t] = f[64 + h];
    for (int c = 0; c < 2; ++c) T->f3[1 + c][t] = f[128 + 2 * h + c];
    for (int c = 0; c < 4; ++c) T->f3[3 + c][t] = f[256 + 4 * h + c];
    for (int c = 0; c < 4; ++c) T->f4[c][t] = f[512 + 4 * t + c];
    for (int c = 0; c < 4; ++c) T->i1[c][t] = g[512 + 4 * t + c];
    for (int c = 0; c < 2; ++c) T->i1[4 + c][t] = g[256 + 2 * t + c];
    T->i1[6][t] = g[128 + t];
  }
  T->n_inv = key_scale;
  T->pad = 0;
}

// Goldilocks: psi = 7^((p-1)/2048); 7 generates Z_p^*, so psi has order
// exactly 2048 (checked: psi^1024 = -1).  Key scale 1/N.
bool make_tables_goldilocks(std::vector<uint8_t>* out) {
  const uint64_t psi = powmod_host(7, (kP - 1) / 2048);
  if (powmod_host(psi, 1024) != kP - 1) return false;
  const uint64_t psi_inv = powmod_host(psi, kP - 2);
  std::vector<uint64_t> f(kN), g(kN);
  for (uint32_t k = 0; k < static_cast<uint32_t>(kN); ++k) {
    f[k] = powmod_host(psi, bitrev10(k));
    g[k] = powmod_host(psi_inv, bitrev10(k));
  }
  out->assign(sizeof(dev::Goldilocks::Tables), 0);
  fill_tables(reinterpret_cast<dev::Goldilocks::Tables*>(out->data()), f, g, powmod_host(kN, kP - 2));
  return true;
}

// Two primes: psi_i = gen_i^((p_i - 1)/2048) (13 and 3 generate the two
// groups; checked psi^1024 = -1); each twiddle residue w comes with its Shoup
// quotient floor(w 2^32 / p_i).  Key scale N^-1 R^2 (R = 2^32), packed
// (low word mod p1, high word mod p2).
bool make_tables_dual(std::vector<uint8_t>* out) {
  const uint64_t P[2] = {dev::kP1, dev::kP2}, gen[2] = {13, 3};
  const uint64_t Pinv[2] = {dev::kP1inv, dev::kP2inv};
  std::vector<uint4> f(kN), g(kN);
  uint64_t scale = 0;
  for (int i = 0; i < 2; ++i) {
    const uint64_t p = P[i];
    if (((p * Pinv[i]) & 0xFFFFFFFFull) != 1 || (p - 1) % 2048 != 0) return false;
    const uint64_t psi = powmod_u32(gen[i], (p - 1) / 2048, p);
    if (powmod_u32(psi, 1024, p) != p - 1) return false;
    const uint64_t psi_inv = powmod_u32(psi, p - 2, p);
    const uint64_t r = (1ull << 32) % p;
    for (uint32_t k = 0; k < static_cast<uint32_t>(kN); ++k) {
      const uint64_t wf = powmod_u32(psi, bitrev10(k), p), wg = powmod_u32(psi_inv, bitrev10(k), p);
      const uint32_t qf = static_cast<uint32_t>((wf << 32) / p), qg = static_cast<uint32_t>((wg << 32) / p);
      if (i == 0) {
        f[k].x = static_cast<uint32_t>(wf), f[k].y = qf;
        g[k].x = static_cast<uint32_t>(wg), g[k].y = qg;
      } else {
        f[k].z = static_cast<uint32_t>(wf), f[k].w = qf;
        g[k].z = static_cast<uint32_t>(wg), g[k].w = qg;
      }
    }
    scale |= (powmod_u32(kN, p - 2, p) * r % p * r % p) << (32 * i);
  }
  // CRT constant: (p1^-1 mod p2) R mod p2
  if (powmod_u32(dev::kP1, dev::kP2 - 2, dev::kP2) * ((1ull << 32) % dev::kP2) % dev::kP2 != dev::kCrtC) return false;
  out->assign(sizeof(dev::DualPrime::Tables), 0);
  fill_tables(reinterpret_cast<dev::DualPrime::Tables*>(out->data()), f, g, scale);
  return true;
}

// The two-prime tables split by prime: NttTablesT<uint2> {w, w'} for p1 then
// for p2, each padded to kSplitBytes.
template <int kSplitBytes>
void split_tables(const std::vector<uint8_t>& dual, std::vector<uint8_t>* out) {
  using TD = NttTablesT<uint4>;
  using TS = NttTablesT<uint2>;
  static_assert(sizeof(TS) <= static_cast<size_t>(kSplitBytes), "split table padding");
  const TD& d = *reinterpret_cast<const TD*>(dual.data());
  out->assign(2 * kSplitBytes, 0);
  for (int pr = 0; pr < 2; ++pr) {
    TS& o = *reinterpret_cast<TS*>(out->data() + pr * kSplitBytes);
    auto pick = [&](const uint4& w) { return pr == 0 ? make_uint2(w.x, w.y) : make_uint2(w.z, w.w); };
    for (int k = 0; k < 64; ++k) o.f_small[k] = pick(d.f_small[k]);
    for (int k = 0; k < 128; ++k) o.g_small[k] = pick(d.g_small[k]);
    for (int t = 0; t < kGroup; ++t) {
      for (int c = 0; c < 7; ++c) o.f3[c][t] = pick(d.f3[c][t]);
      for (int c = 0; c < 4; ++c) o.f4[c][t] = pick(d.f4[c][t]);
      for (int c = 0; c < 7; ++c) o.i1[c][t] = pick(d.i1[c][t]);
    }
    o.n_inv = pr == 0 ? (d.n_inv & 0xFFFFFFFFull) : (d.n_inv >> 32);
    o.pad = 0;
  }
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// The same copy with an L2 eviction-priority hint (a createpolicy descriptor):
// the blind-rotation key is re-read by every gate group while gate inputs and
// outputs stream through L2 once, so key lines are kept last.
__device__ __forceinline__ void cp_async16_hint(void* smem_dst, const void* gsrc, uint64_t policy) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "l"(policy)
               : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t policy;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(policy));
  return policy;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Gate linear forms on the +-q/8 encoding:
// out = (0, .., 0, k) + ca*c1 + cb*c2 + cc*c3.
struct Lin {
  uint32_t k;
  uint32_t ca, cb, cc;
};
__device__ __forceinline__ Lin gate_lin(uint32_t type) {
  const uint32_t E = 1u << 29, M = 0xFFFFFFFFu;  // q/8, -1
  switch (type) {
    case FSQL_NAND: return {E, M, M, 0u};
    case FSQL_AND: return {0u - E, 1u, 1u, 0u};
    case FSQL_OR: return {E, 1u, 1u, 0u};
    case FSQL_XOR: return {2u * E, 2u, 2u, 0u};
    case FSQL_XNOR: return {0u - 2u * E, 0u - 2u, 0u - 2u, 0u};
    case FSQL_NOR: return {0u - E, M, M, 0u};
    case FSQL_ANDNY: return {0u - E, M, 1u, 0u};
    case FSQL_ANDYN: return {0u - E, 1u, M, 0u};
    case FSQL_ORNY: return {E, M, 1u, 0u};
    case FSQL_MAJNYY: return {0u, M, 1u, 1u};  // majority of (not a, b, c): sign of -a + b + c
    case FSQL_XOR3: return {0u, 0u - 2u, 0u - 2u, 0u - 2u};  // parity of (a, b, c): sign of -2(a + b + c)
    case FSQL_MAJ: return {0u, 1u, 1u, 1u};  // majority of (a, b, c): sign of a + b + c
    default: return {E, 1u, M, 0u};  // FSQL_ORYN (other values compute ORYN)
  }
}

// ------------------------------------------------------------------ kernels

template <class Tab>
__device__ __forceinline__ void load_tables(Tab& T, const void* __restrict__ gtab) {
  for (int k = threadIdx.x; k < static_cast<int>(sizeof(Tab) / 8); k += blockDim.x)
    reinterpret_cast<uint64_t*>(&T)[k] = reinterpret_cast<const uint64_t*>(gtab)[k];
}

// Key conversion: one 128-thread CTA per key polynomial (i, row, c): forward
// NTT of the coefficients read as integers in [0, 2^32), times 1/N, stored as
// bkhat[i][row][k][t][c] (slot 8t + k) so that thread t of a gate group reads
// its (k, c = 0..1) pair as one 16-byte word.
template <class F>
__global__ void __launch_bounds__(kGroup) bk_to_ntt_kernel(const uint32_t* __restrict__ bk,
                                                           uint64_t* __restrict__ bkhat,
                                                           const void* __restrict__ gtab) {
  __shared__ typename F::Tables T;
  __shared__ uint64_t bufs[2 * kN];
  load_tables(T, gtab);
  __syncthreads();
  const int w = blockIdx.x, t = threadIdx.x;
  const int i = w / (kRows * 2), row = (w / 2) % kRows, c = w % 2;
  const uint32_t* src = bk + (static_cast<size_t>(i * kRows + row) * 2 + c) * kN;
  uint64_t x[1][8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[0][k] = F::from_u32(src[t + 128 * k]);
  int parity = 0;
  dev::ntt_forward<F, 1, 1>(x, bufs, parity, T, t, 1);
  uint64_t* dst = bkhat + static_cast<size_t>(i * kRows + row) * kChunkU64;
#pragma unroll
  for (int k = 0; k < 8; ++k) dst[(k * kGroup + t) * 2 + c] = F::scale_key(x[0][k], T.n_inv);
}

// Contiguous gate arrays -> descriptors.
__global__ void make_desc_kernel(GateDesc* __restrict__ desc, const uint8_t* __restrict__ types,
                                 const uint32_t* a, const uint32_t* b, uint32_t* out, int count, int words) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  GateDesc d;
  d.a = a + static_cast<size_t>(g) * words;
  d.b = b + static_cast<size_t>(g) * words;
  d.c = nullptr;
  d.out = out ? out + static_cast<size_t>(g) * words : nullptr;
  d.type = types[g];
  d.pad = 0;
  desc[g] = d;
}

// Stage the key rows of step k (kPolys rows, 32 KB, contiguous) into a ring slot.
template <int kThreads, int kStepU64>
__device__ __forceinline__ void issue_step(uint64_t* slot, const uint64_t* __restrict__ bkhat, int k, uint64_t policy) {
  const uint4* src = reinterpret_cast<const uint4*>(bkhat + static_cast<size_t>(k) * kStepU64);
  uint4* dst = reinterpret_cast<uint4*>(slot);
  for (int q = threadIdx.x; q < kStepU64 * 8 / 16; q += kThreads) cp_async16_hint(dst + q, src + q, policy);
}

// Blind rotation + sample extraction for `count` gates (see file comment),
// the body of blind_rotate_kernel and of each segment of scan_walk_kernel.
// big: [count][N+1] extracted samples under the GLWE key.  prepare: load the
// twiddle tables into shared memory first (and build the digit tables).
template <class F, int G, int kPolys, bool kOwn = false>
__device__ __forceinline__ void br_body(const GateDesc* __restrict__ desc, int count,
                                        const uint64_t* __restrict__ bkhat, const void* __restrict__ gtab, int n,
                                        int bg_bits, uint32_t* __restrict__ big, bool prepare) {
  static_assert(kRows % kPolys == 0 && kPolys <= kL, "gadget rows per step must divide 2l and not exceed l");
  constexpr int kThreads = G * kGroup;
  constexpr int kTabBytes = tab_bytes<F>();
  constexpr int kStepsPerCmux = kRows / kPolys;
  constexpr int kStepU64 = kPolys * kChunkU64;
  constexpr int kBufPolys = xbuf_polys<kPolys>();
  constexpr int kNB = xbufs_for<G>();
  constexpr int kGateXbuf = kNB * kBufPolys * kN * 8;
  constexpr int kGateBytes = gate_bytes<kPolys, kNB>();
  constexpr bool kDigitTab = F::kEngine == FSQL_ENGINE_DUAL_PRIME;
  extern __shared__ __align__(128) uint8_t smem[];
  typename F::Tables& T = *reinterpret_cast<typename F::Tables*>(smem);
  uint64_t* dtab = reinterpret_cast<uint64_t*>(smem + kTabBytes);  // digit tables (two-prime engine)
  uint64_t* stage = reinterpret_cast<uint64_t*>(smem + kTabBytes + digit_tab_bytes<F>());
  const int grp = threadIdx.x / kGroup, t = threadIdx.x % kGroup;
  const int bar = 1 + grp;  // named barrier of this gate's 128 threads
  if constexpr (kOwn) stage += grp * kStepU64;  // this group's own slot
  uint8_t* gb = smem + kTabBytes + digit_tab_bytes<F>() + (kOwn ? G : kStages) * kStepU64 * 8 + grp * kGateBytes;
  uint64_t* xbufs = reinterpret_cast<uint64_t*>(gb);                         // [2][kBufPolys][N] u64
  uint32_t* acc_poly = reinterpret_cast<uint32_t*>(gb + kGateXbuf);          // [2][N] u32
  uint16_t* abar = reinterpret_cast<uint16_t*>(gb + kGateXbuf + kGateAcc);   // [n]
  uint32_t* bbar_slot = reinterpret_cast<uint32_t*>(gb + kGateXbuf + kGateAcc + kGateAbar);

  // Signed gadget digits by the offset form: y = x + sum_j 2^(bg-1) 2^(32-bg j)
  // + 2^(31 - bg l); digit j = ((y >> (32 - bg j)) mod 2^bg) - 2^(bg-1).
  uint32_t off = 1u << (31 - bg_bits * kL);
  for (int j = 1; j <= kL; ++j) off += (1u << (bg_bits - 1)) << (32 - bg_bits * j);
  const uint32_t dmask = (1u << bg_bits) - 1, dhalf = 1u << (bg_bits - 1);
  const int total = n * kStepsPerCmux;
  if (prepare) {
    load_tables(T, gtab);
    if constexpr (kDigitTab) {
      __syncthreads();  // twiddle tables loaded
      dev::build_digit_tables(dtab, T, dhalf, threadIdx.x, kThreads);
    }
  }

  // copies of step k into a slot: all the CTA's threads (shared ring) or the
  // group's; key lines are kept in L2 ahead of the streaming gate inputs and
  // outputs (read and written once each, with the streaming cache hint)
  const uint64_t keep = l2_evict_last_policy();
  auto issue = [&](uint64_t* slot, int k) {
    if constexpr (kOwn) {
      const uint4* src = reinterpret_cast<const uint4*>(bkhat + static_cast<size_t>(k) * kStepU64);
      uint4* dst = reinterpret_cast<uint4*>(slot);
      for (int q = t; q < kStepU64 * 8 / 16; q += kGroup) cp_async16_hint(dst + q, src + q, keep);
    } else {
      issue_step<kThreads, kStepU64>(slot, bkhat, k, keep);
    }
  };
  for (int g0 = blockIdx.x * G; g0 < count; g0 += gridDim.x * G) {
    const int gi = g0 + grp;
    const bool active = gi < count;
    __syncthreads();  // tables loaded; previous group finished with the stages
    if (!kOwn || active) issue(stage, 0);
    cp_async_commit();

    if (active) {
      const GateDesc d = desc[gi];
      const Lin lin = gate_lin(d.type);
      // linear combination and modulus switch q -> 2N (round half up)
      const uint32_t* c3 = lin.cc ? d.c : nullptr;  // a missing third input counts as zero
      for (int x = t; x <= n; x += kGroup) {
        uint32_t v = lin.ca * __ldcs(d.a + x) + lin.cb * __ldcs(d.b + x);
        if (c3) v += lin.cc * __ldcs(c3 + x);
        if (x == n) v += lin.k;
        const uint32_t ms = ((v + (1u << 20)) >> 21) & (2 * kN - 1);
        if (x < n) abar[x] = static_cast<uint16_t>(ms);
        else *bbar_slot = ms;
      }
      dev::named_sync(bar);
      // ACC = (0, X^{-bbar} * v), v_k = q/8 for all k
      const uint32_t e = (2 * kN - *bbar_slot) & (2 * kN - 1);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t c = t + 128 * k;
        acc_poly[c] = 0u;
        const uint32_t idx = (c - e) & (2 * kN - 1);
        acc_poly[kN + c] = idx < static_cast<uint32_t>(kN) ? (1u << 29) : (0u - (1u << 29));
      }
    }

    int parity = 0;
    typename F::Acc acc[8];
    uint32_t diff0[8], diff1[8];
    for (int i = 0; i < n; ++i) {
#pragma unroll 1
      for (int s = 0; s < kStepsPerCmux; ++s) {
        const int k = i * kStepsPerCmux + s;
        if constexpr (kOwn) {
          if (!active) continue;
          cp_async_wait<0>();
          dev::named_sync(bar);  // the group's key rows of step k visible; its ACC update done
        } else {
          cp_async_wait<0>();
          __syncthreads();  // key rows of step k visible; everyone done with step k-1 and the ACC update
          if (k + 1 < total) issue(stage + ((k + 1) % kStages) * kStepU64, k + 1);
          cp_async_commit();
        }
        if (active) {
          // X^a ACC_u - ACC_u, formed by the step holding row 3u and reused by
          // the l gadget levels of polynomial u (rows 3u .. 3u+2)
          if (s == 0 || s == kL / kPolys) {
            const uint32_t a_i = abar[i];
            const uint32_t* P = acc_poly + (s == 0 ? 0 : kN);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const uint32_t c = t + 128 * q;
              const uint32_t idx = (c - a_i) & (2 * kN - 1);  // (X^a P)_c = +-P[idx mod N]
              const uint32_t rot = idx < static_cast<uint32_t>(kN) ? P[idx] : 0u - P[idx - kN];
              const uint32_t v = rot - P[c] + off;
              if (s == 0) diff0[q] = v;
              else diff1[q] = v;
            }
          }
          uint64_t x[kPolys][8];
#pragma unroll
          for (int p = 0; p < kPolys; ++p) {
            const int row = s * kPolys + p;
            const int shift = 32 - bg_bits * (row % kL + 1);
            if constexpr (kDigitTab) {
              uint32_t u[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) u[q] = ((row < kL ? diff0[q] : diff1[q]) >> shift) & dmask;
              dev::digit_stages12(u, x[p], dhalf, dtab);
            } else {
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const uint32_t v = row < kL ? diff0[q] : diff1[q];
                x[p][q] = F::from_digit((v >> shift) & dmask, dhalf);
              }
            }
          }
          dev::ntt_forward<F, kPolys, kBufPolys, kNB, kDigitTab>(x, xbufs, parity, T, t, bar);
          const uint64_t* ch = kOwn ? stage : stage + (k % kStages) * kStepU64;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
#pragma unroll
            for (int p = 0; p < kPolys; ++p) {
              const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(ch + p * kChunkU64 + (q * kGroup + t) * 2);
              F::mac(acc[q], x[p][q], w, s == 0 && p == 0);
            }
          }
        }
        if constexpr (kOwn) {
          dev::named_sync(bar);  // the group is done reading its slot
          if (k + 1 < total) issue(stage, k + 1);  // lands while the next step forms and transforms digits
          cp_async_commit();
        }
      }
      if (active) {
        uint64_t y[2][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          y[0][q] = F::acc0(acc[q]);
          y[1][q] = F::acc1(acc[q]);
        }
        dev::ntt_inverse<F, 2, kBufPolys, kNB>(y, xbufs, parity, T, t, bar);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc_poly[c * kN + t + 128 * q] += F::to_torus(y[c][q]);
      }
    }

    if (active) {
      dev::named_sync(bar);
      // sample extraction of coefficient 0: a'_0 = A_0, a'_c = -A_{N-c}, b' = B_0
      uint32_t* out = big + static_cast<size_t>(gi) * (kN + 1);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = t + 128 * q;
        __stcs(out + c, c == 0 ? acc_poly[0] : 0u - acc_poly[kN - c]);
      }
      if (t == 0) __stcs(out + kN, acc_poly[kN]);
    }
  }
}

template <class F, int G, int kPolys, bool kOwn = false>
__global__ void __launch_bounds__(G * kGroup, 1)
    blind_rotate_kernel(const GateDesc* __restrict__ desc, int count, const uint64_t* __restrict__ bkhat,
                        const void* __restrict__ gtab, int n, int bg_bits, uint32_t* __restrict__ big) {
  br_body<F, G, kPolys, kOwn>(desc, count, bkhat, gtab, n, bg_bits, big, true);
}

// ---------------------------------------------------------------- end of blind_rotate_kernel's device code

// Prime-split blind rotation (br_split.cuh): G gates per CTA of 256 threads
// each (half 0: residues mod p1, half 1: mod p2), P gadget rows per step.
constexpr int kSplitTabBytes = (sizeof(dev::SplitTables) + 127) / 128 * 128;
template <int P>
__host__ __device__ constexpr int split_gate_bytes() {
  // per half one exchange buffer (32-bit residues); the CRT buffer [2][N];
  // the accumulator; the switched mask; the switched body
  return 2 * xbuf_polys<P>() * kN * 4 + 2 * kN * 4 + kGateAcc + kGateAbar + 16;
}
template <int G, int P, int S>
__host__ __device__ constexpr int split_smem() {
  return 2 * kSplitTabBytes + S * P * kChunkU64 * 8 + G * split_gate_bytes<P>();
}

// G gates per CTA, P gadget rows per step, S slots in the key-staging ring
// (cp.async of step k + S - 1 is in flight while step k computes).
template <int G, int P, int S>
__global__ void __launch_bounds__(G * 2 * kGroup, 1)
    blind_rotate_split_kernel(const GateDesc* __restrict__ desc, int count, const uint32_t* __restrict__ bks,
                              const void* __restrict__ gtab, int n, int bg_bits, uint32_t* __restrict__ big) {
  static_assert(kRows % P == 0 && P <= kL, "gadget rows per step must divide 2l and not exceed l");
  constexpr int kThreads = G * 2 * kGroup;
  constexpr int kStepsPerCmux = kRows / P;
  constexpr int kRowU32 = 2 * kChunkU64;  // one key row, both primes (16 KB)
  constexpr int kStepU32 = P * kRowU32;
  constexpr int kBufPolys = xbuf_polys<P>();
  constexpr int kGateBytes = split_gate_bytes<P>();
  extern __shared__ __align__(128) uint8_t smem[];
  const int grp = threadIdx.x / (2 * kGroup), h = (threadIdx.x / kGroup) & 1, t = threadIdx.x % kGroup;
  const dev::SplitTables& T = *reinterpret_cast<const dev::SplitTables*>(smem + h * kSplitTabBytes);
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem + 2 * kSplitTabBytes);
  uint8_t* gb = smem + 2 * kSplitTabBytes + S * kStepU32 * 4 + grp * kGateBytes;
  uint32_t* xbuf = reinterpret_cast<uint32_t*>(gb) + h * kBufPolys * kN;  // this half's exchange buffer
  uint32_t* crt = reinterpret_cast<uint32_t*>(gb) + 2 * kBufPolys * kN;   // [2][N]: residues for the other half
  uint32_t* acc_poly = crt + 2 * kN;                                        // [2][N]
  uint16_t* abar = reinterpret_cast<uint16_t*>(acc_poly + 2 * kN);          // [kMaxN]
  uint32_t* bbar_slot = reinterpret_cast<uint32_t*>(abar + kMaxN);
  const int bar_half = 1 + 2 * grp + h;  // this half's 128 threads
  const int bar_gate = 1 + 2 * G + grp;  // the gate's 256 threads
  const uint32_t p = h ? dev::kP2 : dev::kP1, p2 = 2 * p, pinv = h ? dev::kP2inv : dev::kP1inv;
  const uint64_t* bks64 = reinterpret_cast<const uint64_t*>(bks);

  for (int k = threadIdx.x; k < 2 * kSplitTabBytes / 16; k += kThreads)
    reinterpret_cast<uint4*>(smem)[k] = reinterpret_cast<const uint4*>(gtab)[k];

  uint32_t off = 1u << (31 - bg_bits * kL);
  for (int j = 1; j <= kL; ++j) off += (1u << (bg_bits - 1)) << (32 - bg_bits * j);
  const uint32_t dmask = (1u << bg_bits) - 1, lift = p - (1u << (bg_bits - 1));  // digit u - half -> u + p - half
  const int total = n * kStepsPerCmux;
  const uint64_t keep = l2_evict_last_policy();  // key lines stay in L2 ahead of streaming gate I/O

  for (int g0 = blockIdx.x * G; g0 < count; g0 += gridDim.x * G) {
    const int gi = g0 + grp;
    const bool active = gi < count;
    __syncthreads();  // tables loaded; previous gates finished with the stages
#pragma unroll
    for (int k = 0; k < S - 1; ++k) {  // the first S - 1 steps in flight
      if (k < total)
        issue_step<kThreads, P * kChunkU64>(reinterpret_cast<uint64_t*>(stage + k * kStepU32), bks64, k, keep);
      cp_async_commit();
    }

    if (active) {
      const GateDesc d = desc[gi];
      const Lin lin = gate_lin(d.type);
      const uint32_t* c3 = lin.cc ? d.c : nullptr;  // a missing third input counts as zero
      for (int x = h * kGroup + t; x <= n; x += 2 * kGroup) {
        uint32_t v = lin.ca * d.a[x] + lin.cb * d.b[x];
        if (c3) v += lin.cc * c3[x];
        if (x == n) v += lin.k;
        const uint32_t ms = ((v + (1u << 20)) >> 21) & (2 * kN - 1);
        if (x < n) abar[x] = static_cast<uint16_t>(ms);
        else *bbar_slot = ms;
      }
      dev::named_sync_n(bar_gate, 2 * kGroup);
      // ACC = (0, X^{-bbar} v), v_k = q/8: half h writes polynomial h
      const uint32_t e = (2 * kN - *bbar_slot) & (2 * kN - 1);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t c = t + 128 * q;
        const uint32_t idx = (c - e) & (2 * kN - 1);
        acc_poly[h * kN + c] = h == 0 ? 0u : (idx < static_cast<uint32_t>(kN) ? (1u << 29) : (0u - (1u << 29)));
      }
    }

    int parity = 0;
    uint64_t acc0[8], acc1[8];
    uint32_t diff0[8], diff1[8];
    for (int i = 0; i < n; ++i) {
#pragma unroll 1
      for (int s = 0; s < kStepsPerCmux; ++s) {
        const int k = i * kStepsPerCmux + s;
        cp_async_wait<S - 2>();  // this thread's copies of step k have landed
        __syncthreads();  // everyone's copies of step k visible; slot (k - 1) % S free; ACC of the previous CMux complete
        if (k + S - 1 < total)
          issue_step<kThreads, P * kChunkU64>(
              reinterpret_cast<uint64_t*>(stage + ((k + S - 1) % S) * kStepU32), bks64, k + S - 1, keep);
        cp_async_commit();
        if (active) {
          // X^a ACC_u - ACC_u (plus the decomposition offset) for the
          // polynomial(s) of this step's rows
          if (s == 0 || s == kL / P) {
            const uint32_t a_i = abar[i];
            const uint32_t* Pu = acc_poly + (s == 0 ? 0 : kN);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const uint32_t c = t + 128 * q;
              const uint32_t idx = (c - a_i) & (2 * kN - 1);
              const uint32_t rot = idx < static_cast<uint32_t>(kN) ? Pu[idx] : 0u - Pu[idx - kN];
              const uint32_t v = rot - Pu[c] + off;
              if (s == 0) diff0[q] = v;
              else diff1[q] = v;
            }
          }
          uint32_t x[P][8];
#pragma unroll
          for (int r = 0; r < P; ++r) {
            const int row = s * P + r;
            const int shift = 32 - bg_bits * (row % kL + 1);
#pragma unroll
            for (int q = 0; q < 8; ++q) x[r][q] = (((row < kL ? diff0[q] : diff1[q]) >> shift) & dmask) + lift;
          }
          dev::ntt_forward32<P, kBufPolys, 1>(x, xbuf, parity, T, t, bar_half, p, p2);
          const uint32_t* ch = stage + (k % S) * kStepU32 + h * kChunkU64;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
#pragma unroll
            for (int r = 0; r < P; ++r) {
              const uint2 w = *reinterpret_cast<const uint2*>(ch + r * kRowU32 + (q * kGroup + t) * 2);
              const bool first = s == 0 && r == 0;
              acc0[q] = static_cast<uint64_t>(x[r][q]) * w.x + (first ? 0ull : acc0[q]);
              acc1[q] = static_cast<uint64_t>(x[r][q]) * w.y + (first ? 0ull : acc1[q]);
            }
          }
        }
      }
      if (active) {
        uint32_t y[2][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          y[0][q] = dev::DualPrime::settle(acc0[q], p, pinv);
          y[1][q] = dev::DualPrime::settle(acc1[q], p, pinv);
        }
        dev::ntt_inverse32<2, kBufPolys, 1>(y, xbuf, parity, T, t, bar_half, p, p2);
        // CRT: half 0 lifts output polynomial 0, half 1 polynomial 1; each
        // passes its residues of the other polynomial through crt[]
        if (h == 0) {
#pragma unroll
          for (int q = 0; q < 8; ++q) crt[t + 128 * q] = y[1][q];
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) crt[kN + t + 128 * q] = y[0][q];
        }
        dev::named_sync_n(bar_gate, 2 * kGroup);
        if (h == 0) {
#pragma unroll
          for (int q = 0; q < 8; ++q) acc_poly[t + 128 * q] += dev::crt_torus(y[0][q], crt[kN + t + 128 * q]);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) acc_poly[kN + t + 128 * q] += dev::crt_torus(crt[t + 128 * q], y[1][q]);
        }
      }
    }

    if (active) {
      dev::named_sync_n(bar_gate, 2 * kGroup);
      // sample extraction of coefficient 0: a'_0 = A_0, a'_c = -A_{N-c}, b' = B_0
      uint32_t* out = big + static_cast<size_t>(gi) * (kN + 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = h * kGroup + t + 256 * q;
        out[c] = c == 0 ? acc_poly[0] : 0u - acc_poly[kN - c];
      }
      if (h == 0 && t == 0) out[kN] = acc_poly[kN];
    }
  }
}

// Cluster blind rotation: one gate per thread-block cluster of 6 CTAs of 256
// threads, on 6 SMs, for batches too small to fill the GPU (the per-gate
// path and the narrow levels of deep circuits).  A gate's 630 CMux steps are
// a dependent chain, so one gate on one SM is bound by that SM's integer
// pipes and latencies; here its work per CMux is spread over 6 SMs that
// exchange through distributed shared memory.  CTA rank r = 3 pr + s works
// mod prime pr (p1 or p2, 32-bit residues) on gadget rows 2s and 2s + 1, one
// row per 128-thread group g.  Per CMux:
//   1. every CTA keeps a copy of the ACC polynomials its rows read (CTA
//      (pr, 1) both, the others one); group g forms the digits of row
//      2s + g, transforms them mod pr (first two stages by digit table) and
//      multiplies them with the row's staged key words for both output
//      polynomials, reduced to [0, 2p); the two groups add their rows in
//      shared memory, and group g stores the CTA's sum for output polynomial
//      g into the CTA that reduces it (distributed shared memory);
//   2. cluster barrier; group 0 of CTA (pr, 0) for output polynomial 0 and
//      of CTA (pr, 2) for polynomial 1 sums the three partials it received,
//      folds to [0, 2p), runs the inverse transform and stores the residues
//      into the four CTAs whose rows read that polynomial;
//   3. cluster barrier; every CTA lifts by CRT the polynomials its rows read
//      (both groups, half the coefficients each) and adds them into its own
//      ACC; the sample is extracted by CTA (0, 1).
// Only a few tens of GB/s leave each SM through distributed shared memory,
// hence the pre-summed rows, stores only where the data is read, plain
// shared stores for the CTA's own copy, and 4-byte stores coalesced across
// each warp (wider per-thread stores with this layout move the same bytes
// more slowly).  The residues summed are those the packed kernel sums (the
// same integer mod each prime), so the CRT gives the same exact integer and
// the same words.
constexpr int kClusterCtas = 6;
constexpr int kClusterThreads = 2 * kGroup;
constexpr int kClusterSmem = kSplitTabBytes + dev::kDigitTabs * dev::kDigitTabSize * 4 +  // tables
                             2 * 2 * kChunkU64 * 4 +                                        // key rows, 2 slots
                             2 * kN * 4 +                                                   // exchange buffer per group
                             2 * kN * 4 + 2 * kN * 4 +                                      // ACC, rows of the other group
                             3 * kN * 4 + 4 * kN * 4 +                                      // partial sums, residues
                             kMaxN * 2 + 16;                                                // switched mask, body

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads, 1)
    blind_rotate_cluster_kernel(const GateDesc* __restrict__ desc, int count, const uint32_t* __restrict__ bks,
                                const void* __restrict__ gtab, int n, int bg_bits, uint32_t* __restrict__ big) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int pr = rank / 3, s = rank % 3;
  const int grp = threadIdx.x / kGroup, t = threadIdx.x % kGroup, tid = threadIdx.x;
  extern __shared__ __align__(128) uint8_t smem[];
  dev::SplitTables& T = *reinterpret_cast<dev::SplitTables*>(smem);
  uint32_t* dtab = reinterpret_cast<uint32_t*>(smem + kSplitTabBytes);
  uint32_t* keys = dtab + dev::kDigitTabs * dev::kDigitTabSize;  // [2 slots][2 rows][kChunkU64]
  uint32_t* xbuf = keys + 2 * 2 * kChunkU64 + grp * kN;           // this group's exchange buffer [N]
  uint32_t* acc_poly = keys + 2 * 2 * kChunkU64 + 2 * kN;          // [2][N]
  uint32_t* other = acc_poly + 2 * kN;                             // [2][N]: [c] = the other group's row, output c
  uint32_t* part = other + 2 * kN;                                 // [3 senders s][N], slot-major (q * 128 + t)
  uint32_t* resid = part + 3 * kN;                                 // [2 polys][2 primes][N]
  uint16_t* abar = reinterpret_cast<uint16_t*>(resid + 4 * kN);    // [kMaxN]
  uint32_t* bbar_slot = reinterpret_cast<uint32_t*>(abar + kMaxN);
  const uint32_t p = pr ? dev::kP2 : dev::kP1, p2 = 2 * p, pinv = pr ? dev::kP2inv : dev::kP1inv;
  const int bar = 1 + grp;  // the group's named barrier (128 threads)

  for (int k = tid; k < kSplitTabBytes / 16; k += kClusterThreads)
    reinterpret_cast<uint4*>(smem)[k] = reinterpret_cast<const uint4*>(gtab)[pr * (kSplitTabBytes / 16) + k];
  uint32_t off = 1u << (31 - bg_bits * kL);
  for (int j = 1; j <= kL; ++j) off += (1u << (bg_bits - 1)) << (32 - bg_bits * j);
  const uint32_t dmask = (1u << bg_bits) - 1, dhalf = 1u << (bg_bits - 1);
  __syncthreads();
  dev::build_digit_tables32(dtab, T, dhalf, p, tid, kClusterThreads);
  // this group's gadget row and the polynomials the CTA's two rows read
  const int row = 2 * s + grp, u = row / kL, shift = 32 - bg_bits * (row % kL + 1);
  const int u0 = (2 * s) / kL, u1 = (2 * s + 1) / kL;
  auto issue_row = [&](int i, int slot) {  // this group's key row of CMux i, this prime (8 KB)
    const uint4* src = reinterpret_cast<const uint4*>(bks + ((static_cast<size_t>(i) * kRows + row) * 2 + pr) * kChunkU64);
    uint4* dst = reinterpret_cast<uint4*>(keys + (slot * 2 + grp) * kChunkU64);
    for (int q = t; q < kChunkU64 * 4 / 16; q += kGroup) cp_async16(dst + q, src + q);
    cp_async_commit();
  };
  // group g sends the CTA's partial sum of output polynomial g to the CTA that
  // reduces it, (pr, 0) for g = 0 and (pr, 2) for g = 1, slot s (its own
  // shared memory when that is this CTA); the reducing CTA of polynomial c
  // sends its residues (slot [c][pr]) to the CTAs whose rows read c: ranks
  // c, c + 1, c + 3, c + 4
  const int red_c = s == 0 ? 0 : s == 2 ? 1 : -1;  // the polynomial this CTA reduces, if any
  const int part_rank = pr * 3 + 2 * grp;
  uint32_t* const part_to = (part_rank == rank ? part : cl.map_shared_rank(part, part_rank)) + s * kN;
  uint32_t* resid_to[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int m = (red_c < 0 ? 0 : red_c) + (k & 1) + 3 * (k >> 1);
    resid_to[k] = (m == rank ? resid : cl.map_shared_rank(resid, m)) + ((red_c < 0 ? 0 : red_c) * 2 + pr) * kN;
  }

  for (int gi = static_cast<int>(blockIdx.x) / kClusterCtas; gi < count;
       gi += static_cast<int>(gridDim.x) / kClusterCtas) {
    __syncthreads();
    issue_row(0, 0);
    const GateDesc d = desc[gi];
    const Lin lin = gate_lin(d.type);
    const uint32_t* c3 = lin.cc ? d.c : nullptr;
    for (int x = tid; x <= n; x += kClusterThreads) {
      uint32_t v = lin.ca * d.a[x] + lin.cb * d.b[x];
      if (c3) v += lin.cc * c3[x];
      if (x == n) v += lin.k;
      const uint32_t ms = ((v + (1u << 20)) >> 21) & (2 * kN - 1);
      if (x < n) abar[x] = static_cast<uint16_t>(ms);
      else *bbar_slot = ms;
    }
    __syncthreads();
    {
      const uint32_t e = (2 * kN - *bbar_slot) & (2 * kN - 1);
      for (int c = tid; c < kN; c += kClusterThreads) {
        acc_poly[c] = 0u;
        const uint32_t idx = (static_cast<uint32_t>(c) - e) & (2 * kN - 1);
        acc_poly[kN + c] = idx < static_cast<uint32_t>(kN) ? (1u << 29) : (0u - (1u << 29));
      }
    }
    int parity = 0;
    for (int i = 0; i < n; ++i) {
      cp_async_wait<0>();
      __syncthreads();  // key rows of CMux i landed; ACC updated
      if (i + 1 < n) issue_row(i + 1, (i + 1) & 1);
      else cp_async_commit();
      const uint32_t a_i = abar[i];
      uint32_t dg[8];
      const uint32_t* P = acc_poly + u * kN;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t c = t + 128 * q;
        const uint32_t idx = (c - a_i) & (2 * kN - 1);
        const uint32_t r = idx < static_cast<uint32_t>(kN) ? P[idx] : 0u - P[idx - kN];
        dg[q] = ((r - P[c] + off) >> shift) & dmask;
      }
      uint32_t x[1][8];
      dev::digit_stages12_32(dg, x[0], dhalf, dtab, p, p2);
      dev::ntt_forward32<1, 1, 1, true>(x, xbuf, parity, T, t, bar, p, p2);
      const uint32_t* ch = keys + ((i & 1) * 2 + grp) * kChunkU64;
      uint32_t mine[8];  // this row's product with output polynomial grp, below 2p
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint2 w = *reinterpret_cast<const uint2*>(ch + (q * kGroup + t) * 2);
        const uint32_t y0 = dev::DualPrime::settle(static_cast<uint64_t>(x[0][q]) * w.x, p, pinv);
        const uint32_t y1 = dev::DualPrime::settle(static_cast<uint64_t>(x[0][q]) * w.y, p, pinv);
        other[(1 - grp) * kN + q * kGroup + t] = grp ? y0 : y1;  // the output the other group sends
        mine[q] = grp ? y1 : y0;
      }
      __syncthreads();  // both rows' products in shared memory
#pragma unroll
      for (int q = 0; q < 8; ++q) part_to[q * kGroup + t] = mine[q] + other[grp * kN + q * kGroup + t];  // below 4p
      cl.sync();  // 1: every partial sum delivered
      if (red_c >= 0 && grp == 0) {
        uint32_t y[1][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int o = q * kGroup + t;
          const uint32_t v = part[o] + part[kN + o] + part[2 * kN + o];  // three sums below 4p: below 12p
          y[0][q] = dev::fold(dev::fold(dev::fold(v, 4 * p2), 2 * p2), p2);
        }
        dev::ntt_inverse32<1, 1, 1>(y, xbuf, parity, T, t, bar, p, p2);
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int q = 0; q < 8; ++q) resid_to[m][t + 128 * q] = y[0][q];
      }
      cl.sync();  // 2: the residues of the polynomials each CTA reads, mod both primes, delivered
      // lift by CRT the polynomials the CTA's rows read and update ACC (the
      // two groups take alternate coefficients; the buffers are written again
      // only after the next CMux's barrier 1)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c != u0 && c != u1) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + kClusterThreads * q;
          acc_poly[c * kN + e] += dev::crt_torus(resid[(c * 2) * kN + e], resid[(c * 2 + 1) * kN + e]);
        }
      }
    }
    __syncthreads();
    if (rank == 1) {  // CTA (0, 1) keeps both polynomials of ACC
      uint32_t* out = big + static_cast<size_t>(gi) * (kN + 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = tid + kClusterThreads * q;
        out[c] = c == 0 ? acc_poly[0] : 0u - acc_poly[kN - c];
      }
      if (tid == 0) out[kN] = acc_poly[kN];
    }
  }
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

// Packed key (u64: p1 residue low, p2 residue high) -> key split by prime.
__global__ void split_key_kernel(const uint64_t* __restrict__ bkhat, uint32_t* __restrict__ bks, size_t rows) {
  const size_t total = rows * kChunkU64;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t r = e / kChunkU64, w = e % kChunkU64;
    const uint64_t v = bkhat[e];
    bks[r * 2 * kChunkU64 + w] = static_cast<uint32_t>(v);
    bks[r * 2 * kChunkU64 + kChunkU64 + w] = static_cast<uint32_t>(v >> 32);
  }
}

// Latency mode of the blind rotation (batches smaller than two gates per
// SM, where one 128-thread group per gate leaves the SMs mostly idle and a
// gate's 630 CMux steps are a sequential chain).  One gate per CTA of three
// 128-thread groups: in every CMux, group s takes gadget rows 2s and 2s+1
// (the three steps of the throughput kernel run side by side), stages its
// two key rows with cp.async, transforms its two digit polynomials and
// multiply-accumulates them; the groups' reduced sums (each in [0, 2p))
// meet in shared memory, and groups 0 and 1 each add the three partials of
// one output polynomial (below 6p, two folds to [0, 2p)), run its inverse
// transform and add it into ACC.  The arithmetic is the throughput
// kernel's, so the words are the same.  Two-prime engine only.
constexpr int kLatGroups = kRows / 2;  // three groups of two gadget rows

template <class F>
__host__ __device__ constexpr int lat_smem() {
  return tab_bytes<F>() + kLatGroups * 2 * kChunkU64 * 8 + kLatGroups * 2 * kN * 8 + kGateAcc + kGateAbar + 16 +
         digit_tab_bytes<F>();
}

template <class F>
__global__ void __launch_bounds__(kLatGroups * kGroup, 1)
    blind_rotate_latency_kernel(const GateDesc* __restrict__ desc, int count, const uint64_t* __restrict__ bkhat,
                                const void* __restrict__ gtab, int n, int bg_bits, uint32_t* __restrict__ big) {
  static_assert(F::kEngine == FSQL_ENGINE_DUAL_PRIME, "latency mode is built for the two-prime engine");
  constexpr int kThreads = kLatGroups * kGroup;
  extern __shared__ __align__(128) uint8_t smem[];
  typename F::Tables& T = *reinterpret_cast<typename F::Tables*>(smem);
  uint64_t* stage = reinterpret_cast<uint64_t*>(smem + tab_bytes<F>());  // [group][2 rows][kChunkU64]
  uint64_t* xb_all = stage + kLatGroups * 2 * kChunkU64;                   // [group][2 polys][N]
  uint32_t* acc_poly = reinterpret_cast<uint32_t*>(xb_all + kLatGroups * 2 * kN);  // [2][N]
  uint16_t* abar = reinterpret_cast<uint16_t*>(acc_poly + 2 * kN);                 // [n]
  uint32_t* bbar_slot = reinterpret_cast<uint32_t*>(abar + kMaxN);
  uint64_t* dtab = reinterpret_cast<uint64_t*>(bbar_slot + 4);  // digit tables of the first two stages
  const int grp = threadIdx.x / kGroup, t = threadIdx.x % kGroup;
  const int bar = 1 + grp;
  uint64_t* xbufs = xb_all + grp * 2 * kN;
  uint64_t* my_stage = stage + grp * 2 * kChunkU64;

  load_tables(T, gtab);
  uint32_t off = 1u << (31 - bg_bits * kL);
  for (int j = 1; j <= kL; ++j) off += (1u << (bg_bits - 1)) << (32 - bg_bits * j);
  const uint32_t dmask = (1u << bg_bits) - 1, dhalf = 1u << (bg_bits - 1);
  __syncthreads();  // twiddle tables loaded
  dev::build_digit_tables(dtab, T, dhalf, threadIdx.x, kThreads);
  // rows 2 grp and 2 grp + 1 belong to polynomials (2 grp) / l and (2 grp + 1) / l
  const int row0 = 2 * grp, row1 = 2 * grp + 1;
  const int u0 = row0 / kL, u1 = row1 / kL;
  const int shift0 = 32 - bg_bits * (row0 % kL + 1), shift1 = 32 - bg_bits * (row1 % kL + 1);

  for (int gi = blockIdx.x; gi < count; gi += gridDim.x) {
    __syncthreads();  // tables loaded; the previous gate is extracted
    const GateDesc d = desc[gi];
    const Lin lin = gate_lin(d.type);
    const uint32_t* c3 = lin.cc ? d.c : nullptr;
    for (int x = threadIdx.x; x <= n; x += kThreads) {
      uint32_t v = lin.ca * d.a[x] + lin.cb * d.b[x];
      if (c3) v += lin.cc * c3[x];
      if (x == n) v += lin.k;
      const uint32_t ms = ((v + (1u << 20)) >> 21) & (2 * kN - 1);
      if (x < n) abar[x] = static_cast<uint16_t>(ms);
      else *bbar_slot = ms;
    }
    __syncthreads();
    {
      const uint32_t e = (2 * kN - *bbar_slot) & (2 * kN - 1);
      for (int c = threadIdx.x; c < kN; c += kThreads) {
        acc_poly[c] = 0u;
        const uint32_t idx = (static_cast<uint32_t>(c) - e) & (2 * kN - 1);
        acc_poly[kN + c] = idx < static_cast<uint32_t>(kN) ? (1u << 29) : (0u - (1u << 29));
      }
    }
    int parity = 0;
    for (int i = 0; i < n; ++i) {
      __syncthreads();  // ACC of the previous CMux complete; its stage and partials consumed
      {
        const uint4* src = reinterpret_cast<const uint4*>(bkhat + static_cast<size_t>(i * kRows + row0) * kChunkU64);
        uint4* dst = reinterpret_cast<uint4*>(my_stage);
        for (int q = t; q < 2 * kChunkU64 * 8 / 16; q += kGroup) cp_async16(dst + q, src + q);
        cp_async_commit();
      }
      const uint32_t a_i = abar[i];
      uint64_t x[2][8];
      uint32_t d0[8], d1[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t c = t + 128 * q;
        const uint32_t idx = (c - a_i) & (2 * kN - 1);
        uint32_t v[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const uint32_t* Pu = acc_poly + (r == 0 ? u0 : u1) * kN;
          const uint32_t rot = idx < static_cast<uint32_t>(kN) ? Pu[idx] : 0u - Pu[idx - kN];
          v[r] = rot - Pu[c] + off;
        }
        d0[q] = (v[0] >> shift0) & dmask;
        d1[q] = (v[1] >> shift1) & dmask;
      }
      dev::digit_stages12(d0, x[0], dhalf, dtab);
      dev::digit_stages12(d1, x[1], dhalf, dtab);
      dev::ntt_forward<F, 2, 2, 1, true>(x, xbufs, parity, T, t, bar);
      cp_async_wait<0>();
      dev::named_sync(bar);  // the group's key rows are visible to all its threads
      typename F::Acc acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(my_stage + p * kChunkU64 + (q * kGroup + t) * 2);
          F::mac(acc[q], x[p][q], w, p == 0);
        }
      dev::named_sync(bar);  // the group is done reading its key rows: reuse them for the partial sums
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        my_stage[8 * t + q] = F::acc0(acc[q]);       // output polynomial 0, forward-output slot 8t + q
        my_stage[kN + 8 * t + q] = F::acc1(acc[q]);  // output polynomial 1
      }
      __syncthreads();  // every group's partial sums written
      if (grp < 2) {
        uint64_t y[1][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          uint32_t s1 = 0, s2 = 0;
#pragma unroll
          for (int g = 0; g < kLatGroups; ++g) {
            const uint64_t v = stage[g * 2 * kChunkU64 + grp * kN + 8 * t + q];
            s1 += dev::lo32(v);
            s2 += dev::hi32(v);
          }
          y[0][q] = dev::pack(dev::fold(dev::fold(s1, 4 * dev::kP1), 2 * dev::kP1),
                              dev::fold(dev::fold(s2, 4 * dev::kP2), 2 * dev::kP2));
        }
        dev::ntt_inverse<F, 1, 2, 1>(y, xbufs, parity, T, t, bar);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc_poly[grp * kN + t + 128 * q] += F::to_torus(y[0][q]);
      }
    }
    __syncthreads();
    uint32_t* out = big + static_cast<size_t>(gi) * (kN + 1);
    for (int c = threadIdx.x; c < kN; c += kThreads) out[c] = c == 0 ? acc_poly[0] : 0u - acc_poly[kN - c];
    if (threadIdx.x == 0) out[kN] = acc_poly[kN];
  }
}

// Keyswitch N -> n (see file comment).  Rounding: a + 2^15, keep the top 16
// bits, 8 base-4 digits most significant first; digit v at level j selects
// key row KSK[i][j][v-1]; out = (0, .., 0, b) - sum of the selected rows.
// Grid: (gate groups of kKsGates, column tiles of kKsCols); each thread owns
// one output column of every gate of its group.  For each position i the
// thread copies its column of the 3 x 8 nonzero-digit key rows into its own
// slots of a shared table whose digit-0 rows are zero, so each gate's term is
// one table load indexed by its digit (no compare or select); only the
// owning thread reads a slot, so no barrier is needed.  Output of gate g goes
// to desc[g].out when desc is given, else to out_contig + g*(n+1).
// One keyswitch tile: gates [g0, g0 + 16) of the batch (fewer at its end),
// output columns [tile * 128, tile * 128 + 128), by 128 threads (tc = 0..127)
// that synchronise on named barrier `bar` (0: the whole 128-thread CTA).
// dig and tbl are the tile's shared buffers; the caller orders their reuse.
__device__ __forceinline__ void ks_tile(const uint32_t* __restrict__ big, const GateDesc* __restrict__ desc,
                                        uint32_t* __restrict__ out_contig, int count, const uint32_t* __restrict__ ksk,
                                        int n, int g0, int tile, uint16_t (*dig)[kN],
                                        uint32_t (*tbl)[4][kKsCols], int tc, int bar) {
  const int ng = min(kKsGates, count - g0);
  for (int q = tc; q < kKsGates * kN; q += kKsCols) {
    const int g = q / kN, i = q % kN;
    uint16_t v = 0;
    if (g < ng) v = static_cast<uint16_t>((big[static_cast<size_t>(g0 + g) * (kN + 1) + i] + (1u << 15)) >> 16);
    dig[g][i] = v;
  }
#pragma unroll
  for (int j = 0; j < kKsT; ++j) tbl[j][0][tc] = 0u;
  asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "r"(kKsCols) : "memory");
  const int col = tile * kKsCols + tc;
  uint32_t acc[kKsGates];
#pragma unroll
  for (int g = 0; g < kKsGates; ++g) acc[g] = 0u;
  const uint32_t* base = ksk + col;
  // the 24 key words of position i + 1 are loaded while position i is summed
  uint32_t nxt[kKsT][kKsDigits];
#pragma unroll
  for (int j = 0; j < kKsT; ++j)
#pragma unroll
    for (int v = 0; v < kKsDigits; ++v) nxt[j][v] = __ldg(base + static_cast<size_t>(j * kKsDigits + v) * kKsRowWords);
#pragma unroll 1
  for (int i = 0; i < kN; ++i) {
#pragma unroll
    for (int j = 0; j < kKsT; ++j)
#pragma unroll
      for (int v = 0; v < kKsDigits; ++v) tbl[j][1 + v][tc] = nxt[j][v];
    if (i + 1 < kN) {
      const uint32_t* rows = base + static_cast<size_t>((i + 1) * kKsT * kKsDigits) * kKsRowWords;
#pragma unroll
      for (int j = 0; j < kKsT; ++j)
#pragma unroll
        for (int v = 0; v < kKsDigits; ++v) nxt[j][v] = __ldg(rows + static_cast<size_t>(j * kKsDigits + v) * kKsRowWords);
    }
#pragma unroll
    for (int g = 0; g < kKsGates; ++g) {
      const uint32_t dv = dig[g][i];
#pragma unroll
      for (int j = 0; j < kKsT; ++j) acc[g] -= tbl[j][(dv >> (14 - 2 * j)) & 3u][tc];
    }
  }
  if (col > n) return;
#pragma unroll
  for (int g = 0; g < kKsGates; ++g) {
    if (g >= ng) break;
    uint32_t* out = desc ? desc[g0 + g].out : out_contig + static_cast<size_t>(g0 + g) * (n + 1);
    const uint32_t body = col == n ? big[static_cast<size_t>(g0 + g) * (kN + 1) + kN] : 0u;
    out[col] = acc[g] + body;
  }
}

__global__ void __launch_bounds__(kKsCols)
    keyswitch_kernel(const uint32_t* __restrict__ big, const GateDesc* __restrict__ desc,
                     uint32_t* __restrict__ out_contig, int count, const uint32_t* __restrict__ ksk, int n) {
  __shared__ uint16_t dig[kKsGates][kN];
  __shared__ uint32_t tbl[kKsT][4][kKsCols];  // [level][digit][column of this tile]
  ks_tile(big, desc, out_contig, count, ksk, n, blockIdx.x * kKsGates, blockIdx.y, dig, tbl, threadIdx.x, 0);
}

// ------------------------------------------------------------------ device level walker
// scan_walk_kernel runs a whole batched scan in one cooperative launch (one
// CTA per SM, all resident): for each segment (a circuit level, or a part of
// one no larger than the extracted-sample scratch) the CTAs bootstrap its
// gates (br_body, persistent over gate groups), meet at a grid barrier, then
// keyswitch them (16-gate x 128-column tiles spread over every 128-thread
// group of every CTA), and meet again before the next level, whose gates read
// the outputs just written.  The host issues one launch per scan instead of
// two per level.  Every barrier wait is bounded (see grid_barrier): a wait
// that runs out of time raises an error word and every CTA returns, so the
// GPU context stays usable and the host reads FSQL_ERR_TIMEOUT.
struct WalkSeg {
  uint32_t begin, count;  // descriptors [begin, begin + count)
};
constexpr int kKsSmem = kKsGates * kN * 2 + kKsT * 4 * kKsCols * 4;  // dig + tbl of one keyswitch tile

__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch.  Thread 0 of every CTA adds one
// arrival (unless `skip`: a test hook that makes this CTA never arrive) and
// polls, with a pause between reads, until the arrivals of this barrier are
// complete (target = (index + 1) x CTAs; the counter only grows), an error
// is raised, or timeout_ns of device time (or a fixed number of polls)
// passes, in which case it raises the error and records the barrier index.
// The fences make every write of the CTAs before the barrier visible to every
// read after it.  Returns false on error, the same answer in every thread.
__device__ bool grid_barrier(WalkSync* sync, unsigned int& target, unsigned int index, long long timeout_ns,
                             bool skip) {
  __syncthreads();
  target += gridDim.x;
  int ok = 1;
  if (threadIdx.x == 0) {
    if (!skip) {
      __threadfence();
      atomicAdd(&sync->arrived, 1u);
    }
    const long long t0 = globaltimer_ns();
    for (long long polls = 0;; ++polls) {
      unsigned int a;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(a) : "l"(&sync->arrived) : "memory");
      if (a >= target) break;
      if (*reinterpret_cast<volatile unsigned int*>(&sync->error)) {
        ok = 0;
        break;
      }
      if (globaltimer_ns() - t0 > timeout_ns || polls > (1ll << 26)) {
        if (atomicCAS(&sync->error, 0u, 1u) == 0u) sync->barrier = index;
        ok = 0;
        break;
      }
      __nanosleep(200);
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

template <class F, int G, int kPolys, bool kOwn>
__host__ __device__ constexpr int walk_smem() {
  return br_smem<F, G, kPolys, kOwn>() > tab_bytes<F>() + digit_tab_bytes<F>() + G * kKsSmem
             ? br_smem<F, G, kPolys, kOwn>()
             : tab_bytes<F>() + digit_tab_bytes<F>() + G * kKsSmem;
}

template <class F, int G, int kPolys, bool kOwn>
__global__ void __launch_bounds__(G * kGroup, 1)
    scan_walk_kernel(const GateDesc* __restrict__ desc, const WalkSeg* __restrict__ segs, int nsegs,
                     const uint64_t* __restrict__ bkhat, const void* __restrict__ gtab, int n, int bg_bits,
                     uint32_t* __restrict__ big, const uint32_t* __restrict__ ksk, WalkSync* sync,
                     long long timeout_ns, int skip_block) {
  extern __shared__ __align__(128) uint8_t smem[];
  const bool skip = skip_block == static_cast<int>(blockIdx.x);
  const int grp = threadIdx.x / kGroup, tc = threadIdx.x % kGroup;
  // keyswitch buffers after the twiddle and digit tables, which every segment keeps
  uint8_t* ksb = smem + tab_bytes<F>() + digit_tab_bytes<F>() + grp * kKsSmem;
  auto* dig = reinterpret_cast<uint16_t(*)[kN]>(ksb);
  auto* tbl = reinterpret_cast<uint32_t(*)[4][kKsCols]>(ksb + kKsGates * kN * 2);
  unsigned int target = 0, index = 0;
  for (int sg = 0; sg < nsegs; ++sg) {
    const WalkSeg seg = segs[sg];
    const GateDesc* d = desc + seg.begin;
    const int count = static_cast<int>(seg.count);
    br_body<F, G, kPolys, kOwn>(d, count, bkhat, gtab, n, bg_bits, big, sg == 0);
    if (!grid_barrier(sync, target, index++, timeout_ns, skip)) return;
    const int items = (count + kKsGates - 1) / kKsGates * kKsTiles;
    for (int it = blockIdx.x * G + grp; it < items; it += gridDim.x * G) {
      dev::named_sync(1 + grp);  // the group's previous tile is done with dig and tbl
      ks_tile(big, d, nullptr, count, ksk, n, (it / kKsTiles) * kKsGates, it % kKsTiles, dig, tbl, tc, 1 + grp);
    }
    if (!grid_barrier(sync, target, index++, timeout_ns, skip)) return;
  }
}

// Keyswitch of small batches (latency): the 1024 input positions are split
// over `splits` CTAs per (gate group, column tile); CTA s sums the key rows
// of positions [s 1024/splits, (s+1) 1024/splits) into its own partial
// (part[s][gate][column], kKsPartGates gates per split) and
// keyswitch_reduce_kernel adds the partials and the body.  Addition mod 2^32
// is associative, so the words equal the single-pass kernel's.
constexpr int kKsPartGates = 128;  // largest batch that takes the split path
constexpr int kKsMaxSplits = 16;

__global__ void __launch_bounds__(kKsCols)
    keyswitch_part_kernel(const uint32_t* __restrict__ big, int count, const uint32_t* __restrict__ ksk, int splits,
                          uint32_t* __restrict__ part) {
  __shared__ uint16_t dig[kKsGates][kN / 2];
  __shared__ uint32_t tbl[kKsT][4][kKsCols];
  const int g0 = blockIdx.x * kKsGates;
  const int ng = min(kKsGates, count - g0);
  const int span = kN / splits, i0 = blockIdx.z * span;
  for (int q = threadIdx.x; q < kKsGates * span; q += kKsCols) {
    const int g = q / span, i = q % span;
    uint16_t v = 0;
    if (g < ng) v = static_cast<uint16_t>((big[static_cast<size_t>(g0 + g) * (kN + 1) + i0 + i] + (1u << 15)) >> 16);
    dig[g][i] = v;
  }
  const int tc = threadIdx.x;
#pragma unroll
  for (int j = 0; j < kKsT; ++j) tbl[j][0][tc] = 0u;
  __syncthreads();
  const int col = blockIdx.y * kKsCols + tc;
  uint32_t acc[kKsGates];
#pragma unroll
  for (int g = 0; g < kKsGates; ++g) acc[g] = 0u;
  const uint32_t* base = ksk + col;
#pragma unroll 1
  for (int i = 0; i < span; ++i) {
#pragma unroll
    for (int j = 0; j < kKsT; ++j) {
      const uint32_t* rows = base + static_cast<size_t>(((i0 + i) * kKsT + j) * kKsDigits) * kKsRowWords;
      tbl[j][1][tc] = __ldg(rows);
      tbl[j][2][tc] = __ldg(rows + kKsRowWords);
      tbl[j][3][tc] = __ldg(rows + 2 * kKsRowWords);
    }
#pragma unroll
    for (int g = 0; g < kKsGates; ++g) {
      const uint32_t dv = dig[g][i];
#pragma unroll
      for (int j = 0; j < kKsT; ++j) acc[g] -= tbl[j][(dv >> (14 - 2 * j)) & 3u][tc];
    }
  }
#pragma unroll
  for (int g = 0; g < kKsGates; ++g) {
    if (g >= ng) break;
    part[(static_cast<size_t>(blockIdx.z) * kKsPartGates + g0 + g) * kKsRowWords + col] = acc[g];
  }
}

// One CTA per gate: out = (0, .., 0, b') + the sum of the splits' partials.
__global__ void __launch_bounds__(kKsCols)
    keyswitch_reduce_kernel(const uint32_t* __restrict__ part, int splits, const uint32_t* __restrict__ big,
                            const GateDesc* __restrict__ desc, uint32_t* __restrict__ out_contig, int n) {
  const int g = blockIdx.x;
  uint32_t* out = desc ? desc[g].out : out_contig + static_cast<size_t>(g) * (n + 1);
  for (int col = threadIdx.x; col <= n; col += kKsCols) {
    uint32_t v = col == n ? big[static_cast<size_t>(g) * (kN + 1) + kN] : 0u;
    for (int s = 0; s < splits; ++s) v += part[(static_cast<size_t>(s) * kKsPartGates + g) * kKsRowWords + col];
    out[col] = v;
  }
}

// Keyswitch-first order (ciphertexts of N + 1 words under the N-bit key):
// the gate's linear combination is formed on the fly from its N + 1-word
// inputs while digits are extracted, and the single keyswitched result goes
// to out_contig[g] (n + 1 words), the blind rotation's input.
__global__ void __launch_bounds__(kKsCols)
    keyswitch_lincomb_kernel(const GateDesc* __restrict__ desc, int count, const uint32_t* __restrict__ ksk, int n,
                             uint32_t* __restrict__ out_contig) {
  __shared__ uint16_t dig[kKsGates][kN];
  __shared__ uint32_t tbl[kKsT][4][kKsCols];
  const int g0 = blockIdx.x * kKsGates;
  const int ng = min(kKsGates, count - g0);
  for (int q = threadIdx.x; q < kKsGates * kN; q += kKsCols) {
    const int g = q / kN, i = q % kN;
    uint32_t v = 0;
    if (g < ng) {
      const GateDesc d = desc[g0 + g];
      const Lin lin = gate_lin(d.type);
      v = lin.ca * d.a[i] + lin.cb * d.b[i];
      if (lin.cc && d.c) v += lin.cc * d.c[i];
    }
    dig[g][i] = static_cast<uint16_t>((v + (1u << 15)) >> 16);
  }
  const int tc = threadIdx.x;
#pragma unroll
  for (int j = 0; j < kKsT; ++j) tbl[j][0][tc] = 0u;
  __syncthreads();
  const int col = blockIdx.y * kKsCols + tc;
  uint32_t acc[kKsGates];
#pragma unroll
  for (int g = 0; g < kKsGates; ++g) acc[g] = 0u;
  const uint32_t* base = ksk + col;
  // the 24 key words of position i + 1 are loaded while position i is summed
  uint32_t nxt[kKsT][kKsDigits];
#pragma unroll
  for (int j = 0; j < kKsT; ++j)
#pragma unroll
    for (int v = 0; v < kKsDigits; ++v) nxt[j][v] = __ldg(base + static_cast<size_t>(j * kKsDigits + v) * kKsRowWords);
#pragma unroll 1
  for (int i = 0; i < kN; ++i) {
#pragma unroll
    for (int j = 0; j < kKsT; ++j)
#pragma unroll
      for (int v = 0; v < kKsDigits; ++v) tbl[j][1 + v][tc] = nxt[j][v];
    if (i + 1 < kN) {
      const uint32_t* rows = base + static_cast<size_t>((i + 1) * kKsT * kKsDigits) * kKsRowWords;
#pragma unroll
      for (int j = 0; j < kKsT; ++j)
#pragma unroll
        for (int v = 0; v < kKsDigits; ++v) nxt[j][v] = __ldg(rows + static_cast<size_t>(j * kKsDigits + v) * kKsRowWords);
    }
#pragma unroll
    for (int g = 0; g < kKsGates; ++g) {
      const uint32_t dv = dig[g][i];
#pragma unroll
      for (int j = 0; j < kKsT; ++j) acc[g] -= tbl[j][(dv >> (14 - 2 * j)) & 3u][tc];
    }
  }
  if (col > n) return;
#pragma unroll
  for (int g = 0; g < kKsGates; ++g) {
    if (g >= ng) break;
    uint32_t body = 0u;  // the linear combination's body word
    if (col == n) {
      const GateDesc d = desc[g0 + g];
      const Lin lin = gate_lin(d.type);
      body = lin.ca * d.a[kN] + lin.cb * d.b[kN] + lin.k;
      if (lin.cc && d.c) body += lin.cc * d.c[kN];
    }
    out_contig[static_cast<size_t>(g0 + g) * (n + 1) + col] = acc[g] + body;
  }
}

// Blind-rotation descriptors of the keyswitched samples: AND with the
// noiseless trivial true (0, .., 0, q/8) is the identity on the linear
// combination (-q/8 + x + q/8 = x), so the bootstrap sees x unchanged.
__global__ void identity_desc_kernel(GateDesc* __restrict__ desc, int count, const uint32_t* __restrict__ small,
                                     const uint32_t* __restrict__ trivial_true, int words) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  GateDesc d;
  d.a = small + static_cast<size_t>(g) * words;
  d.b = trivial_true;
  d.c = nullptr;
  d.out = nullptr;
  d.type = FSQL_AND;
  d.pad = 0;
  desc[g] = d;
}

// Extracted samples (N + 1 words) to the gates' outputs.
__global__ void copy_out_kernel(const GateDesc* __restrict__ desc, const uint32_t* __restrict__ big, int count) {
  for (int g = blockIdx.x; g < count; g += gridDim.x) {
    uint32_t* out = desc[g].out;
    for (int x = threadIdx.x; x <= kN; x += blockDim.x) out[x] = big[static_cast<size_t>(g) * (kN + 1) + x];
  }
}

// Exact negacyclic product through the device NTT (test hook), 128 threads.
template <class F>
__global__ void __launch_bounds__(kGroup) ntt_mul_kernel(const int32_t* __restrict__ digits,
                                                         const uint32_t* __restrict__ poly,
                                                         uint32_t* __restrict__ out,
                                                         const void* __restrict__ gtab) {
  __shared__ typename F::Tables T;
  __shared__ uint64_t bufs[2 * kN];
  load_tables(T, gtab);
  __syncthreads();
  const int t = threadIdx.x;
  uint64_t x[1][8], y[1][8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[0][k] = F::from_int(digits[t + 128 * k]);
    y[0][k] = F::from_u32(poly[t + 128 * k]);
  }
  int parity = 0;
  dev::ntt_forward<F, 1, 1>(x, bufs, parity, T, t, 1);
  __syncthreads();  // the next transform's first exchange writes across warps
  dev::ntt_forward<F, 1, 1>(y, bufs, parity, T, t, 1);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint64_t ys = F::scale_key(y[0][k], T.n_inv);
    typename F::Acc a;
    F::mac(a, x[0][k], make_ulonglong2(ys, ys), true);
    x[0][k] = F::acc0(a);
  }
  dev::ntt_inverse<F, 1, 1>(x, bufs, parity, T, t, 1);
#pragma unroll
  for (int k = 0; k < 8; ++k) out[t + 128 * k] = F::to_torus(x[0][k]);
}

}  // namespace

// ------------------------------------------------------------------ host side

// Tuned launch shape (index + 1; 0 = none), per (device, engine), for later
// contexts of this process.
static std::mutex g_tune_mu;
static int g_tuned[64][2] = {};
void remember_tuning(int device, int engine, int shape) {
  if (device < 0 || device >= 64 || engine < 0 || engine > 1) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[device][engine] = shape + 1;
}
static int tuned_shape(int device, int engine) {
  if (device < 0 || device >= 64 || engine < 0 || engine > 1) return 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tuned[device][engine];
}

long scan_internal_wires(const Netlist& nl) {
  long k = 0;
  for (int g = 0; g < nl.first_mask_gate; ++g)
    if (nl.n_inputs + g != nl.match_wire) ++k;
  return k;
}

void scan_literals(const Netlist& nl, const ScanIO& io, std::vector<OutDesc>* out) {
  out->clear();
  if (nl.literal_outs.empty()) return;
  const size_t W = io.words;
  const int w = static_cast<int>(io.width);
  const int pw = static_cast<int>(io.payload_width);
  std::vector<long> scratch_index(nl.type.size(), -1);
  long n_int = 0;
  for (int g = 0; g < nl.first_mask_gate; ++g)
    if (nl.n_inputs + g != nl.match_wire) scratch_index[g] = n_int++;
  auto wire_ptr = [&](int id, size_t row) -> const uint32_t* {
    if (id < 0) return nullptr;
    if (id < w) return io.column + (row * io.width + id) * W;
    if (id < w + nl.n_const) return io.cst + static_cast<size_t>(id - w) * W;
    if (id < nl.n_inputs) {
      const int m = id - w - nl.n_const;
      return io.payloads[m / pw] + (row * pw + m % pw) * W;
    }
    // an intermediate gate output (the mask gates and the match gate are never literal sources)
    return io.wires + (row * n_int + scratch_index[id - nl.n_inputs]) * W;
  };
  out->reserve(io.rows * nl.literal_outs.size());
  for (size_t row = 0; row < io.rows; ++row)
    for (const auto& l : nl.literal_outs) {
      OutDesc d;
      d.src = wire_ptr(l.wire, row);
      d.dst = l.target < 0 ? io.match + row * W : io.outs[l.target / pw] + (row * pw + l.target % pw) * W;
      d.mode = l.mode;
      d.pad = 0;
      out->push_back(d);
    }
}

// ------------------------------------------------------------------ scan plan

struct Plan {
  // key of the cached plan
  const uint32_t* column = nullptr;
  size_t rows = 0;
  uint32_t width = 0, pred = 0, n_payloads = 0, payload_width = 0;
  const uint32_t* cst = nullptr;
  std::vector<const uint32_t*> payloads;
  uint32_t* match = nullptr;
  std::vector<uint32_t*> outs;
  uint32_t* wires = nullptr;
  bool plain = false;  // plaintext constants k0 (and k1 for RANGE)
  bool ks_first = false;  // keyswitch-first order: every ciphertext N + 1 words
  uint64_t k0 = 0, k1 = 0;
  // plan
  std::vector<size_t> level_offset;  // descriptors of level L: [level_offset[L], level_offset[L+1])
  size_t total = 0;
  size_t n_lits = 0;  // outputs no gate writes, descriptors in Ctx::d_lits
  // the plan's level launches captured as a CUDA graph (rebuilt if the
  // context's descriptor or sample buffers move or its launch shape changes)
  cudaGraphExec_t graph = nullptr;
  const GateDesc* graph_desc = nullptr;
  const uint32_t* graph_big = nullptr;
  const OutDesc* graph_lits = nullptr;
  int graph_br_shape = -1;  // launch shape: 4 x shape index + latency mode
  uint64_t graph_ks_gen = 0;  // keyswitch-first scratch generation the graph was captured with
  long long graph_walk = -1;  // walker arguments when the graph was captured (0: no walker)
  // device walker: the plan's segments (levels split at the sample scratch)
  WalkSeg* d_segs = nullptr;
  int nsegs = 0;
  size_t segs_chunk = 0;      // sample-scratch capacity the segments were cut for
  // aggregation plans (SUM, MAX, MIN): key and the buffers they own
  int agg_kind = -1;
  const uint32_t* agg_in = nullptr;
  const uint32_t* agg_match = nullptr;
  uint32_t* agg_out = nullptr;
  uint32_t agg_width = 0, agg_out_width = 0;
  GateDesc* own_desc = nullptr;
  OutDesc* own_lits = nullptr;
  uint32_t* own_wires = nullptr;
  ~Plan() {
    if (graph) cudaGraphExecDestroy(graph);
    cudaFree(d_segs);
    cudaFree(own_desc);
    cudaFree(own_lits);
    cudaFree(own_wires);
  }
};


// Kernel timing: an event pair around each launch while profiling.
struct Profile {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> br, ks;  // indices into pool
  size_t used = 0;
  uint64_t gates = 0;
  bool recording = false;
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  ~Profile() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// Records an event pair around one launch when the context is profiling.
struct LaunchTimer {
  Profile* p;
  cudaStream_t st;
  int a = -1;
  LaunchTimer(Ctx& c, cudaStream_t s) : p(static_cast<Profile*>(c.prof)), st(s) {
    if (p && !p->recording) p = nullptr;
    if (p) {
      a = static_cast<int>(p->used);
      cudaEvent_t e = p->get();
      if (e) cudaEventRecord(e, st);
      else a = -1;
    }
  }
  void done(bool is_br, size_t gates) {
    if (!p || a < 0) return;
    const int b = static_cast<int>(p->used);
    cudaEvent_t e = p->get();
    if (!e) return;
    cudaEventRecord(e, st);
    (is_br ? p->br : p->ks).emplace_back(a, b);
    if (is_br) p->gates += gates;
  }
};

int device_init(Ctx& c) {
  const fsql_params& p = c.p;
  if (p.N != static_cast<uint32_t>(kN) || p.l != static_cast<uint32_t>(kL) || p.bg_bits < 2 || p.bg_bits > 10 ||
      p.ks_base_bits != static_cast<uint32_t>(kKsBaseBits) || p.ks_t != static_cast<uint32_t>(kKsT) ||
      p.n > static_cast<uint32_t>(kMaxN) || p.n + 1 > static_cast<uint32_t>(kKsRowWords)) {
    set_error("the GPU kernels implement N=1024, l=3, bg_bits in [2,10], ks base 4 x 8 levels, n <= 639");
    return FSQL_ERR_UNSUPPORTED;
  }
  CK(cudaSetDevice(c.device));
  // gates per CTA for large batches: measured best on B300 unless tuned in this process
  c.br_shape = c.engine == FSQL_ENGINE_GOLDILOCKS ? 3 : 8;  // packed 4 gates / 3 gates with a key slot per group
  if (const int g = tuned_shape(c.device, c.engine)) c.br_shape = g - 1;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
  c.sm_count = sms;
  if (!(c.engine == FSQL_ENGINE_GOLDILOCKS ? make_tables_goldilocks(&c.tables) : make_tables_dual(&c.tables))) {
    set_error("NTT root of unity check failed");
    return FSQL_ERR_ARG;
  }
  const size_t bkhat_words = static_cast<size_t>(p.n) * kRows * kChunkU64;
  const size_t ksk_words = static_cast<size_t>(kN) * kKsT * kKsDigits * kKsRowWords;
  CK(cudaMalloc(&c.d_tables, c.tables.size()));
  CK(cudaMalloc(&c.d_bkhat, bkhat_words * 8));
  CK(cudaMalloc(&c.d_ksk, ksk_words * 4));
  CK(cudaMalloc(&c.d_ks_part, static_cast<size_t>(kKsMaxSplits) * kKsPartGates * kKsRowWords * 4));
  c.key_bytes = bkhat_words * 8 + ksk_words * 4 + c.tables.size();
  CK(cudaMemcpy(c.d_tables, c.tables.data(), c.tables.size(), cudaMemcpyHostToDevice));

  // keyswitching key rows padded to kKsRowWords
  std::vector<uint32_t> kp(ksk_words, 0u);
  const size_t rows = static_cast<size_t>(kN) * kKsT * kKsDigits;
  for (size_t r = 0; r < rows; ++r)
    std::memcpy(kp.data() + r * kKsRowWords, c.ksk.data() + r * (p.n + 1), (p.n + 1) * 4);
  CK(cudaMemcpy(c.d_ksk, kp.data(), ksk_words * 4, cudaMemcpyHostToDevice));

  uint32_t* d_bk = nullptr;
  CK(cudaMalloc(&d_bk, c.bk.size() * 4));
  cudaError_t e = cudaMemcpy(d_bk, c.bk.data(), c.bk.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int polys = static_cast<int>(p.n) * kRows * 2;
    if (c.engine == FSQL_ENGINE_GOLDILOCKS)
      bk_to_ntt_kernel<dev::Goldilocks><<<polys, kGroup>>>(d_bk, c.d_bkhat, c.d_tables);
    else
      bk_to_ntt_kernel<dev::DualPrime><<<polys, kGroup>>>(d_bk, c.d_bkhat, c.d_tables);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(d_bk);
  if (e != cudaSuccess) {
    set_error(std::string("bootstrapping key conversion: ") + cudaGetErrorString(e));
    return FSQL_ERR_CUDA;
  }
  CK(cudaMalloc(&c.d_walk_sync, sizeof(WalkSync)));
  CK(cudaMemset(c.d_walk_sync, 0, sizeof(WalkSync)));
  if (c.engine == FSQL_ENGINE_DUAL_PRIME) {
    // the prime-split kernel's copy of the key and its per-prime twiddle tables
    std::vector<uint8_t> st;
    split_tables<kSplitTabBytes>(c.tables, &st);
    CK(cudaMalloc(&c.d_tables_split, st.size()));
    CK(cudaMemcpy(c.d_tables_split, st.data(), st.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c.d_bks, bkhat_words * 8));
    const size_t key_rows = static_cast<size_t>(p.n) * kRows;
    split_key_kernel<<<1184, 256>>>(c.d_bkhat, c.d_bks, key_rows);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    c.key_bytes += bkhat_words * 8 + st.size();
  }
  return FSQL_OK;
}

void device_free(Ctx& c) {
  if (c.device < 0) return;
  cudaSetDevice(c.device);
  cudaFree(c.d_bkhat);
  cudaFree(c.d_ksk);
  cudaFree(c.d_tables);
  cudaFree(c.d_bks);
  cudaFree(c.d_tables_split);
  cudaFree(c.d_walk_sync);
  c.d_walk_sync = nullptr;
  c.d_bks = nullptr;
  c.d_tables_split = nullptr;
  cudaFree(c.d_big);
  cudaFree(c.d_desc);
  cudaFree(c.d_wires);
  cudaFree(c.d_stage);
  cudaFree(c.d_prog);
  c.d_prog = nullptr;
  c.prog_cap = 0;
  cudaFree(c.d_ks_part);
  c.d_ks_part = nullptr;
  cudaFree(c.d_ks_small);
  cudaFree(c.d_ks_desc);
  cudaFree(c.d_true);
  c.d_ks_small = nullptr;
  c.d_ks_desc = nullptr;
  c.d_true = nullptr;
  c.ks_small_cap = 0;
  cudaFree(c.d_lits);
  c.d_lits = nullptr;
  c.lits_cap = 0;
  if (c.capture_stream) cudaStreamDestroy(static_cast<cudaStream_t>(c.capture_stream));
  c.capture_stream = nullptr;
  delete static_cast<Profile*>(c.prof);
  c.prof = nullptr;
  delete c.plan;
  c.plan = nullptr;
  delete c.agg_plan;
  c.agg_plan = nullptr;
  c.d_bkhat = nullptr;
  c.d_ksk = nullptr;
  c.d_tables = nullptr;
  c.d_big = nullptr;
  c.d_desc = nullptr;
  c.d_wires = nullptr;
  c.d_stage = nullptr;
}

// Launch the blind rotation with G gates per CTA and P gadget rows per step
// (persistent grid of at most one CTA per SM).
template <class F, int G, int P, bool kOwn = false>
static cudaError_t launch_br_engine(int sm_count, const GateDesc* d_desc, size_t count, const uint64_t* bkhat,
                                    const void* tables, int n, int bg_bits, uint32_t* d_big, cudaStream_t st) {
  static_assert(br_smem<F, G, P, kOwn>() <= 227 * 1024, "blind-rotation shared memory over budget");
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(blind_rotate_kernel<F, G, P, kOwn>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, br_smem<F, G, P, kOwn>());
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const size_t groups = (count + G - 1) / G;
  const int grid = static_cast<int>(std::min<size_t>(groups, static_cast<size_t>(sm_count)));
  blind_rotate_kernel<F, G, P, kOwn><<<grid, G * kGroup, br_smem<F, G, P, kOwn>(), st>>>(
      d_desc, static_cast<int>(count), bkhat, tables, n, bg_bits, d_big);
  return cudaGetLastError();
}

// Prime-split kernel: G gates per CTA (2 x 128 threads each), P gadget rows
// per step, persistent grid of at most one CTA per SM.
template <int G, int P, int S>
static cudaError_t launch_br_split(int sm_count, const GateDesc* d_desc, size_t count, const uint32_t* bks,
                                   const void* tables, int n, int bg_bits, uint32_t* d_big, cudaStream_t st) {
  static_assert(split_smem<G, P, S>() <= 227 * 1024, "prime-split shared memory over budget");
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(blind_rotate_split_kernel<G, P, S>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, split_smem<G, P, S>());
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const size_t groups = (count + G - 1) / G;
  const int grid = static_cast<int>(std::min<size_t>(groups, static_cast<size_t>(sm_count)));
  blind_rotate_split_kernel<G, P, S><<<grid, G * 2 * kGroup, split_smem<G, P, S>(), st>>>(
      d_desc, static_cast<int>(count), bks, tables, n, bg_bits, d_big);
  return cudaGetLastError();
}

// Cluster mode (two-prime engine): one gate per cluster of 6 CTAs, each on an
// SM of its own (the dynamic shared memory requested, above half an SM's,
// keeps a second CTA off the SM).  Returns cudaErrorNotSupported when the
// device cannot hold a cluster, so the caller falls back.
constexpr int kClusterSmemLaunch = kClusterSmem > 120 * 1024 ? kClusterSmem : 120 * 1024;
static cudaError_t cluster_capacity(int* clusters) {
  static int cap[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (cap[dev] == 0) {
    cudaError_t e = cudaFuncSetAttribute(blind_rotate_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kClusterSmemLaunch);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = kClusterSmemLaunch;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, blind_rotate_cluster_kernel, &cfg);
    if (e != cudaSuccess) return e;
    cap[dev] = n > 0 ? n : -1;
  }
  *clusters = cap[dev];
  return cap[dev] > 0 ? cudaSuccess : cudaErrorNotSupported;
}

static cudaError_t launch_br_cluster(size_t count, const GateDesc* d_desc, const uint32_t* bks, const void* tables,
                                     int n, int bg_bits, uint32_t* d_big, cudaStream_t st) {
  int clusters = 0;
  const cudaError_t e = cluster_capacity(&clusters);
  if (e != cudaSuccess) return e;
  const int grid = static_cast<int>(std::min<size_t>(count, static_cast<size_t>(clusters))) * kClusterCtas;
  blind_rotate_cluster_kernel<<<grid, kClusterThreads, kClusterSmemLaunch, st>>>(d_desc, static_cast<int>(count), bks, tables,
                                                                        n, bg_bits, d_big);
  return cudaGetLastError();
}

// Latency mode (two-prime engine): one gate per CTA of three groups.// Latency mode (two-prime engine): one gate per CTA of three groups.
template <class F>
static cudaError_t launch_br_latency(int sm_count, const GateDesc* d_desc, size_t count, const uint64_t* bkhat,
                                     const void* tables, int n, int bg_bits, uint32_t* d_big, cudaStream_t st) {
  static_assert(lat_smem<F>() <= 227 * 1024, "latency-mode shared memory over budget");
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(blind_rotate_latency_kernel<F>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, lat_smem<F>());
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int grid = static_cast<int>(std::min<size_t>(count, static_cast<size_t>(sm_count)));
  blind_rotate_latency_kernel<F><<<grid, kLatGroups * kGroup, lat_smem<F>(), st>>>(d_desc, static_cast<int>(count),
                                                                                    bkhat, tables, n, bg_bits, d_big);
  return cudaGetLastError();
}

// Launch shapes measured best on B300 per engine: the 64-bit prime is ALU
// bound and wants more resident gates (one gadget row per step, 4 gates per
// CTA); the two-prime engine is latency bound and wants independent work per
// thread (two rows per step) and resident warps (3 gates per CTA: 158
// registers, one exchange buffer per gate so that 3 fit in shared memory).
// Batches smaller than two gates per SM always use one gate per CTA.
static cudaError_t launch_br_any(Ctx& c, const GateDesc* d_desc, size_t count, uint32_t* d_big, cudaStream_t st) {
  const int n = static_cast<int>(c.p.n), bg = static_cast<int>(c.p.bg_bits);
  const bool small = count < static_cast<size_t>(2 * c.sm_count);
  const BrShape sh = kBrShapes[c.br_shape];
  if (c.engine == FSQL_ENGINE_GOLDILOCKS) {
    using F = dev::Goldilocks;
    if (small || sh.gates == 1)
      return launch_br_engine<F, 1, 1>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
    if (sh.gates == 2)
      return launch_br_engine<F, 2, 1>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
    return launch_br_engine<F, 4, 1>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
  }
  using F = dev::DualPrime;
  if (small && c.latency_mode == 2) {
    // a cluster per gate while every gate gets a cluster of its own at once
    int clusters = 0;
    if (cluster_capacity(&clusters) == cudaSuccess && count <= static_cast<size_t>(clusters))
      return launch_br_cluster(count, d_desc, c.d_bks, c.d_tables_split, n, bg, d_big, st);
  }
  // Between one and two gates per SM the one-gate-per-CTA latency kernel
  // needs two waves (4.6 ms each), and the three-gate CTAs of the large-batch
  // shapes run their SMs three gates deep (9.2 ms); one wave of two-gate
  // CTAs takes about 7.3 ms.
  if (c.latency_mode && count > static_cast<size_t>(c.sm_count) && count <= static_cast<size_t>(2 * c.sm_count))
    return launch_br_engine<F, 2, 2>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
  if (small && c.latency_mode)
    return launch_br_latency<F>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
  if (!small && sh.kind == 1) {
    const uint32_t* k = c.d_bks;
    const void* tb = c.d_tables_split;
    if (sh.rows == 3) return launch_br_split<2, 3, 2>(c.sm_count, d_desc, count, k, tb, n, bg, d_big, st);
    if (sh.gates == 3) return launch_br_split<3, 2, 2>(c.sm_count, d_desc, count, k, tb, n, bg, d_big, st);
    if (sh.stages == 3) return launch_br_split<2, 2, 3>(c.sm_count, d_desc, count, k, tb, n, bg, d_big, st);
    return launch_br_split<2, 2, 2>(c.sm_count, d_desc, count, k, tb, n, bg, d_big, st);
  }
  if (small || sh.gates == 1)
    return launch_br_engine<F, 1, 2>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
  if (sh.kind == 2)
    return launch_br_engine<F, 3, 2, true>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
  if (sh.gates == 3)
    return launch_br_engine<F, 3, 2>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
  if (sh.gates == 4)
    return launch_br_engine<F, 4, 2>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
  return launch_br_engine<F, 2, 2>(c.sm_count, d_desc, count, c.d_bkhat, c.d_tables, n, bg, d_big, st);
}

// The device level walker over nsegs segments (cooperative launch, one CTA
// per SM), for the packed two-prime kernel with G gates per CTA.
template <int G, bool kOwn>
static cudaError_t launch_walk_engine(Ctx& c, const GateDesc* d_desc, const WalkSeg* d_segs, int nsegs,
                                      uint32_t* d_big, cudaStream_t st) {
  using F = dev::DualPrime;
  constexpr int kP = 2;
  static_assert(walk_smem<F, G, kP, kOwn>() <= 227 * 1024, "walker shared memory over budget");
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(scan_walk_kernel<F, G, kP, kOwn>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               walk_smem<F, G, kP, kOwn>());
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  cudaError_t e = cudaMemsetAsync(c.d_walk_sync, 0, sizeof(WalkSync), st);
  if (e != cudaSuccess) return e;
  int n = static_cast<int>(c.p.n), bg = static_cast<int>(c.p.bg_bits), skip = c.walk_skip_block;
  long long tmo = static_cast<long long>(c.walk_timeout_ms * 1e6);
  const uint64_t* bk = c.d_bkhat;
  const void* tb = c.d_tables;
  const uint32_t* ksk = c.d_ksk;
  WalkSync* sy = c.d_walk_sync;
  void* args[] = {&d_desc, &d_segs, &nsegs, &bk, &tb, &n, &bg, &d_big, &ksk, &sy, &tmo, &skip};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(scan_walk_kernel<F, G, kP, kOwn>),
                                     dim3(c.sm_count), dim3(G * kGroup), args, walk_smem<F, G, kP, kOwn>(), st);
}

// Whether a scan's levels can run on the device walker: the two-prime engine
// on a packed launch shape, and every segment large enough for the
// persistent multi-gate kernel (at least two gates per SM).
bool walk_supported(const Ctx& c) {
  const BrShape sh = kBrShapes[c.br_shape];
  return c.walk_mode && c.engine == FSQL_ENGINE_DUAL_PRIME &&
         ((sh.kind == 0 && (sh.gates == 2 || sh.gates == 3)) || sh.kind == 2) && c.d_walk_sync;
}

int launch_walk(Ctx& c, const GateDesc* d_desc, const WalkSeg* d_segs, int nsegs, size_t gates, uint32_t* d_big,
                void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LaunchTimer tm(c, st);
  const BrShape sh = kBrShapes[c.br_shape];
  cudaError_t e = sh.kind == 2   ? launch_walk_engine<3, true>(c, d_desc, d_segs, nsegs, d_big, st)
                  : sh.gates == 2 ? launch_walk_engine<2, false>(c, d_desc, d_segs, nsegs, d_big, st)
                                  : launch_walk_engine<3, false>(c, d_desc, d_segs, nsegs, d_big, st);
  if (e != cudaSuccess) {
    set_error(std::string("walker launch: ") + cudaGetErrorString(e));
    return FSQL_ERR_CUDA;
  }
  tm.done(true, gates);  // one launch: blind rotations and keyswitches of every level
  return FSQL_OK;
}

int launch_blind_rotate(Ctx& c, const GateDesc* d_desc, size_t count, uint32_t* d_big, void* stream) {
  if (count == 0) return FSQL_OK;
  LaunchTimer tm(c, static_cast<cudaStream_t>(stream));
  CK(launch_br_any(c, d_desc, count, d_big, static_cast<cudaStream_t>(stream)));
  tm.done(true, count);
  return FSQL_OK;
}

int launch_keyswitch(Ctx& c, const uint32_t* d_big, const GateDesc* d_desc, uint32_t* d_out_contig, size_t count,
                     void* stream) {
  if (count == 0) return FSQL_OK;
  const unsigned groups = static_cast<unsigned>((count + kKsGates - 1) / kKsGates);
  LaunchTimer tm(c, static_cast<cudaStream_t>(stream));
  // splits so that a small batch still fills about two CTAs per SM
  int splits = 1;
  while (c.d_ks_part && count <= static_cast<size_t>(kKsPartGates) && splits < kKsMaxSplits &&
         groups * kKsTiles * splits < static_cast<unsigned>(2 * c.sm_count))
    splits *= 2;
  if (splits > 1) {
    keyswitch_part_kernel<<<dim3(groups, kKsTiles, splits), kKsCols, 0, static_cast<cudaStream_t>(stream)>>>(
        d_big, static_cast<int>(count), c.d_ksk, splits, c.d_ks_part);
    CK(cudaGetLastError());
    keyswitch_reduce_kernel<<<static_cast<unsigned>(count), kKsCols, 0, static_cast<cudaStream_t>(stream)>>>(
        c.d_ks_part, splits, d_big, d_desc, d_out_contig, static_cast<int>(c.p.n));
  } else {
    keyswitch_kernel<<<dim3(groups, kKsTiles), kKsCols, 0, static_cast<cudaStream_t>(stream)>>>(
        d_big, d_desc, d_out_contig, static_cast<int>(count), c.d_ksk, static_cast<int>(c.p.n));
  }
  CK(cudaGetLastError());
  tm.done(false, count);
  return FSQL_OK;
}

static int ensure_big(Ctx& c, size_t count) {
  if (count <= c.big_cap) return FSQL_OK;
  cudaFree(c.d_big);
  c.d_big = nullptr;
  c.big_cap = 0;
  CK(cudaMalloc(&c.d_big, count * (kN + 1) * 4));
  c.big_cap = count;
  return FSQL_OK;
}

static int ensure_desc(Ctx& c, size_t count) {
  if (count <= c.desc_cap) return FSQL_OK;
  cudaFree(c.d_desc);
  c.d_desc = nullptr;
  c.desc_cap = 0;
  CK(cudaMalloc(&c.d_desc, count * sizeof(GateDesc)));
  c.desc_cap = count;
  return FSQL_OK;
}

// Largest number of gates one blind-rotation launch takes (bounds the
// extracted-sample scratch to 1 GiB).
constexpr size_t kMaxChunk = 1u << 18;

int launch_gates(Ctx& c, const GateDesc* d_desc, size_t count, uint32_t* d_big, void* stream) {
  for (size_t off = 0; off < count; off += kMaxChunk) {
    const size_t cnt = std::min(kMaxChunk, count - off);
    int rc = launch_blind_rotate(c, d_desc + off, cnt, d_big, stream);
    if (rc) return rc;
    rc = launch_keyswitch(c, d_big, d_desc + off, nullptr, cnt, stream);
    if (rc) return rc;
  }
  return FSQL_OK;
}

// Scratch of the keyswitch-first order for up to `count` gates per launch:
// the keyswitched samples, their blind-rotation descriptors (built once for
// the whole capacity) and the trivial true ciphertext.
static int ensure_ks_first(Ctx& c, size_t count) {
  if (count <= c.ks_small_cap) return FSQL_OK;
  cudaFree(c.d_ks_small);
  cudaFree(c.d_ks_desc);
  c.d_ks_small = nullptr;
  c.d_ks_desc = nullptr;
  c.ks_small_cap = 0;
  const size_t words = c.p.n + 1;
  CK(cudaMalloc(&c.d_ks_small, count * words * 4));
  CK(cudaMalloc(&c.d_ks_desc, count * sizeof(GateDesc)));
  if (!c.d_true) {
    CK(cudaMalloc(&c.d_true, words * 4));
    std::vector<uint32_t> t(words, 0u);
    t[words - 1] = 1u << 29;
    CK(cudaMemcpy(c.d_true, t.data(), words * 4, cudaMemcpyHostToDevice));
  }
  identity_desc_kernel<<<static_cast<unsigned>((count + 255) / 256), 256>>>(c.d_ks_desc, static_cast<int>(count),
                                                                            c.d_ks_small, c.d_true,
                                                                            static_cast<int>(words));
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  c.ks_small_cap = count;
  ++c.ks_gen;  // a captured graph holds the old addresses of all three buffers
  return FSQL_OK;
}

// Gates in keyswitch-first order: inputs and outputs N + 1 words.  Per chunk:
// lincomb + keyswitch, bootstrap of the keyswitched samples, copy of the
// extracted samples to the outputs.  ensure_ks_first and ensure_big must
// cover min(count, kMaxChunk) gates.
int launch_gates_ks_first(Ctx& c, const GateDesc* d_desc, size_t count, uint32_t* d_big, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (size_t off = 0; off < count; off += kMaxChunk) {
    const size_t cnt = std::min(kMaxChunk, count - off);
    if (cnt > c.ks_small_cap) {
      set_error("keyswitch-first scratch too small");
      return FSQL_ERR_ARG;
    }
    {
      LaunchTimer tm(c, st);
      keyswitch_lincomb_kernel<<<dim3(static_cast<unsigned>((cnt + kKsGates - 1) / kKsGates), kKsTiles), kKsCols, 0,
                                 st>>>(d_desc + off, static_cast<int>(cnt), c.d_ksk, static_cast<int>(c.p.n),
                                       c.d_ks_small);
      CK(cudaGetLastError());
      tm.done(false, cnt);
    }
    int rc = launch_blind_rotate(c, c.d_ks_desc, cnt, d_big, stream);
    if (rc) return rc;
    copy_out_kernel<<<static_cast<unsigned>(std::min<size_t>(cnt, 16 * static_cast<size_t>(c.sm_count))), 256, 0,
                      st>>>(d_desc + off, d_big, static_cast<int>(cnt));
    CK(cudaGetLastError());
  }
  return FSQL_OK;
}

}  // namespace fsql

// ------------------------------------------------------------------ no-allocation gate path
// Scratch of fsql_gate_batch_noalloc: the extracted samples between the
// blind-rotation and keyswitch kernels and the gate descriptors, for at most
// kNoAllocMaxGates gates.  These arrays live in the library's device image,
// so every GPU that loads the library holds them (4.0 MiB + 40 KiB) until the
// process exits, and every call of the entry point on that GPU reuses them.
namespace fsql {
constexpr size_t kNoAllocMaxGates = 1024;
static __device__ __align__(256) uint32_t g_noalloc_big[kNoAllocMaxGates * (kN + 1)];
static __device__ __align__(256) GateDesc g_noalloc_desc[kNoAllocMaxGates];

// Device addresses of the two arrays, looked up once per device.  In host
// code the array names are host-side stand-ins, not device addresses, so
// kernels only ever receive the addresses cudaGetSymbolAddress returns.
struct NoAllocScratch {
  uint32_t* big = nullptr;
  GateDesc* desc = nullptr;
  bool ready = false;
};
static NoAllocScratch g_noalloc[64];
static std::mutex g_noalloc_mu;

static int noalloc_setup(int device, NoAllocScratch* out) {
  if (device < 0 || device >= 64) {
    set_error("device ordinal out of range for the no-allocation gate path");
    return FSQL_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocScratch& s = g_noalloc[device];
  if (!s.ready) {
    void* big = nullptr;
    void* desc = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&big, g_noalloc_big);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&desc, g_noalloc_desc);
    if (e != cudaSuccess) {
      set_error(std::string("cudaGetSymbolAddress of the no-allocation scratch: ") + cudaGetErrorString(e));
      return FSQL_ERR_CUDA;
    }
    s.big = static_cast<uint32_t*>(big);
    s.desc = static_cast<GateDesc*>(desc);
    s.ready = true;
  }
  *out = s;
  return FSQL_OK;
}
}  // namespace fsql

using fsql::Ctx;
using fsql::GateDesc;

namespace {

int arg_error(const char* msg) {
  fsql::set_error(msg);
  return FSQL_ERR_ARG;
}

Ctx* device_ctx(fsql_ctx* ctx) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) {
    fsql::set_error("null context");
    return nullptr;
  }
  if (c->device < 0 || !c->d_bkhat) {
    fsql::set_error("context has no device keys (created with device = -1)");
    return nullptr;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) {
    fsql::set_error("cudaSetDevice failed");
    return nullptr;
  }
  return c;
}

int check_types_host(size_t count) { return count > (size_t(1) << 31) ? arg_error("too many gates") : FSQL_OK; }

// Build (or reuse) the descriptor plan of a scan and upload it to c.d_desc
// (and the outputs no gate writes to c.d_lits).  plain: the constants are the
// plaintext values k0 (and k1), d_const is unused.
int prepare_scan(Ctx& c, const uint32_t* d_column, size_t rows, uint32_t width, uint32_t pred,
                 const uint32_t* d_const, uint32_t n_payloads, const uint32_t* const* d_payloads,
                 uint32_t payload_width, uint32_t* d_match, uint32_t* const* d_out_payloads, void* stream,
                 bool plain = false, uint64_t k0 = 0, uint64_t k1 = 0, bool ks_first = false) {
  fsql::Netlist nl;
  const bool ok = plain ? fsql::build_netlist_plain(pred, width, n_payloads, payload_width, k0, k1, &nl)
                        : fsql::build_netlist(pred, width, n_payloads, payload_width, &nl);
  if (!ok) return arg_error("bad predicate shape");
  const size_t W = ks_first ? static_cast<size_t>(c.p.N) + 1 : c.p.n + 1;
  const int G = static_cast<int>(nl.type.size());
  const long n_int = fsql::scan_internal_wires(nl);
  const size_t wire_words = rows * static_cast<size_t>(n_int) * W;
  if (wire_words > c.wires_cap) {
    cudaFree(c.d_wires);
    c.d_wires = nullptr;
    c.wires_cap = 0;
    if (cudaMalloc(&c.d_wires, wire_words * 4) != cudaSuccess) {
      fsql::set_error("scan scratch allocation failed");
      return FSQL_ERR_OOM;
    }
    c.wires_cap = wire_words;
    delete c.plan;
    c.plan = nullptr;
  }

  fsql::Plan* pl = c.plan;
  bool same = pl && pl->column == d_column && pl->rows == rows && pl->width == width && pl->pred == pred &&
              pl->n_payloads == n_payloads && pl->payload_width == payload_width && pl->cst == d_const &&
              pl->match == d_match && pl->wires == c.d_wires && pl->plain == plain && pl->k0 == k0 && pl->k1 == k1 && pl->ks_first == ks_first;
  for (uint32_t q = 0; same && q < n_payloads; ++q)
    same = pl->payloads[q] == d_payloads[q] && pl->outs[q] == d_out_payloads[q];
  if (same) return FSQL_OK;

  delete c.plan;
  c.plan = nullptr;
  pl = new fsql::Plan();
  pl->column = d_column;
  pl->rows = rows;
  pl->width = width;
  pl->pred = pred;
  pl->n_payloads = n_payloads;
  pl->payload_width = payload_width;
  pl->cst = d_const;
  pl->payloads.assign(d_payloads, d_payloads + n_payloads);
  pl->match = d_match;
  pl->outs.assign(d_out_payloads, d_out_payloads + n_payloads);
  pl->wires = c.d_wires;
  pl->plain = plain;
  pl->k0 = k0;
  pl->k1 = k1;
  pl->ks_first = ks_first;

  const size_t total = rows * static_cast<size_t>(G);
  fsql::ScanIO io;
  io.column = d_column;
  io.rows = rows;
  io.width = width;
  io.pred = pred;
  io.cst = d_const;
  io.n_payloads = n_payloads;
  io.payloads = d_payloads;
  io.payload_width = payload_width;
  io.match = d_match;
  io.outs = d_out_payloads;
  io.wires = c.d_wires;
  io.words = W;
  // the scan program (netlist + pointers, a few KB): descriptors are
  // generated from it on the device
  std::vector<uint8_t> prog;
  if (!fsql::build_scan_program(nl, io, &prog, &pl->level_offset)) {
    delete pl;
    return arg_error("too many payload columns for a scan program");
  }
  pl->total = pl->level_offset.back();
  if (prog.size() > c.prog_cap) {
    cudaFree(c.d_prog);
    c.d_prog = nullptr;
    c.prog_cap = 0;
    if (cudaMalloc(&c.d_prog, prog.size()) != cudaSuccess) {
      fsql::set_error("scan program allocation failed");
      delete pl;
      return FSQL_ERR_OOM;
    }
    c.prog_cap = prog.size();
  }
  int rc = fsql::ensure_desc(c, total);
  if (rc) {
    delete pl;
    return rc;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<fsql::OutDesc> lits;
  fsql::scan_literals(nl, io, &lits);
  pl->n_lits = lits.size();
  if (!lits.empty()) {
    if (lits.size() > c.lits_cap) {
      cudaFree(c.d_lits);
      c.d_lits = nullptr;
      c.lits_cap = 0;
      if (cudaMalloc(&c.d_lits, lits.size() * sizeof(fsql::OutDesc)) != cudaSuccess) {
        fsql::set_error("scan literal descriptor allocation failed");
        delete pl;
        return FSQL_ERR_OOM;
      }
      c.lits_cap = lits.size();
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(c.d_lits, lits.data(), lits.size() * sizeof(fsql::OutDesc), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      fsql::set_error("literal descriptor upload failed");
      delete pl;
      return FSQL_ERR_CUDA;
    }
  }
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  if (cudaMemcpyAsync(c.d_prog, prog.data(), prog.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      fsql::launch_gen_desc(c.d_prog, c.d_desc, total, st) != FSQL_OK) {
    fsql::set_error("scan program upload or descriptor generation failed");
    delete pl;
    return FSQL_ERR_CUDA;
  }
  c.plan = pl;
  return FSQL_OK;
}

enum { kAggSum = 0, kAggMax = 1, kAggMin = 2 };

// Build (or reuse) the aggregation plan (SUM, MAX or MIN) for these
// arguments: the circuit's descriptors, output descriptors and intermediate
// wires live in buffers the plan owns.  d_match: MIN's match bits.
int prepare_aggregate(Ctx& c, int kind, const uint32_t* d_in, const uint32_t* d_match, size_t rows, uint32_t width,
                      uint32_t out_width, uint32_t* d_out, void* stream) {
  fsql::Plan* pl = c.agg_plan;
  if (pl && pl->agg_kind == kind && pl->agg_in == d_in && pl->agg_match == d_match && pl->rows == rows &&
      pl->agg_width == width && pl->agg_out_width == out_width && pl->agg_out == d_out)
    return FSQL_OK;
  delete c.agg_plan;
  c.agg_plan = nullptr;
  fsql::Netlist nl;
  const bool ok = kind == kAggSum ? fsql::build_sum_netlist(rows, width, out_width, &nl)
                                  : fsql::build_extreme_netlist(kind == kAggMin, rows, width, &nl);
  if (!ok) return arg_error("bad aggregation shape");
  const size_t W = c.p.n + 1, G = nl.type.size();
  const int value_wires = static_cast<int>(rows * width);
  pl = new fsql::Plan();
  pl->agg_kind = kind;
  pl->agg_in = d_in;
  pl->agg_match = d_match;
  pl->rows = rows;
  pl->agg_width = width;
  pl->agg_out_width = out_width;
  pl->agg_out = d_out;
  if ((G && (cudaMalloc(&pl->own_desc, G * sizeof(fsql::GateDesc)) != cudaSuccess ||
             cudaMalloc(&pl->own_wires, G * W * 4) != cudaSuccess)) ||
      cudaMalloc(&pl->own_lits, nl.literal_outs.size() * sizeof(fsql::OutDesc)) != cudaSuccess) {
    delete pl;
    fsql::set_error("aggregation scratch allocation failed");
    return FSQL_ERR_OOM;
  }
  auto wire_ptr = [&](int id) -> const uint32_t* {
    if (id < value_wires) return d_in + static_cast<size_t>(id) * W;  // value bit (r, j) = r * width + j
    if (id < nl.n_inputs) return d_match + static_cast<size_t>(id - value_wires) * W;  // MIN: match bit of row r
    return pl->own_wires + static_cast<size_t>(id - nl.n_inputs) * W;
  };
  std::vector<fsql::GateDesc> desc(G);
  pl->level_offset.assign(nl.levels + 1, 0);
  size_t pos = 0;
  for (int L = 1; L <= nl.levels; ++L) {
    pl->level_offset[L - 1] = pos;
    for (size_t g = 0; g < G; ++g) {
      if (nl.level[g] != L) continue;
      fsql::GateDesc& d = desc[pos++];
      d.a = wire_ptr(nl.a[g]);
      d.b = wire_ptr(nl.b[g]);
      d.c = nl.c[g] >= 0 ? wire_ptr(nl.c[g]) : nullptr;
      d.out = pl->own_wires + g * W;
      d.type = static_cast<uint32_t>(nl.type[g]);
      d.pad = 0;
    }
  }
  pl->level_offset[nl.levels] = pos;
  pl->total = pos;
  std::vector<fsql::OutDesc> lits;
  for (const auto& l : nl.literal_outs) {
    fsql::OutDesc d;
    d.src = l.wire >= 0 ? wire_ptr(l.wire) : nullptr;
    d.dst = d_out + static_cast<size_t>(l.target) * W;
    d.mode = l.mode;
    d.pad = 0;
    lits.push_back(d);
  }
  pl->n_lits = lits.size();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // pageable sources: each copy is staged before cudaMemcpyAsync returns
  if ((G && cudaMemcpyAsync(pl->own_desc, desc.data(), G * sizeof(fsql::GateDesc), cudaMemcpyHostToDevice, st) !=
                cudaSuccess) ||
      cudaMemcpyAsync(pl->own_lits, lits.data(), lits.size() * sizeof(fsql::OutDesc), cudaMemcpyHostToDevice, st) !=
          cudaSuccess) {
    delete pl;
    fsql::set_error("aggregation descriptor upload failed");
    return FSQL_ERR_CUDA;
  }
  c.agg_plan = pl;
  return FSQL_OK;
}

int validate_scan(Ctx* c, const uint32_t* column, size_t rows, uint32_t width, uint32_t pred, const uint32_t* cst,
                  uint32_t n_payloads, const uint32_t* const* payloads, uint32_t payload_width, uint32_t* match,
                  uint32_t* const* outs) {
  if (rows == 0) return FSQL_OK;
  if (!column || !cst || !match) return arg_error("null column, constant or match pointer");
  if (width < 1 || width > 64) return arg_error("width must be in [1, 64]");
  if (pred > FSQL_RANGE_MAJ) return arg_error("unknown predicate");
  if (n_payloads > 64 || (n_payloads && (!payloads || !outs || payload_width < 1 || payload_width > 64)))
    return arg_error("bad payload arguments");
  for (uint32_t q = 0; q < n_payloads; ++q)
    if (!payloads[q] || !outs[q]) return arg_error("null payload pointer");
  if (rows > (size_t(1) << 26)) return arg_error("too many rows");
  (void)c;
  return FSQL_OK;
}

// Run the prepared plan: every level's gates (batched, or one gate per
// launch), then the outputs no gate writes.  The batched sequence is
// captured once per plan as a CUDA graph on the context's capture stream and
// replayed on the caller's stream.  Called with c->mu held.
int execute_plan(Ctx* c, fsql::Plan& pl, const fsql::GateDesc* d_desc, const fsql::OutDesc* d_lits, int per_gate,
                 void* stream) {
  const int n = static_cast<int>(c->p.n);
  size_t widest = 0;
  for (size_t L = 0; L + 1 < pl.level_offset.size(); ++L)
    widest = std::max(widest, pl.level_offset[L + 1] - pl.level_offset[L]);
  const size_t chunk = per_gate ? 1 : std::min(widest, fsql::kMaxChunk);
  int rc = fsql::ensure_big(*c, chunk);
  if (!rc && pl.ks_first) rc = fsql::ensure_ks_first(*c, chunk);
  if (rc) return rc;
  auto gates = [&](const fsql::GateDesc* dd, size_t cnt, void* st) -> int {
    return pl.ks_first ? fsql::launch_gates_ks_first(*c, dd, cnt, c->d_big, st)
                       : fsql::launch_gates(*c, dd, cnt, c->d_big, st);
  };
  if (per_gate) {
    for (size_t g = 0; g < pl.total; ++g) {
      rc = gates(d_desc + g, 1, stream);
      if (rc) return rc;
    }
    return fsql::launch_literals(d_lits, pl.n_lits, n, stream);
  }
  // the device walker (one launch for all levels) when the context asks for
  // it and every segment keeps the persistent kernel busy
  bool walk = !pl.ks_first && fsql::walk_supported(*c);
  for (size_t L = 0; walk && L + 1 < pl.level_offset.size(); ++L)
    if (pl.level_offset[L + 1] - pl.level_offset[L] < static_cast<size_t>(2 * c->sm_count)) walk = false;
  // the walker's kernel arguments a captured graph holds (0: no walker)
  const long long walk_key =
      walk ? static_cast<long long>(c->walk_timeout_ms * 1e3) * 4099 + c->walk_skip_block + 2 : 0;
  if (walk && (pl.nsegs == 0 || pl.segs_chunk != chunk)) {
    std::vector<fsql::WalkSeg> segs;
    for (size_t L = 0; L + 1 < pl.level_offset.size(); ++L)
      for (size_t b = pl.level_offset[L]; b < pl.level_offset[L + 1]; b += chunk)
        segs.push_back({static_cast<uint32_t>(b), static_cast<uint32_t>(std::min(chunk, pl.level_offset[L + 1] - b))});
    cudaFree(pl.d_segs);
    pl.d_segs = nullptr;
    pl.nsegs = 0;
    if (cudaMalloc(&pl.d_segs, segs.size() * sizeof(fsql::WalkSeg)) != cudaSuccess ||
        cudaMemcpy(pl.d_segs, segs.data(), segs.size() * sizeof(fsql::WalkSeg), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      fsql::set_error("walker segment upload failed");
      return FSQL_ERR_CUDA;
    }
    pl.nsegs = static_cast<int>(segs.size());
    pl.segs_chunk = chunk;
  }
  auto launch_all = [&](void* st) -> int {
    if (walk) {
      const int r = fsql::launch_walk(*c, d_desc, pl.d_segs, pl.nsegs, pl.total, c->d_big, st);
      if (r) return r;
      return fsql::launch_literals(d_lits, pl.n_lits, n, st);
    }
    for (size_t L = 0; L + 1 < pl.level_offset.size(); ++L) {
      const int r = gates(d_desc + pl.level_offset[L], pl.level_offset[L + 1] - pl.level_offset[L], st);
      if (r) return r;
    }
    return fsql::launch_literals(d_lits, pl.n_lits, n, st);
  };
  const auto* prof = static_cast<const fsql::Profile*>(c->prof);
  if (prof && prof->recording) return launch_all(stream);  // per-launch events need plain launches
  fsql::Plan& mp = pl;
  if (!mp.graph || mp.graph_desc != d_desc || mp.graph_big != c->d_big || mp.graph_lits != d_lits ||
      mp.graph_br_shape != 4 * c->br_shape + c->latency_mode ||
      (pl.ks_first && mp.graph_ks_gen != c->ks_gen) || mp.graph_walk != walk_key) {
    if (mp.graph) cudaGraphExecDestroy(mp.graph);
    mp.graph = nullptr;
    cudaStream_t cs = static_cast<cudaStream_t>(c->capture_stream);
    if (!cs) {
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return launch_all(stream);
      c->capture_stream = cs;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return launch_all(stream);
    rc = launch_all(cs);
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (rc || ec != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc ? rc : launch_all(stream);
    }
    const cudaError_t ei = cudaGraphInstantiate(&mp.graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      mp.graph = nullptr;
      cudaGetLastError();
      return launch_all(stream);
    }
    mp.graph_desc = d_desc;
    mp.graph_big = c->d_big;
    mp.graph_lits = d_lits;
    mp.graph_br_shape = 4 * c->br_shape + c->latency_mode;
    mp.graph_ks_gen = c->ks_gen;
    mp.graph_walk = walk_key;
  }
  if (cudaGraphLaunch(mp.graph, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    fsql::set_error("scan graph launch failed");
    return FSQL_ERR_CUDA;
  }
  return FSQL_OK;
}

}  // namespace

extern "C" {

int fsql_gate_batch(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a, const uint32_t* d_b,
                    uint32_t* d_out, size_t count, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (count == 0) return FSQL_OK;
  if (!d_types || !d_a || !d_b || !d_out) return arg_error("null device pointer");
  if (int rc = check_types_host(count)) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = fsql::ensure_desc(*c, count);
  if (!rc) rc = fsql::ensure_big(*c, std::min(count, fsql::kMaxChunk));
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fsql::make_desc_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(
      c->d_desc, d_types, d_a, d_b, d_out, static_cast<int>(count), static_cast<int>(c->p.n + 1));
  if (cudaGetLastError() != cudaSuccess) return arg_error("descriptor kernel launch failed");
  delete c->plan;  // descriptors overwritten
  c->plan = nullptr;
  return fsql::launch_gates(*c, c->d_desc, count, c->d_big, stream);
}

int fsql_blind_rotate_extract(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a, const uint32_t* d_b,
                              uint32_t* d_big, size_t count, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (count == 0) return FSQL_OK;
  if (!d_types || !d_a || !d_b || !d_big) return arg_error("null device pointer");
  if (int rc = check_types_host(count)) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = fsql::ensure_desc(*c, count);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fsql::make_desc_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(
      c->d_desc, d_types, d_a, d_b, nullptr, static_cast<int>(count), static_cast<int>(c->p.n + 1));
  if (cudaGetLastError() != cudaSuccess) return arg_error("descriptor kernel launch failed");
  delete c->plan;
  c->plan = nullptr;
  for (size_t off = 0; off < count; off += fsql::kMaxChunk) {
    const size_t cnt = std::min(fsql::kMaxChunk, count - off);
    rc = fsql::launch_blind_rotate(*c, c->d_desc + off, cnt, d_big + off * (fsql::kN + 1), stream);
    if (rc) return rc;
  }
  return FSQL_OK;
}

int fsql_keyswitch(fsql_ctx* ctx, const uint32_t* d_big, uint32_t* d_out, size_t count, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (count == 0) return FSQL_OK;
  if (!d_big || !d_out) return arg_error("null device pointer");
  if (int rc = check_types_host(count)) return rc;
  return fsql::launch_keyswitch(*c, d_big, nullptr, d_out, count, stream);
}

int fsql_debug_ntt_mul(fsql_ctx* ctx, const int32_t* d_digits, const uint32_t* d_poly, uint32_t* d_out,
                       void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (!d_digits || !d_poly || !d_out) return arg_error("null device pointer");
  if (c->engine == FSQL_ENGINE_GOLDILOCKS)
    fsql::ntt_mul_kernel<fsql::dev::Goldilocks>
        <<<1, fsql::kGroup, 0, static_cast<cudaStream_t>(stream)>>>(d_digits, d_poly, d_out, c->d_tables);
  else
    fsql::ntt_mul_kernel<fsql::dev::DualPrime>
        <<<1, fsql::kGroup, 0, static_cast<cudaStream_t>(stream)>>>(d_digits, d_poly, d_out, c->d_tables);
  if (cudaGetLastError() != cudaSuccess) return arg_error("ntt test kernel launch failed");
  return FSQL_OK;
}

int fsql_scan_select(fsql_ctx* ctx, const uint32_t* d_column, size_t rows, uint32_t width, uint32_t pred,
                     const uint32_t* d_const, uint32_t n_payloads, const uint32_t* const* d_payloads,
                     uint32_t payload_width, uint32_t* d_match, uint32_t* const* d_out_payloads, int per_gate,
                     void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (int rc = validate_scan(c, d_column, rows, width, pred, d_const, n_payloads, d_payloads, payload_width,
                             d_match, d_out_payloads))
    return rc;
  if (rows == 0) return FSQL_OK;
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = prepare_scan(*c, d_column, rows, width, pred, d_const, n_payloads, d_payloads, payload_width, d_match,
                        d_out_payloads, stream);
  if (rc) return rc;
  return execute_plan(c, *c->plan, c->d_desc, c->d_lits, per_gate, stream);
}

int fsql_aggregate_sum(fsql_ctx* ctx, const uint32_t* d_values, size_t rows, uint32_t width, uint32_t out_width,
                       uint32_t* d_out, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if ((rows && !d_values) || !d_out) return arg_error("null values or output pointer");
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = prepare_aggregate(*c, kAggSum, d_values, nullptr, rows, width, out_width, d_out, stream);
  if (rc) return rc;
  return execute_plan(c, *c->agg_plan, c->agg_plan->own_desc, c->agg_plan->own_lits, 0, stream);
}

int fsql_aggregate_max(fsql_ctx* ctx, const uint32_t* d_values, size_t rows, uint32_t width, uint32_t* d_out,
                       void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if ((rows && !d_values) || !d_out) return arg_error("null values or output pointer");
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = prepare_aggregate(*c, kAggMax, d_values, nullptr, rows, width, width, d_out, stream);
  if (rc) return rc;
  return execute_plan(c, *c->agg_plan, c->agg_plan->own_desc, c->agg_plan->own_lits, 0, stream);
}

int fsql_aggregate_min(fsql_ctx* ctx, const uint32_t* d_values, const uint32_t* d_match, size_t rows,
                       uint32_t width, uint32_t* d_out, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if ((rows && (!d_values || !d_match)) || !d_out) return arg_error("null values, match or output pointer");
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = prepare_aggregate(*c, kAggMin, d_values, d_match, rows, width, width, d_out, stream);
  if (rc) return rc;
  return execute_plan(c, *c->agg_plan, c->agg_plan->own_desc, c->agg_plan->own_lits, 0, stream);
}

int fsql_scan_select_ks_first(fsql_ctx* ctx, const uint32_t* d_column, size_t rows, uint32_t width, uint32_t pred,
                              const uint32_t* d_const, uint32_t n_payloads, const uint32_t* const* d_payloads,
                              uint32_t payload_width, uint32_t* d_match, uint32_t* const* d_out_payloads,
                              int per_gate, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (int rc = validate_scan(c, d_column, rows, width, pred, d_const, n_payloads, d_payloads, payload_width,
                             d_match, d_out_payloads))
    return rc;
  if (rows == 0) return FSQL_OK;
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = prepare_scan(*c, d_column, rows, width, pred, d_const, n_payloads, d_payloads, payload_width, d_match,
                        d_out_payloads, stream, false, 0, 0, true);
  if (rc) return rc;
  return execute_plan(c, *c->plan, c->d_desc, c->d_lits, per_gate, stream);
}

int fsql_gate_batch_ks_first(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a, const uint32_t* d_b,
                             uint32_t* d_out, size_t count, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (count == 0) return FSQL_OK;
  if (!d_types || !d_a || !d_b || !d_out) return arg_error("null device pointer");
  if (int rc = check_types_host(count)) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  const size_t chunk = std::min(count, fsql::kMaxChunk);
  int rc = fsql::ensure_desc(*c, count);
  if (!rc) rc = fsql::ensure_big(*c, chunk);
  if (!rc) rc = fsql::ensure_ks_first(*c, chunk);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fsql::make_desc_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(
      c->d_desc, d_types, d_a, d_b, d_out, static_cast<int>(count), static_cast<int>(c->p.N + 1));
  if (cudaGetLastError() != cudaSuccess) return arg_error("descriptor kernel launch failed");
  delete c->plan;  // descriptors overwritten
  c->plan = nullptr;
  return fsql::launch_gates_ks_first(*c, c->d_desc, count, c->d_big, stream);
}

int fsql_scan_select_plain(fsql_ctx* ctx, const uint32_t* d_column, size_t rows, uint32_t width, uint32_t pred,
                           const uint64_t* consts, uint32_t n_payloads, const uint32_t* const* d_payloads,
                           uint32_t payload_width, uint32_t* d_match, uint32_t* const* d_out_payloads, int per_gate,
                           void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (!consts) return arg_error("null constants");
  // the constant pointer is host memory here; only its presence is checked by validate_scan
  if (int rc = validate_scan(c, d_column, rows, width, pred, d_column, n_payloads, d_payloads, payload_width,
                             d_match, d_out_payloads))
    return rc;
  const bool range = pred == FSQL_RANGE || pred == FSQL_RANGE_MAJ;
  const uint64_t k0 = consts[0], k1 = range ? consts[1] : 0;
  if (width < 64 && (k0 >> width || k1 >> width)) return arg_error("constant wider than the column");
  if (rows == 0) return FSQL_OK;
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = prepare_scan(*c, d_column, rows, width, pred, nullptr, n_payloads, d_payloads, payload_width, d_match,
                        d_out_payloads, stream, true, k0, k1);
  if (rc) return rc;
  return execute_plan(c, *c->plan, c->d_desc, c->d_lits, per_gate, stream);
}

int fsql_scan_select_host(fsql_ctx* ctx, const uint32_t* h_column, size_t rows, uint32_t width, uint32_t pred,
                          const uint32_t* h_const, uint32_t n_payloads, const uint32_t* const* h_payloads,
                          uint32_t payload_width, uint32_t* h_match, uint32_t* const* h_out_payloads, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (int rc = validate_scan(c, h_column, rows, width, pred, h_const, n_payloads, h_payloads, payload_width,
                             h_match, h_out_payloads))
    return rc;
  if (rows == 0) return FSQL_OK;
  const size_t W = c->p.n + 1;
  const size_t col_w = rows * width * W;
  const size_t cst_w = ((pred == FSQL_RANGE || pred == FSQL_RANGE_MAJ) ? 2 : 1) * static_cast<size_t>(width) * W;
  const size_t pay_w = rows * static_cast<size_t>(payload_width) * W;
  const size_t total = col_w + cst_w + 2 * n_payloads * pay_w + rows * W;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (total > c->stage_cap) {
      cudaFree(c->d_stage);
      c->d_stage = nullptr;
      c->stage_cap = 0;
      if (cudaMalloc(&c->d_stage, total * 4) != cudaSuccess) {
        fsql::set_error("device staging allocation failed");
        return FSQL_ERR_OOM;
      }
      c->stage_cap = total;
    }
  }
  uint32_t* d_col = c->d_stage;
  uint32_t* d_cst = d_col + col_w;
  uint32_t* d_match = d_cst + cst_w;
  std::vector<const uint32_t*> d_pay(n_payloads);
  std::vector<uint32_t*> d_out(n_payloads);
  uint32_t* q = d_match + rows * W;
  for (uint32_t k = 0; k < n_payloads; ++k) {
    d_pay[k] = q;
    q += pay_w;
    d_out[k] = q;
    q += pay_w;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto h2d = [&](void* dst, const void* src, size_t words) {
    return cudaMemcpyAsync(dst, src, words * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = h2d(d_col, h_column, col_w) && h2d(d_cst, h_const, cst_w);
  for (uint32_t k = 0; ok && k < n_payloads; ++k) ok = h2d(const_cast<uint32_t*>(d_pay[k]), h_payloads[k], pay_w);
  if (!ok) {
    fsql::set_error("host to device copy failed");
    return FSQL_ERR_CUDA;
  }
  int rc = fsql_scan_select(ctx, d_col, rows, width, pred, d_cst, n_payloads, d_pay.data(), payload_width, d_match,
                            d_out.data(), 0, stream);
  if (rc) return rc;
  ok = cudaMemcpyAsync(h_match, d_match, rows * W * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  for (uint32_t k = 0; ok && k < n_payloads; ++k)
    ok = cudaMemcpyAsync(h_out_payloads[k], d_out[k], pay_w * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (!ok || cudaStreamSynchronize(st) != cudaSuccess) {
    fsql::set_error(std::string("device to host copy or scan failed: ") + cudaGetErrorString(cudaGetLastError()));
    return FSQL_ERR_CUDA;
  }
  return FSQL_OK;
}

int fsql_ctx_set_walk(fsql_ctx* ctx, int on, double timeout_ms) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (!(timeout_ms > 0.0) || timeout_ms > 600000.0) return arg_error("walker timeout must be in (0, 600000] ms");
  std::lock_guard<std::mutex> lk(c->mu);
  c->walk_mode = on != 0;
  c->walk_timeout_ms = timeout_ms;
  return FSQL_OK;
}

int fsql_debug_walk_skip_block(fsql_ctx* ctx, int block) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->walk_skip_block = block < 0 ? -1 : block;
  return FSQL_OK;
}

int fsql_walk_status(fsql_ctx* ctx, void* stream, unsigned int* barrier) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (barrier) *barrier = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fsql::WalkSync h{};
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(&h, c->d_walk_sync, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
    fsql::set_error(std::string("walker status: ") + cudaGetErrorString(cudaGetLastError()));
    return FSQL_ERR_CUDA;
  }
  if (h.error) {
    if (barrier) *barrier = h.barrier;
    fsql::set_error("a grid-barrier wait of the level walker ran out of time (barrier " + std::to_string(h.barrier) +
                    "); the scan's outputs are incomplete");
    return FSQL_ERR_TIMEOUT;
  }
  return FSQL_OK;
}

int fsql_profile_begin(fsql_ctx* ctx) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  auto* p = static_cast<fsql::Profile*>(c->prof);
  if (!p) c->prof = p = new fsql::Profile();
  p->used = 0;
  p->br.clear();
  p->ks.clear();
  p->gates = 0;
  p->recording = true;
  return FSQL_OK;
}

int fsql_profile_end(fsql_ctx* ctx, fsql_kernel_times* out) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (!out) return arg_error("null output");
  std::lock_guard<std::mutex> lk(c->mu);
  auto* p = static_cast<fsql::Profile*>(c->prof);
  *out = fsql_kernel_times{0.0, 0.0, 0, 0, 0};
  if (!p) return FSQL_OK;
  auto sum = [&](const std::vector<std::pair<int, int>>& v, double* ms) -> bool {
    for (auto& ab : v) {
      if (cudaEventSynchronize(p->pool[ab.second]) != cudaSuccess) return false;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p->pool[ab.first], p->pool[ab.second]) != cudaSuccess) return false;
      *ms += t;
    }
    return true;
  };
  const bool ok = sum(p->br, &out->blind_rotate_ms) && sum(p->ks, &out->keyswitch_ms);
  out->blind_rotate_launches = p->br.size();
  out->keyswitch_launches = p->ks.size();
  out->gates = p->gates;
  p->recording = false;  // keep the event pool for the next session
  p->used = 0;
  p->br.clear();
  p->ks.clear();
  if (!ok) {
    fsql::set_error("kernel timing events failed");
    return FSQL_ERR_CUDA;
  }
  return FSQL_OK;
}

int fsql_gate_batch_noalloc(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a, const uint32_t* d_b,
                            uint32_t* d_out, size_t count, void* stream) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  if (count == 0) return FSQL_OK;
  if (count > fsql::kNoAllocMaxGates) {
    fsql::set_error("fsql_gate_batch_noalloc takes at most 1024 gates per call (its scratch is a fixed array)");
    return FSQL_ERR_ARG;
  }
  if (!d_types || !d_a || !d_b || !d_out) return arg_error("null device pointer");
  fsql::NoAllocScratch scr;
  int rc = fsql::noalloc_setup(c->device, &scr);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = static_cast<int>(c->p.n);
  // Descriptors and extracted samples are fully rewritten by this call before
  // they are read, so nothing left by an earlier call needs clearing.
  fsql::make_desc_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(
      scr.desc, d_types, d_a, d_b, d_out, static_cast<int>(count), n + 1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    fsql::LaunchTimer tm(*c, st);
    e = fsql::launch_br_any(*c, scr.desc, count, scr.big, st);
    if (e == cudaSuccess) tm.done(true, count);
  }
  if (e == cudaSuccess) {
    fsql::LaunchTimer tm(*c, st);
    const dim3 grid(static_cast<unsigned>((count + fsql::kKsGates - 1) / fsql::kKsGates), fsql::kKsTiles);
    fsql::keyswitch_kernel<<<grid, fsql::kKsCols, 0, st>>>(scr.big, scr.desc, nullptr, static_cast<int>(count),
                                                               c->d_ksk, n);
    e = cudaGetLastError();
    if (e == cudaSuccess) tm.done(false, count);
  }
  if (e != cudaSuccess) {
    fsql::set_error(std::string("no-allocation gate path launch: ") + cudaGetErrorString(e));
    return FSQL_ERR_CUDA;
  }
  return FSQL_OK;
}

int fsql_autotune(fsql_ctx* ctx, size_t probe_gates, void* stream, int* best_shape, double* ms_out) {
  Ctx* c = device_ctx(ctx);
  if (!c) return FSQL_ERR_ARG;
  // default probe: 48 gates per SM, a whole number of waves for every shape
  // (1, 2, 3 or 4 gates per CTA), so no shape is favoured by its last wave
  const size_t count = probe_gates ? probe_gates : static_cast<size_t>(48 * c->sm_count);
  if (count > (size_t(1) << 20)) return arg_error("probe_gates above 2^20");
  if (count < static_cast<size_t>(2 * c->sm_count)) return arg_error("probe_gates below two gates per SM");
  const size_t words = c->p.n + 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(c->mu);
  // probe inputs: arbitrary words (the work per gate does not depend on the data)
  uint32_t* d_in = nullptr;
  uint8_t* d_types = nullptr;
  uint32_t* d_big = nullptr;
  fsql::GateDesc* d_desc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FSQL_OK;
  double ms[fsql::kBrShapeCount];
  for (double& v : ms) v = -1.0;
  const int saved = c->br_shape;
  int best = saved;
  double best_ms = 0.0;
  auto fail = [&](const char* what, cudaError_t e) {
    fsql::set_error(std::string(what) + ": " + cudaGetErrorString(e));
    rc = FSQL_ERR_CUDA;
  };
  cudaError_t e = cudaMalloc(&d_in, 2 * count * words * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d_types, count);
  if (e == cudaSuccess) e = cudaMalloc(&d_big, count * (fsql::kN + 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d_desc, count * sizeof(fsql::GateDesc));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_in, 0x5a, 2 * count * words * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_types, 1, count, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) fail("autotune set-up", e);
  if (rc == FSQL_OK) {
    fsql::make_desc_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(
        d_desc, d_types, d_in, d_in + count * words, nullptr, static_cast<int>(count), static_cast<int>(words));
    for (int si = 0; si < fsql::kBrShapeCount && rc == FSQL_OK; ++si) {
      if (!fsql::shape_offered(c->engine, si)) continue;
      c->br_shape = si;
      float t = 0.f;
      e = fsql::launch_br_any(*c, d_desc, count, d_big, st);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = fsql::launch_br_any(*c, d_desc, count, d_big, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) {
        fail("autotune probe", e);
        break;
      }
      ms[si] = t;
      if (best_ms == 0.0 || t < best_ms) {
        best_ms = t;
        best = si;
      }
    }
  }
  c->br_shape = rc == FSQL_OK ? best : saved;
  if (rc == FSQL_OK) fsql::remember_tuning(c->device, c->engine, best);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_in);
  cudaFree(d_types);
  cudaFree(d_big);
  cudaFree(d_desc);
  if (best_shape) *best_shape = c->br_shape;
  if (ms_out)
    for (int i = 0; i < fsql::kBrShapeCount; ++i) ms_out[i] = ms[i];
  return rc;
}

}  // extern "C"
