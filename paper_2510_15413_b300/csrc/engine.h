// engine.h -- internal declarations shared by the host side (host.cpp) and
// the device side (kernels.cu) of the library.  Not part of the C interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fhesql.h"

namespace fsql {

// Goldilocks prime p = 2^64 - 2^32 + 1 used by the exact NTT.
constexpr uint64_t kP = 0xFFFFFFFF00000001ull;

// Fixed shape the GPU kernels implement (checked at context creation).
constexpr int kN = 1024;     // GLWE polynomial size
constexpr int kL = 3;        // bootstrap gadget levels
constexpr int kRows = 2 * kL;  // rows of a GGSW (2 polynomials x l levels)
constexpr int kKsT = 8;      // keyswitch levels
constexpr int kKsBaseBits = 2;
constexpr int kKsDigits = (1 << kKsBaseBits) - 1;  // nonzero digit values
constexpr int kKsRowWords = 640;  // n+1 padded to a multiple of 4 words (16 B)
constexpr int kMaxN = 1024;  // largest LWE dimension the kernels take

// Launch shapes of the blind rotation for batches of at least two gates per
// SM.  kind 0: the packed kernel (each thread holds both primes' residues;
// one gadget row per step for the 64-bit prime, two for the two primes);
// kind 1: the prime-split kernel of the two-prime engine; kind 2: the packed
// kernel with one key slot per gate group (groups run unsynchronised).
// stages: slots of the key-staging ring (per group for kind 2).
struct BrShape {
  int kind, gates, rows, stages;
};
constexpr int kBrShapeCount = 9;
constexpr BrShape kBrShapes[kBrShapeCount] = {
    {0, 1, 0, 2}, {0, 2, 0, 2}, {0, 3, 0, 2}, {0, 4, 0, 2},  // packed, 1-4 gates per CTA (rows per engine)
    {1, 2, 2, 2}, {1, 2, 2, 3}, {1, 3, 2, 2}, {1, 2, 3, 2},  // prime-split
    {2, 3, 2, 1},                                            // packed, 3 gates, each group its own key slot
};
// Whether an engine offers a shape (the 64-bit prime: packed 1, 2 or 4 gates per CTA).
inline bool shape_offered(int engine, int shape) {
  if (shape < 0 || shape >= kBrShapeCount) return false;
  if (engine == FSQL_ENGINE_GOLDILOCKS) return shape == 0 || shape == 1 || shape == 3;
  return true;
}

// One bootstrapped gate: inputs a, b (and c for three-input gates, else
// null) and output pointer, all [n+1] words.
struct GateDesc {
  const uint32_t* a;
  const uint32_t* b;
  const uint32_t* c;
  uint32_t* out;
  uint32_t type;
  uint32_t pad;
};

// Twiddle tables of the 1024-point negacyclic NTT (see ntt.cuh for the
// thread layouts).  f = psi^bitrev(k), g = psi^-bitrev(k); the entry type Tw
// is the engine's twiddle form (one u64 for the 64-bit prime; for the two
// primes, each residue with its Shoup quotient: {w1, w1', w2, w2'}).
template <class Tw>
struct NttTablesT {
  Tw f_small[64];   // f[k], k < 64 (forward passes 1-2)
  Tw g_small[128];  // g[k], k < 128 (inverse passes 2-4)
  Tw f3[7][128];    // forward pass 3, per thread: f[64+h], f[128+2h+c], f[256+4h+c], h = t>>1
  Tw f4[4][128];    // forward pass 4, per thread: f[512+4t+c]
  Tw i1[7][128];    // inverse pass 1, per thread: g[512+4t+c], g[256+2t+c], g[128+t]
  uint64_t n_inv;   // key scale: N^-1 mod p (one prime), N^-1 R^2 mod p_i (two primes)
  uint64_t pad;
};

// How a scan output that no gate writes is produced (plaintext constants):
// a copy or a negation (every word negated) of an input or intermediate
// ciphertext, or the trivial ciphertext (0, .., 0, -q/8 or +q/8) of a known bit.
enum : uint32_t { kOutCopy = 0, kOutNegate = 1, kOutFalse = 2, kOutTrue = 3 };

struct OutDesc {
  const uint32_t* src;  // [n+1] words; null for kOutFalse / kOutTrue
  uint32_t* dst;        // [n+1] words
  uint32_t mode;
  uint32_t pad;
};

struct Plan;  // scan plan (kernels.cu)

// Grid-barrier state of one scan_walk_kernel launch (zeroed before it):
// CTA arrivals (barrier b completes at (b + 1) x CTAs), the error word (1: a
// barrier wait ran out of time) and the index of the barrier where it did.
struct WalkSync {
  unsigned int arrived;
  unsigned int error;
  unsigned int barrier;
  unsigned int pad;
};

struct Ctx {
  fsql_params p{};
  uint64_t seed = 0;
  int device = -1;
  int engine = FSQL_ENGINE_DUAL_PRIME;
  int br_shape = 2;              // launch shape of the blind rotation for large batches (index into kBrShapes)
  int latency_mode = 2;          // small batches (two-prime engine): 0 one gate per 128-thread CTA,
                                 // 1 one gate per CTA of three groups, 2 one gate per cluster of 6 CTAs
                                 // (while every gate gets a cluster at once, else 1)
  bool walk_mode = false;        // batched scans as one device-walked launch (scan_walk_kernel)
  double walk_timeout_ms = 2000.0;  // limit of each grid-barrier wait of the walker
  int walk_skip_block = -1;      // test hook: this CTA never arrives at the walker's barriers
  WalkSync* d_walk_sync = nullptr;
  // host-side secrets and standard-domain keys (client side)
  std::vector<uint8_t> s;    // LWE key [n]
  std::vector<uint8_t> S;    // GLWE key [N]
  std::vector<uint32_t> bk;  // [n][2l][2][N]
  std::vector<uint32_t> ksk; // [N][t][digits][n+1]
  // device-resident keys
  uint64_t* d_bkhat = nullptr;   // [n][2l][32][32][2] u64, NTT domain, times N^-1
  uint32_t* d_ksk = nullptr;     // [N][t][digits][kKsRowWords]
  uint32_t* d_ks_part = nullptr; // keyswitch partial sums of small batches [16][128][kKsRowWords]
  // keyswitch-first order: keyswitched samples [cap][n+1], their blind-rotation
  // descriptors [cap], the trivial true ciphertext [n+1]
  uint32_t* d_ks_small = nullptr;
  GateDesc* d_ks_desc = nullptr;
  uint32_t* d_true = nullptr;
  size_t ks_small_cap = 0;
  uint64_t ks_gen = 0;           // bumped whenever the keyswitch-first scratch is reallocated
  void* d_tables = nullptr;      // NttTablesT of the engine
  uint32_t* d_bks = nullptr;     // two-prime engine: the key split by prime [n][2l][2 primes][8][128][2] u32
  void* d_tables_split = nullptr;  // two-prime engine: NttTablesT<uint2> per prime (each padded to 128 B)
  std::vector<uint8_t> tables;   // host copy
  size_t key_bytes = 0;
  // scratch (grown on demand, freed with the context)
  uint32_t* d_big = nullptr;     // extracted samples [cap][N+1]
  size_t big_cap = 0;
  GateDesc* d_desc = nullptr;
  size_t desc_cap = 0;
  uint32_t* d_wires = nullptr;   // intermediate wires of a scan
  size_t wires_cap = 0;          // in words
  void* d_prog = nullptr;        // the current scan plan's program (netlist + pointers), see schedule.cu
  size_t prog_cap = 0;           // in bytes
  uint32_t* d_stage = nullptr;   // device staging for the host-buffer scan
  size_t stage_cap = 0;
  OutDesc* d_lits = nullptr;     // scan outputs no gate writes (plaintext constants)
  size_t lits_cap = 0;
  Plan* plan = nullptr;
  Plan* agg_plan = nullptr;      // SUM aggregation plan (owns its buffers)
  void* prof = nullptr;          // kernel-timing events while profiling (kernels.cu)
  void* capture_stream = nullptr;  // cudaStream_t used to capture scan graphs
  int sm_count = 0;
  std::mutex mu;
};

// host.cpp
void set_error(const std::string& msg);
std::vector<uint8_t> sample_key_bits(uint64_t seed, uint64_t stream, size_t count);
void keygen(Ctx& c);
uint32_t encode_bit(bool b);

// Per-row netlist of a predicate (circuit scheduler, host side).
struct Netlist {
  int n_inputs = 0;          // column bits, constant bits, payload bits
  int n_const = 0;           // constant-ciphertext inputs (none with plaintext constants)
  int match_wire = -1;       // -1: no gate writes the match bit (see literal_outs)
  int first_mask_gate = 0;   // gates [first_mask_gate, count) are the payload masks
  std::vector<int> type, a, b, c;  // gate g writes wire n_inputs + g; c = -1 for two inputs
  std::vector<int> level;       // 1-based level of each gate
  int levels = 0;
  // outputs that no gate writes: target -1 is the match bit, m >= 0 the
  // m-th masked payload bit; wire -1 for a known bit
  struct LiteralOut {
    int target;
    int wire;
    uint32_t mode;
  };
  std::vector<LiteralOut> literal_outs;
};
bool build_netlist(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width, Netlist* out);
// The SUM-aggregation circuit over rows x width input bits (input bit (r, j)
// is wire r * width + j); every output bit j is a literal output with target j.
bool build_sum_netlist(size_t rows, uint32_t width, uint32_t out_width, Netlist* out);
// MAX / MIN over `rows` values (MIN's match bit of row r is wire rows * width + r).
bool build_extreme_netlist(bool is_min, size_t rows, uint32_t width, Netlist* out);
// The netlist for plaintext constants k0 (EQ, LT) or lo = k0, hi = k1 (RANGE):
// gates with a known input are reduced away (see host.cpp).
bool build_netlist_plain(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width, uint64_t k0,
                         uint64_t k1, Netlist* out);

// Device buffers of one scan (layouts as in fsql_scan_select) plus its
// intermediate-wire scratch [rows][internal wires][n+1].
struct ScanIO {
  const uint32_t* column = nullptr;
  size_t rows = 0;
  uint32_t width = 0, pred = 0;
  const uint32_t* cst = nullptr;
  uint32_t n_payloads = 0;
  const uint32_t* const* payloads = nullptr;
  uint32_t payload_width = 0;
  uint32_t* match = nullptr;
  uint32_t* const* outs = nullptr;
  uint32_t* wires = nullptr;
  size_t words = 0;  // n + 1
};
// Gates of a row that are neither the match bit nor a mask gate (they need scratch).
long scan_internal_wires(const Netlist& nl);
// Descriptors of the outputs no gate writes, every row.
void scan_literals(const Netlist& nl, const ScanIO& io, std::vector<OutDesc>* out);

// schedule.cu: descriptors generated on the device from a scan program
// (the per-row netlist plus the scan's buffer pointers, a few KB).
size_t scan_program_bytes(const Netlist& nl);
// The program of a scan (host bytes to copy to the device as they are) and
// the descriptor offsets of its levels (levels + 1 entries); false if the
// scan has more payload columns than a program holds (64).
bool build_scan_program(const Netlist& nl, const ScanIO& io, std::vector<uint8_t>* out,
                        std::vector<size_t>* level_offset);
// Writes all rows x gates descriptors of the program at d_prog to d_out
// (level by level, gate-major within a level, rows in order), on `stream`.
int launch_gen_desc(const void* d_prog, GateDesc* d_out, size_t total, void* stream);

// kernels.cu
int device_init(Ctx& c);     // tables, BK -> NTT domain, KSK upload
void device_free(Ctx& c);
int launch_gates(Ctx& c, const GateDesc* d_desc, size_t count, uint32_t* d_big, void* stream);
int launch_blind_rotate(Ctx& c, const GateDesc* d_desc, size_t count, uint32_t* d_big, void* stream);
int launch_keyswitch(Ctx& c, const uint32_t* d_big, const GateDesc* d_desc, uint32_t* d_out_contig,
                     size_t count, void* stream);

// plain.cu
int launch_literals(const OutDesc* d_lits, size_t count, int n, void* stream);

}  // namespace fsql
