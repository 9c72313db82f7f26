// host.cpp -- client-side half of the library: parameters, seeded key
// generation (KeyGen of §2.2), encryption and decryption (Alg. 1 EncryptQuery /
// Decrypt), and the circuit scheduler that lowers a WHERE predicate to levels
// of bootstrapped gates (Alg. 2 EvaluateHomomorphicTree, §4.2 B).
//
// Randomness is SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
// counter-addressed generator: value #k of a generator started at state x is
// mix(x + (k+1) * golden_gamma).  Word (seed, stream, k) is value #k of the
// generator whose start state is value #stream of the generator started at the
// seed.  Floating point appears only in the Gaussian sampler and is compiled
// without contraction or fast-math.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <thread>

#include "engine.h"

namespace fsql {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ull;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// A SplitMix64 stream positioned by counter.
struct Stream {
  uint64_t start;
  Stream(uint64_t seed, uint64_t stream_id) : start(mix64(seed + (stream_id + 1) * kGamma)) {}
  uint64_t at(uint64_t k) const { return mix64(start + (k + 1) * kGamma); }
  uint32_t u32(uint64_t k) const { return static_cast<uint32_t>(at(k) >> 32); }
  // Discrete Gaussian on the torus: z = sqrt(-2 ln u1) cos(2 pi u2) from the
  // words k and k+1 (u1 in (0,1], u2 in [0,1) with 53-bit resolution), then
  // sigma*z*2^32 rounded half away from zero, wrapped mod 2^32.
  uint32_t noise(uint64_t k, double sigma) const {
    const double u1 = static_cast<double>((at(k) >> 11) + 1) * 0x1p-53;
    const double u2 = static_cast<double>(at(k + 1) >> 11) * 0x1p-53;
    const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    const double scaled = (sigma * z) * 4294967296.0;
    return static_cast<uint32_t>(static_cast<uint64_t>(std::llround(scaled)));
  }
};

// Run body(i) for i in [0, count) on up to hardware_concurrency threads.
template <class F>
void parallel_for(size_t count, F body) {
  size_t nt = std::max<size_t>(1, std::min<size_t>(std::thread::hardware_concurrency(), 64));
  nt = std::min(nt, std::max<size_t>(1, count / 16));
  if (nt <= 1) {
    for (size_t i = 0; i < count; ++i) body(i);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (size_t t = 0; t < nt; ++t)
    pool.emplace_back([=, &body] {
      for (size_t i = t; i < count; i += nt) body(i);
    });
  for (auto& th : pool) th.join();
}

// LWE sample of message mu under binary key `key` (length dim): uniform mask
// from words base .. base+dim-1, noise from words base+dim, base+dim+1.
void lwe_sample(const Stream& st, uint64_t base, const uint8_t* key, uint32_t dim, uint32_t mu, double sigma,
                uint32_t* ct) {
  uint32_t acc = mu + st.noise(base + dim, sigma);
  for (uint32_t x = 0; x < dim; ++x) {
    const uint32_t a = st.u32(base + x);
    ct[x] = a;
    acc += key[x] ? a : 0u;
  }
  ct[dim] = acc;
}

}  // namespace

std::vector<uint8_t> sample_key_bits(uint64_t seed, uint64_t stream, size_t count) {
  Stream st(seed, stream);
  std::vector<uint8_t> bits(count);
  for (size_t i = 0; i < count; ++i) bits[i] = static_cast<uint8_t>(st.at(i) >> 63);
  return bits;
}

uint32_t encode_bit(bool b) { return b ? (1u << 29) : (0u - (1u << 29)); }

// Key generation.  Bootstrapping key row (i, u, j): a GLWE encryption of zero
// under S -- mask A uniform, body B = A*S + e in Z_q[X]/(X^N+1) -- with the
// gadget value s_i * 2^(32 - bg*j) added to the constant coefficient of
// polynomial u (0 = A, 1 = B).  Since S is binary, A*S is the sum of the
// negacyclic shifts X^m * A over the positions m where S_m = 1.
// Keyswitching key entry (i, j, v): LWE_s(v * S_i * 2^(32 - kb*(j+1))).
void keygen(Ctx& c) {
  const fsql_params& p = c.p;
  const uint32_t n = p.n, N = p.N, l = p.l;
  c.s = sample_key_bits(c.seed, 0, n);
  c.S = sample_key_bits(c.seed, 1, N);

  std::vector<uint32_t> ones;
  for (uint32_t m = 0; m < N; ++m)
    if (c.S[m]) ones.push_back(m);

  c.bk.assign(static_cast<size_t>(n) * 2 * l * 2 * N, 0u);
  const Stream bst(c.seed, 2);
  parallel_for(static_cast<size_t>(n) * 2 * l, [&](size_t R) {
    const uint32_t i = static_cast<uint32_t>(R / (2 * l));
    const uint32_t row = static_cast<uint32_t>(R % (2 * l));
    const uint32_t u = row / l, j = row % l + 1;
    const uint64_t base = static_cast<uint64_t>(R) * 3 * N;
    uint32_t* A = c.bk.data() + R * 2 * N;
    uint32_t* B = A + N;
    for (uint32_t x = 0; x < N; ++x) A[x] = bst.u32(base + x);
    for (uint32_t x = 0; x < N; ++x) B[x] = bst.noise(base + N + 2 * x, p.glwe_sigma);
    for (uint32_t m : ones) {
      // B += X^m * A:  coefficient k gets A[k-m] for k >= m, -A[k-m+N] below.
      for (uint32_t k = 0; k < m; ++k) B[k] -= A[k + N - m];
      for (uint32_t k = m; k < N; ++k) B[k] += A[k - m];
    }
    if (c.s[i]) (u == 0 ? A : B)[0] += 1u << (32 - p.bg_bits * j);
  });

  const uint32_t digits = (1u << p.ks_base_bits) - 1;
  c.ksk.assign(static_cast<size_t>(N) * p.ks_t * digits * (n + 1), 0u);
  const Stream kst(c.seed, 3);
  parallel_for(static_cast<size_t>(N) * p.ks_t * digits, [&](size_t idx) {
    const uint32_t i = static_cast<uint32_t>(idx / (p.ks_t * digits));
    const uint32_t j = static_cast<uint32_t>((idx / digits) % p.ks_t);
    const uint32_t v = static_cast<uint32_t>(idx % digits) + 1;
    const uint32_t mu = c.S[i] ? v << (32 - p.ks_base_bits * (j + 1)) : 0u;
    lwe_sample(kst, static_cast<uint64_t>(idx) * (n + 2), c.s.data(), n, mu, p.lwe_sigma,
               c.ksk.data() + idx * (n + 1));
  });
}

// ---------------------------------------------------------------------------
// Circuit scheduler.  Wire numbering of one row: column bits [0, w), constant
// bits [w, w + nc) (nc = w, or 2w for RANGE: lo then hi), payload bits after
// them (payload column major, LSB first), gate outputs after the inputs in
// emission order.  Level of a gate = 1 + max level of its inputs (inputs are
// level 0).  The gate order is canonical: any change changes output words.
// ---------------------------------------------------------------------------
namespace {

struct Builder {
  Netlist& nl;
  std::vector<int> wire_level;
  explicit Builder(Netlist& n) : nl(n), wire_level(n.n_inputs, 0) {}
  int gate(int type, int a, int b, int c = -1) {
    int lv = 1 + std::max(wire_level[a], wire_level[b]);
    if (c >= 0) lv = std::max(lv, 1 + wire_level[c]);
    nl.type.push_back(type);
    nl.a.push_back(a);
    nl.b.push_back(b);
    nl.c.push_back(c);
    nl.level.push_back(lv);
    nl.levels = std::max(nl.levels, lv);
    wire_level.push_back(lv);
    return static_cast<int>(wire_level.size()) - 1;
  }
  // c == k: bitwise XNOR, then a balanced AND reduction that pairs neighbours
  // (0,1), (2,3), ... each round and passes an unpaired last element on.
  int equal(int c0, int k0, int w) {
    std::vector<int> cur;
    for (int i = 0; i < w; ++i) cur.push_back(gate(FSQL_XNOR, c0 + i, k0 + i));
    while (cur.size() > 1) {
      std::vector<int> next;
      size_t i = 0;
      for (; i + 1 < cur.size(); i += 2) next.push_back(gate(FSQL_AND, cur[i], cur[i + 1]));
      if (i < cur.size()) next.push_back(cur[i]);
      cur.swap(next);
    }
    return cur[0];
  }
  // c < k (unsigned), LSB-first ripple: less_0 = !c_0 & k_0;
  // less_i = (!c_i & k_i) | (c_i == k_i & less_{i-1}).
  int less(int c0, int k0, int w) {
    int lt = gate(FSQL_ANDNY, c0, k0);
    for (int i = 1; i < w; ++i) {
      const int strictly = gate(FSQL_ANDNY, c0 + i, k0 + i);
      const int same = gate(FSQL_XNOR, c0 + i, k0 + i);
      const int carried = gate(FSQL_AND, same, lt);
      lt = gate(FSQL_OR, strictly, carried);
    }
    return lt;
  }
  // c < k as a majority chain: less_0 = !c_0 & k_0;
  // less_i = MAJ(!c_i, k_i, less_{i-1}) (same truth table, one gate per bit).
  int less_maj(int c0, int k0, int w) {
    int lt = gate(FSQL_ANDNY, c0, k0);
    for (int i = 1; i < w; ++i) lt = gate(FSQL_MAJNYY, c0 + i, k0 + i, lt);
    return lt;
  }
};

// Values of the plaintext-constant netlist: a wire, possibly negated, or a
// bit the server already knows.
struct Lit {
  int wire = -1;      // -1: known bit
  bool flip = false;  // wire: negated; known bit: its value
  static Lit known(bool v) {
    Lit l;
    l.flip = v;
    return l;
  }
  static Lit of(int w, bool negated) {
    Lit l;
    l.wire = w;
    l.flip = negated;
    return l;
  }
  bool is_known() const { return wire < 0; }
  Lit operator!() const {
    Lit l = *this;
    l.flip = !l.flip;
    return l;
  }
};

// Boolean algebra on literals over a Builder: a known operand decides the
// result or drops out; two wires make one gate whose type absorbs the
// negations, so every gate output is a plain wire.
struct LitBuilder {
  Builder& b;
  explicit LitBuilder(Builder& bb) : b(bb) {}
  Lit both(Lit x, Lit y) {
    if (x.is_known()) return x.flip ? y : Lit::known(false);
    if (y.is_known()) return y.flip ? x : Lit::known(false);
    int type = FSQL_AND;
    if (x.flip && y.flip) type = FSQL_NOR;      // !x & !y
    else if (x.flip) type = FSQL_ANDNY;         // !x & y
    else if (y.flip) type = FSQL_ANDYN;         // x & !y
    return Lit::of(b.gate(type, x.wire, y.wire), false);
  }
  Lit either(Lit x, Lit y) {
    if (x.is_known()) return x.flip ? Lit::known(true) : y;
    if (y.is_known()) return y.flip ? Lit::known(true) : x;
    int type = FSQL_OR;
    if (x.flip && y.flip) type = FSQL_NAND;     // !x | !y
    else if (x.flip) type = FSQL_ORNY;          // !x | y
    else if (y.flip) type = FSQL_ORYN;          // x | !y
    return Lit::of(b.gate(type, x.wire, y.wire), false);
  }
  // c == k with k known: bit i is c_i or !c_i; then the same neighbour-pairing
  // AND reduction as the encrypted-constant circuit.
  Lit equal(int c0, int w, uint64_t k) {
    std::vector<Lit> cur;
    for (int i = 0; i < w; ++i) cur.push_back(Lit::of(c0 + i, ((k >> i) & 1) == 0));
    while (cur.size() > 1) {
      std::vector<Lit> next;
      size_t i = 0;
      for (; i + 1 < cur.size(); i += 2) next.push_back(both(cur[i], cur[i + 1]));
      if (i < cur.size()) next.push_back(cur[i]);
      cur.swap(next);
    }
    return cur[0];
  }
  // c < k with k known: less_i = MAJ(!c_i, k_i, less_{i-1}) is
  // !c_i | less_{i-1} when k_i = 1 and !c_i & less_{i-1} when k_i = 0
  // (less_{-1} = false).
  Lit less(int c0, int w, uint64_t k) {
    Lit lt = Lit::known(false);
    for (int i = 0; i < w; ++i) {
      const Lit not_c = Lit::of(c0 + i, true);
      lt = ((k >> i) & 1) ? either(not_c, lt) : both(not_c, lt);
    }
    return lt;
  }
};

}  // namespace

bool build_netlist_plain(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width, uint64_t k0,
                         uint64_t k1, Netlist* out) {
  if (width < 1 || width > 64 || pred > FSQL_RANGE_MAJ || n_payloads > 64 || payload_width > 64) return false;
  if (n_payloads > 0 && payload_width == 0) return false;
  Netlist nl;
  const int w = static_cast<int>(width);
  nl.n_const = 0;
  nl.n_inputs = w + static_cast<int>(n_payloads * payload_width);
  Builder b(nl);
  LitBuilder lb(b);
  Lit match;
  if (pred == FSQL_EQ) {
    match = lb.equal(0, w, k0);
  } else if (pred == FSQL_LT || pred == FSQL_LT_MAJ) {
    match = lb.less(0, w, k0);
  } else {
    const Lit below_lo = lb.less(0, w, k0);
    const Lit below_hi = lb.less(0, w, k1);
    match = lb.both(!below_lo, below_hi);  // !(c < lo) & (c < hi)
  }
  const bool match_is_gate = !match.is_known() && !match.flip && match.wire >= nl.n_inputs;
  nl.match_wire = match_is_gate ? match.wire : -1;
  if (!match_is_gate) {
    const uint32_t mode = match.is_known() ? (match.flip ? kOutTrue : kOutFalse) : (match.flip ? kOutNegate : kOutCopy);
    nl.literal_outs.push_back({-1, match.wire, mode});
  }
  nl.first_mask_gate = static_cast<int>(nl.type.size());
  // cmux(m, v, 0) = m AND v per payload bit; with a known m it is v or 0
  int m_index = 0;
  for (uint32_t q = 0; q < n_payloads; ++q)
    for (uint32_t bit = 0; bit < payload_width; ++bit, ++m_index) {
      const Lit v = Lit::of(w + static_cast<int>(q * payload_width + bit), false);
      const Lit o = lb.both(match, v);
      if (o.is_known()) nl.literal_outs.push_back({m_index, -1, o.flip ? kOutTrue : kOutFalse});
      else if (o.wire < nl.n_inputs) nl.literal_outs.push_back({m_index, o.wire, o.flip ? kOutNegate : kOutCopy});
    }
  *out = std::move(nl);
  return true;
}

// SUM of `rows` values of `width` bits mod 2^out_width as a carry-save tree.
// Bit columns hold the wires of weight 2^j; a layer turns each group of three
// wires of a column (in order) into a full adder whose sum stays in the
// column and whose carry joins the next column of the next layer (columns
// are visited low to high, so a column's next list is: carries from below,
// its own sums, its 0-2 leftover wires).  When no column has more than two
// wires, a ripple-carry adder finishes: per column its wires plus the
// incoming carry, 0 operands -> known 0, 1 -> that wire, 2 -> half adder
// (XOR, AND), 3 -> full adder (XOR3, MAJ); the top column drops its carry.
// Every output is a literal output (copy of a wire, or known 0).
bool build_sum_netlist(size_t rows, uint32_t width, uint32_t out_width, Netlist* out) {
  if (width < 1 || width > 64 || out_width < 1 || out_width > 64 || rows > (size_t(1) << 22) ||
      rows * width > (size_t(1) << 24))
    return false;
  Netlist nl;
  const int w = static_cast<int>(width), ow = static_cast<int>(out_width);
  nl.n_inputs = static_cast<int>(rows * width);
  nl.n_const = 0;
  nl.match_wire = -1;
  Builder b(nl);
  std::vector<std::vector<int>> column(ow);
  for (int j = 0; j < std::min(w, ow); ++j)
    for (size_t r = 0; r < rows; ++r) column[j].push_back(static_cast<int>(r * width) + j);
  auto crowded = [&]() {
    for (const auto& c : column)
      if (c.size() > 2) return true;
    return false;
  };
  while (crowded()) {
    std::vector<std::vector<int>> next(ow);
    for (int j = 0; j < ow; ++j) {
      const std::vector<int>& wires = column[j];
      size_t i = 0;
      for (; i + 3 <= wires.size(); i += 3) {
        next[j].push_back(b.gate(FSQL_XOR3, wires[i], wires[i + 1], wires[i + 2]));
        if (j + 1 < ow) next[j + 1].push_back(b.gate(FSQL_MAJ, wires[i], wires[i + 1], wires[i + 2]));
      }
      next[j].insert(next[j].end(), wires.begin() + static_cast<long>(i), wires.end());
    }
    column.swap(next);
  }
  int carry = -1;
  for (int j = 0; j < ow; ++j) {
    std::vector<int> ops = column[j];
    if (carry >= 0) ops.push_back(carry);
    const bool top = j + 1 == ow;
    carry = -1;
    int result = -1;
    if (ops.size() == 1) {
      result = ops[0];
    } else if (ops.size() == 2) {
      result = b.gate(FSQL_XOR, ops[0], ops[1]);
      if (!top) carry = b.gate(FSQL_AND, ops[0], ops[1]);
    } else if (ops.size() == 3) {
      result = b.gate(FSQL_XOR3, ops[0], ops[1], ops[2]);
      if (!top) carry = b.gate(FSQL_MAJ, ops[0], ops[1], ops[2]);
    }
    nl.literal_outs.push_back({j, result, result < 0 ? kOutFalse : kOutCopy});
  }
  nl.first_mask_gate = static_cast<int>(nl.type.size());
  *out = std::move(nl);
  return true;
}

// MAX (is_min false) or MIN of `rows` unsigned values of `width` bits.
// Pairwise step: s = [a < b] from the majority comparator (ANDNY on bit 0,
// MAJNYY above), then per bit the multiplexer s ? x : y as
// OR(AND(s, x), ANDNY(s, y)), x = b, y = a for max and x = a, y = b for min.
// Values meet in a tournament paired like the equality AND tree
// (neighbours (0,1), (2,3), ..., an unpaired last value moves on).  MIN
// first sets every bit of a row that does not match to 1 (ORYN(v, m)), so
// such rows cannot win.  No rows: MAX is 0 and MIN is all ones (known bits).
// Inputs: value bit (r, j) = wire r * width + j; MIN's match bit of row r
// is wire rows * width + r.  Output bit j is a literal output with target j.
bool build_extreme_netlist(bool is_min, size_t rows, uint32_t width, Netlist* out) {
  if (width < 1 || width > 64 || rows > (size_t(1) << 22) || rows * width > (size_t(1) << 24)) return false;
  Netlist nl;
  const int w = static_cast<int>(width), R = static_cast<int>(rows);
  nl.n_inputs = R * w + (is_min ? R : 0);
  nl.n_const = 0;
  nl.match_wire = -1;
  Builder b(nl);
  std::vector<std::vector<int>> vals(rows, std::vector<int>(w));
  for (int r = 0; r < R; ++r)
    for (int j = 0; j < w; ++j)
      vals[r][j] = is_min ? b.gate(FSQL_ORYN, r * w + j, R * w + r) : r * w + j;
  while (vals.size() > 1) {
    std::vector<std::vector<int>> next;
    size_t i = 0;
    for (; i + 1 < vals.size(); i += 2) {
      const std::vector<int>& lo = vals[i];
      const std::vector<int>& hi = vals[i + 1];
      int s = b.gate(FSQL_ANDNY, lo[0], hi[0]);  // [lo < hi]
      for (int j = 1; j < w; ++j) s = b.gate(FSQL_MAJNYY, lo[j], hi[j], s);
      std::vector<int> pick(w);
      for (int j = 0; j < w; ++j) {
        const int when_less = is_min ? lo[j] : hi[j], otherwise = is_min ? hi[j] : lo[j];
        const int taken = b.gate(FSQL_AND, s, when_less);
        const int kept = b.gate(FSQL_ANDNY, s, otherwise);
        pick[j] = b.gate(FSQL_OR, taken, kept);
      }
      next.push_back(std::move(pick));
    }
    if (i < vals.size()) next.push_back(std::move(vals[i]));
    vals.swap(next);
  }
  for (int j = 0; j < w; ++j) {
    if (R > 0) nl.literal_outs.push_back({j, vals[0][j], kOutCopy});
    else nl.literal_outs.push_back({j, -1, is_min ? kOutTrue : kOutFalse});
  }
  nl.first_mask_gate = static_cast<int>(nl.type.size());
  *out = std::move(nl);
  return true;
}

bool build_netlist(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width, Netlist* out) {
  if (width < 1 || width > 64 || pred > FSQL_RANGE_MAJ || n_payloads > 64 || payload_width > 64) return false;
  if (n_payloads > 0 && payload_width == 0) return false;
  Netlist nl;
  const int w = static_cast<int>(width);
  const bool range = pred == FSQL_RANGE || pred == FSQL_RANGE_MAJ;
  const int nconst = range ? 2 * w : w;
  nl.n_const = nconst;
  nl.n_inputs = w + nconst + static_cast<int>(n_payloads * payload_width);
  Builder b(nl);
  if (pred == FSQL_EQ) {
    nl.match_wire = b.equal(0, w, w);
  } else if (pred == FSQL_LT) {
    nl.match_wire = b.less(0, w, w);
  } else if (pred == FSQL_LT_MAJ) {
    nl.match_wire = b.less_maj(0, w, w);
  } else {
    const bool maj = pred == FSQL_RANGE_MAJ;
    const int below_lo = maj ? b.less_maj(0, w, w) : b.less(0, w, w);
    const int below_hi = maj ? b.less_maj(0, 2 * w, w) : b.less(0, 2 * w, w);
    nl.match_wire = b.gate(FSQL_ANDNY, below_lo, below_hi);  // !(c < lo) & (c < hi)
  }
  nl.first_mask_gate = static_cast<int>(nl.type.size());
  // Homomorphic If-Then-Else per payload bit: cmux(m, v, 0) = m AND v.
  for (uint32_t q = 0; q < n_payloads; ++q)
    for (uint32_t bit = 0; bit < payload_width; ++bit)
      b.gate(FSQL_AND, nl.match_wire, w + nconst + static_cast<int>(q * payload_width + bit));
  *out = std::move(nl);
  return true;
}

}  // namespace fsql

using fsql::Ctx;

namespace {

template <class F>
int guarded(F f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    fsql::set_error("host allocation failed");
    return FSQL_ERR_OOM;
  } catch (const std::exception& e) {
    fsql::set_error(e.what());
    return FSQL_ERR_ARG;
  } catch (...) {
    fsql::set_error("unknown exception");
    return FSQL_ERR_ARG;
  }
}

int arg_error(const char* msg) {
  fsql::set_error(msg);
  return FSQL_ERR_ARG;
}

bool params_valid(const fsql_params& p, std::string* why) {
  auto pow2 = [](uint32_t v) { return v && !(v & (v - 1)); };
  if (p.n < 1 || p.n > 4096) return *why = "n must be in [1, 4096]", false;
  if (!pow2(p.N) || p.N < 4 || p.N > 4096) return *why = "N must be a power of two in [4, 4096]", false;
  if (p.bg_bits < 1 || p.l < 1 || p.bg_bits * p.l > 31) return *why = "need bg_bits*l <= 31", false;
  if (p.ks_base_bits < 1 || p.ks_base_bits > 8 || p.ks_t < 1 || p.ks_base_bits * p.ks_t > 31)
    return *why = "need ks_base_bits*ks_t <= 31", false;
  if (!(p.lwe_sigma >= 0.0 && p.lwe_sigma < 1.0) || !(p.glwe_sigma >= 0.0 && p.glwe_sigma < 1.0))
    return *why = "noise std-devs must be in [0, 1)", false;
  return true;
}

}  // namespace

extern "C" {

int fsql_params_default(fsql_params* out) {
  if (!out) return arg_error("null params");
  *out = fsql_params{630, 1024, 7, 3, 2, 8, 0x1p-15, 0x1p-25};
  return FSQL_OK;
}

int fsql_params_toy(fsql_params* out) {
  if (!out) return arg_error("null params");
  *out = fsql_params{16, 64, 7, 3, 2, 8, 0x1p-25, 0x1p-25};
  return FSQL_OK;
}

const char* fsql_last_error(void) { return fsql::g_last_error.c_str(); }

int fsql_ctx_create_engine(const fsql_params* params, uint64_t seed, int device, int engine, fsql_ctx** out) {
  return guarded([&]() -> int {
    if (!params || !out) return arg_error("null argument");
    *out = nullptr;
    std::string why;
    if (!params_valid(*params, &why)) return arg_error(why.c_str());
    if (engine == FSQL_ENGINE_DEFAULT) engine = FSQL_ENGINE_DUAL_PRIME;
    if (engine != FSQL_ENGINE_GOLDILOCKS && engine != FSQL_ENGINE_DUAL_PRIME) return arg_error("unknown NTT engine");
    auto* c = new Ctx();
    c->p = *params;
    c->seed = seed;
    c->device = device;
    c->engine = engine;
    c->br_shape = engine == FSQL_ENGINE_GOLDILOCKS ? 3 : 2;
    fsql::keygen(*c);
    if (device >= 0) {
      const int rc = fsql::device_init(*c);
      if (rc != FSQL_OK) {
        fsql::device_free(*c);
        delete c;
        return rc;
      }
    }
    *out = reinterpret_cast<fsql_ctx*>(c);
    return FSQL_OK;
  });
}

int fsql_ctx_create(const fsql_params* params, uint64_t seed, int device, fsql_ctx** out) {
  return fsql_ctx_create_engine(params, seed, device, FSQL_ENGINE_DEFAULT, out);
}

int fsql_ctx_set_br_gates(fsql_ctx* ctx, int gates_per_cta) {
  if (!ctx) return arg_error("null context");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (gates_per_cta < 1 || gates_per_cta > 4 || !fsql::shape_offered(c->engine, gates_per_cta - 1))
    return arg_error("gates per CTA: 1, 2 or 4 (Goldilocks engine), 1 to 4 (dual-prime engine)");
  c->br_shape = gates_per_cta - 1;  // the packed kernel with that many gates per CTA
  return FSQL_OK;
}

int fsql_ctx_set_br_shape(fsql_ctx* ctx, int shape) {
  if (!ctx) return arg_error("null context");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!fsql::shape_offered(c->engine, shape)) return arg_error("launch shape not offered by this engine");
  c->br_shape = shape;
  return FSQL_OK;
}

int fsql_ctx_br_shape(const fsql_ctx* ctx, int* shape) {
  if (!ctx || !shape) return arg_error("null argument");
  *shape = reinterpret_cast<const Ctx*>(ctx)->br_shape;
  return FSQL_OK;
}

int fsql_br_shape_info(int shape, int* kind, int* gates_per_cta, int* rows_per_step, int* stages) {
  if (shape < 0 || shape >= fsql::kBrShapeCount) return arg_error("no such launch shape");
  const fsql::BrShape& s = fsql::kBrShapes[shape];
  if (kind) *kind = s.kind;
  if (gates_per_cta) *gates_per_cta = s.gates;
  if (rows_per_step) *rows_per_step = s.rows;
  if (stages) *stages = s.stages;
  return FSQL_OK;
}

int fsql_ctx_set_latency_mode(fsql_ctx* ctx, int on) {
  if (!ctx) return arg_error("null context");
  if (on < 0 || on > 2) return arg_error("latency mode: 0, 1 or 2");
  reinterpret_cast<Ctx*>(ctx)->latency_mode = on;
  return FSQL_OK;
}

int fsql_ctx_br_gates(const fsql_ctx* ctx, int* gates_per_cta) {
  if (!ctx || !gates_per_cta) return arg_error("null argument");
  *gates_per_cta = fsql::kBrShapes[reinterpret_cast<const Ctx*>(ctx)->br_shape].gates;
  return FSQL_OK;
}

int fsql_ctx_engine(const fsql_ctx* ctx, int* engine) {
  if (!ctx || !engine) return arg_error("null argument");
  *engine = reinterpret_cast<const Ctx*>(ctx)->engine;
  return FSQL_OK;
}

void fsql_ctx_destroy(fsql_ctx* ctx) {
  if (!ctx) return;
  auto* c = reinterpret_cast<Ctx*>(ctx);
  fsql::device_free(*c);
  delete c;
}

int fsql_ctx_params(const fsql_ctx* ctx, fsql_params* out) {
  if (!ctx || !out) return arg_error("null argument");
  *out = reinterpret_cast<const Ctx*>(ctx)->p;
  return FSQL_OK;
}

int fsql_ctx_device_bytes(const fsql_ctx* ctx, size_t* key_bytes, size_t* scratch_bytes) {
  if (!ctx) return arg_error("null context");
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  if (key_bytes) *key_bytes = c->key_bytes;
  if (scratch_bytes)
    *scratch_bytes = c->big_cap * (c->p.N + 1) * 4 + c->desc_cap * sizeof(fsql::GateDesc) + c->wires_cap * 4 +
                     c->stage_cap * 4;
  return FSQL_OK;
}

int fsql_export_keys(const fsql_ctx* ctx, uint8_t* lwe_key, uint8_t* glwe_key, uint32_t* bk, uint32_t* ksk) {
  if (!ctx) return arg_error("null context");
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  if (lwe_key) std::memcpy(lwe_key, c->s.data(), c->s.size());
  if (glwe_key) std::memcpy(glwe_key, c->S.data(), c->S.size());
  if (bk) std::memcpy(bk, c->bk.data(), c->bk.size() * 4);
  if (ksk) std::memcpy(ksk, c->ksk.data(), c->ksk.size() * 4);
  return FSQL_OK;
}

int fsql_encrypt(const fsql_ctx* ctx, const uint32_t* mu, size_t count, uint64_t stream, uint64_t first_index,
                 uint32_t* out) {
  return guarded([&]() -> int {
    if (!ctx || (count && (!mu || !out))) return arg_error("null argument");
    const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
    const uint32_t n = c->p.n;
    const fsql::Stream st(c->seed, stream);
    fsql::parallel_for(count, [&](size_t k) {
      fsql::lwe_sample(st, (first_index + k) * (n + 2), c->s.data(), n, mu[k], c->p.lwe_sigma,
                       out + k * (n + 1));
    });
    return FSQL_OK;
  });
}

int fsql_encrypt_bits(const fsql_ctx* ctx, const uint8_t* bits, size_t count, uint64_t stream,
                      uint64_t first_index, uint32_t* out) {
  return guarded([&]() -> int {
    if (!ctx || (count && (!bits || !out))) return arg_error("null argument");
    std::vector<uint32_t> mu(count);
    for (size_t k = 0; k < count; ++k) mu[k] = fsql::encode_bit(bits[k] != 0);
    return fsql_encrypt(ctx, mu.data(), count, stream, first_index, out);
  });
}

int fsql_encrypt_big_bits(const fsql_ctx* ctx, const uint8_t* bits, size_t count, uint64_t stream,
                          uint64_t first_index, uint32_t* out) {
  return guarded([&]() -> int {
    if (!ctx || (count && (!bits || !out))) return arg_error("null argument");
    const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
    const uint32_t N = c->p.N;
    const fsql::Stream st(c->seed, stream);
    fsql::parallel_for(count, [&](size_t k) {
      fsql::lwe_sample(st, (first_index + k) * (N + 2), c->S.data(), N, fsql::encode_bit(bits[k] != 0),
                       c->p.glwe_sigma, out + k * (N + 1));
    });
    return FSQL_OK;
  });
}

int fsql_decrypt_big_bits(const fsql_ctx* ctx, const uint32_t* ct, size_t count, uint8_t* out) {
  return guarded([&]() -> int {
    if (!ctx || (count && (!ct || !out))) return arg_error("null argument");
    const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
    const uint32_t N = c->p.N;
    for (size_t k = 0; k < count; ++k) {
      const uint32_t* row = ct + k * (N + 1);
      uint32_t dot = 0;
      for (uint32_t x = 0; x < N; ++x) dot += c->S[x] ? row[x] : 0u;
      out[k] = static_cast<int32_t>(row[N] - dot) > 0 ? 1 : 0;
    }
    return FSQL_OK;
  });
}

int fsql_encrypt_uint(const fsql_ctx* ctx, const uint64_t* values, size_t rows, uint32_t width, uint64_t stream,
                      uint64_t first_index, uint32_t* out) {
  return guarded([&]() -> int {
    if (!ctx || (rows && (!values || !out))) return arg_error("null argument");
    if (width < 1 || width > 64) return arg_error("width must be in [1, 64]");
    std::vector<uint32_t> mu(rows * width);
    for (size_t r = 0; r < rows; ++r)
      for (uint32_t b = 0; b < width; ++b) mu[r * width + b] = fsql::encode_bit((values[r] >> b) & 1u);
    return fsql_encrypt(ctx, mu.data(), mu.size(), stream, first_index, out);
  });
}

int fsql_phase(const fsql_ctx* ctx, const uint32_t* ct, size_t count, uint32_t* out) {
  if (!ctx || (count && (!ct || !out))) return arg_error("null argument");
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  const uint32_t n = c->p.n;
  for (size_t k = 0; k < count; ++k) {
    const uint32_t* v = ct + k * (n + 1);
    uint32_t dot = 0;
    for (uint32_t x = 0; x < n; ++x) dot += c->s[x] ? v[x] : 0u;
    out[k] = v[n] - dot;
  }
  return FSQL_OK;
}

int fsql_decrypt_bits(const fsql_ctx* ctx, const uint32_t* ct, size_t count, uint8_t* out) {
  return guarded([&]() -> int {
    if (!ctx || (count && (!ct || !out))) return arg_error("null argument");
    std::vector<uint32_t> ph(count);
    const int rc = fsql_phase(ctx, ct, count, ph.data());
    if (rc) return rc;
    for (size_t k = 0; k < count; ++k) out[k] = static_cast<int32_t>(ph[k]) > 0 ? 1 : 0;
    return FSQL_OK;
  });
}

int fsql_decrypt_uint(const fsql_ctx* ctx, const uint32_t* ct, size_t rows, uint32_t width, uint64_t* out) {
  return guarded([&]() -> int {
    if (!ctx || (rows && (!ct || !out))) return arg_error("null argument");
    if (width < 1 || width > 64) return arg_error("width must be in [1, 64]");
    std::vector<uint8_t> bits(rows * width);
    const int rc = fsql_decrypt_bits(ctx, ct, bits.size(), bits.data());
    if (rc) return rc;
    for (size_t r = 0; r < rows; ++r) {
      uint64_t v = 0;
      for (uint32_t b = 0; b < width; ++b) v |= static_cast<uint64_t>(bits[r * width + b]) << b;
      out[r] = v;
    }
    return FSQL_OK;
  });
}

int fsql_plan_info(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width,
                   uint32_t* gates_per_row, uint32_t* levels, uint32_t* level_widths, uint32_t max_levels) {
  return guarded([&]() -> int {
    fsql::Netlist nl;
    if (!fsql::build_netlist(pred, width, n_payloads, payload_width, &nl)) return arg_error("bad predicate shape");
    if (gates_per_row) *gates_per_row = static_cast<uint32_t>(nl.type.size());
    if (levels) *levels = static_cast<uint32_t>(nl.levels);
    if (level_widths) {
      for (uint32_t k = 0; k < max_levels; ++k) level_widths[k] = 0;
      for (int lv : nl.level)
        if (static_cast<uint32_t>(lv) <= max_levels) level_widths[lv - 1]++;
    }
    return FSQL_OK;
  });
}

int fsql_sum_plan_info(size_t rows, uint32_t width, uint32_t out_width, uint32_t* gates, uint32_t* levels,
                       uint32_t* literal_outputs) {
  return guarded([&]() -> int {
    fsql::Netlist nl;
    if (!fsql::build_sum_netlist(rows, width, out_width, &nl)) return arg_error("bad aggregation shape");
    if (gates) *gates = static_cast<uint32_t>(nl.type.size());
    if (levels) *levels = static_cast<uint32_t>(nl.levels);
    if (literal_outputs) *literal_outputs = static_cast<uint32_t>(nl.literal_outs.size());
    return FSQL_OK;
  });
}

int fsql_extreme_plan_info(int is_min, size_t rows, uint32_t width, uint32_t* gates, uint32_t* levels) {
  return guarded([&]() -> int {
    fsql::Netlist nl;
    if (!fsql::build_extreme_netlist(is_min != 0, rows, width, &nl)) return arg_error("bad aggregation shape");
    if (gates) *gates = static_cast<uint32_t>(nl.type.size());
    if (levels) *levels = static_cast<uint32_t>(nl.levels);
    return FSQL_OK;
  });
}

int fsql_plan_info_plain(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width,
                         const uint64_t* consts, uint32_t* gates_per_row, uint32_t* levels, uint32_t* level_widths,
                         uint32_t max_levels, uint32_t* literal_outputs) {
  return guarded([&]() -> int {
    if (!consts) return arg_error("null constants");
    const bool range = pred == FSQL_RANGE || pred == FSQL_RANGE_MAJ;
    const uint64_t k0 = consts[0], k1 = range ? consts[1] : 0;
    if (width >= 1 && width < 64 && (k0 >> width || k1 >> width)) return arg_error("constant wider than the column");
    fsql::Netlist nl;
    if (!fsql::build_netlist_plain(pred, width, n_payloads, payload_width, k0, k1, &nl))
      return arg_error("bad predicate shape");
    if (gates_per_row) *gates_per_row = static_cast<uint32_t>(nl.type.size());
    if (levels) *levels = static_cast<uint32_t>(nl.levels);
    if (level_widths) {
      for (uint32_t k = 0; k < max_levels; ++k) level_widths[k] = 0;
      for (int lv : nl.level)
        if (static_cast<uint32_t>(lv) <= max_levels) level_widths[lv - 1]++;
    }
    if (literal_outputs) *literal_outputs = static_cast<uint32_t>(nl.literal_outs.size());
    return FSQL_OK;
  });
}

}  // extern "C"
