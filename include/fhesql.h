/*
 * fhesql.h -- C interface of the B300 (sm_103a) engine for the oblivious
 * scan-select of FHE-SQL (arXiv 2510.15413).
 *
 * The paper's server (Alg. 2, ProcessQuery) evaluates the WHERE predicate of a
 * query homomorphically on every encrypted row, collects the encrypted mask
 * bits, and applies them to the selected columns with a homomorphic
 * If-Then-Else so that non-matching rows become encryptions of zero (§4.2;
 * §6.1 D, eq. (1)-(3)).  The client (Alg. 1) encrypts the query constants and
 * decrypts the result.  FHE is the TFHE scheme the paper cites (§1, §2.2):
 * here one LWE ciphertext per bit, every binary gate one gate bootstrap.
 *
 * Conventions shared by every call:
 *   - A ciphertext is n+1 uint32 words (a_0 .. a_{n-1}, b), body last, a
 *     Torus32 value mod 2^32; phase = b - sum a_i s_i.  A bit is encoded as
 *     +2^29 (true) or -2^29 (false).
 *   - Multi-bit values are [rows][width][n+1], bit 0 (LSB) first.
 *   - Pointers named d_* are device pointers (any allocator, e.g. PyTorch's
 *     caching allocator) owned by the caller; the library never frees them.
 *     Pointers named h_* or without prefix are host pointers.
 *   - Every call returns FSQL_OK (0) or an FSQL_ERR_* code and never throws;
 *     fsql_last_error() gives a message for the calling thread.  Argument
 *     checks are synchronous.  Device work is asynchronous on the given
 *     cudaStream_t (passed as void*, NULL = legacy default stream); a CUDA
 *     launch failure is reported by the call that launched it, a fault
 *     during execution by the next synchronising call.
 *   - One context must be driven from one stream at a time: its scratch and
 *     plan buffers are reused by the next call on the same context.
 */
#ifndef FHESQL_H
#define FHESQL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FSQL_API __attribute__((visibility("default")))
#else
#define FSQL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define FSQL_OK 0
#define FSQL_ERR_ARG 1         /* bad argument (null pointer, size, enum) */
#define FSQL_ERR_OOM 2         /* device or host allocation failed */
#define FSQL_ERR_CUDA 3        /* a CUDA runtime call failed */
#define FSQL_ERR_TIMEOUT 4     /* a bounded device wait gave up */
#define FSQL_ERR_ADMISSION 5   /* serving: request does not fit the memory budget */
#define FSQL_ERR_UNSUPPORTED 6 /* parameters outside what the kernels implement */

/* Gate types of the bootstrapped gates.  ANDNY(a,b) = (not a) and b,
 * ANDYN(a,b) = a and (not b), ORNY(a,b) = (not a) or b, ORYN(a,b) = a or (not b).
 * NOT needs no bootstrap (negate every word) and has no code here. */
#define FSQL_NAND 0
#define FSQL_AND 1
#define FSQL_OR 2
#define FSQL_XOR 3
#define FSQL_XNOR 4
#define FSQL_NOR 5
#define FSQL_ANDNY 6
#define FSQL_ANDYN 7
#define FSQL_ORNY 8
#define FSQL_ORYN 9
/* Three-input gates, used only inside scan and aggregation circuits (not by
 * fsql_gate_batch).  MAJNYY(a, b, c) = majority of (not a, b, c): one
 * bootstrap of -a + b + c.  XOR3(a, b, c) = a xor b xor c: one bootstrap of
 * -2(a + b + c) (t true inputs give phase -(2t - 3) q/4, positive iff t is
 * odd).  MAJ(a, b, c) = majority: one bootstrap of a + b + c.  XOR3 and MAJ
 * are the sum and carry of a full adder. */
#define FSQL_MAJNYY 10
#define FSQL_XOR3 11
#define FSQL_MAJ 12

/* Predicates of the WHERE clause (§4.2 B: equality and comparison).
 * EQ: c = k.  LT: c < k (unsigned).  RANGE: lo <= c < hi (unsigned).
 * LT and RANGE use an LSB-first ripple comparator of 4w - 3 gates;
 * LT_MAJ and RANGE_MAJ compute the same predicates with a majority chain of
 * w gates per comparator (lt_i = MAJ(not c_i, k_i, lt_{i-1})), not in the
 * paper: different gates, hence different output words, same plaintext. */
#define FSQL_EQ 0
#define FSQL_LT 1
#define FSQL_RANGE 2
#define FSQL_LT_MAJ 3
#define FSQL_RANGE_MAJ 4

/* TFHE parameters.  Torus32; GLWE dimension k = 1.  The GPU kernels
 * implement N = 1024, l = 3, 2 <= bg_bits <= 10, ks_base_bits = 2, ks_t = 8
 * and n <= 639; other values are accepted by the host-side calls only. */
typedef struct fsql_params {
    uint32_t n;            /* LWE dimension */
    uint32_t N;            /* GLWE polynomial size */
    uint32_t bg_bits;      /* log2 bootstrap gadget base */
    uint32_t l;            /* bootstrap gadget levels */
    uint32_t ks_base_bits; /* log2 keyswitch base */
    uint32_t ks_t;         /* keyswitch levels */
    double lwe_sigma;      /* LWE noise std-dev as a fraction of the torus */
    double glwe_sigma;     /* GLWE noise std-dev as a fraction of the torus */
} fsql_params;

typedef struct fsql_ctx fsql_ctx;

/* Exact NTT engines of the blind rotation (results are identical words; only
 * speed differs).  GOLDILOCKS: one prime p = 2^64 - 2^32 + 1.  DUAL_PRIME:
 * two primes below 2^29 with 32-bit Montgomery arithmetic and a CRT lift.
 * DEFAULT picks the faster one on B300 (DUAL_PRIME). */
#define FSQL_ENGINE_DEFAULT (-1)
#define FSQL_ENGINE_GOLDILOCKS 0
#define FSQL_ENGINE_DUAL_PRIME 1

/* Default parameter set: n=630, N=1024, base 2^7 x 3, keyswitch base 4 x 8,
 * sigma 2^-15 (LWE) and 2^-25 (GLWE). */
FSQL_API int fsql_params_default(fsql_params* out);
/* Toy parameter set (n=16, N=64) for host-side tests; not runnable on the GPU. */
FSQL_API int fsql_params_toy(fsql_params* out);

/* Key generation (KeyGen of §2.2) from one 64-bit seed, with the SplitMix64
 * generator (Steele, Lea & Flood 2014): stream 0 LWE key bits, 1 GLWE key
 * bits, 2 bootstrapping key, 3 keyswitching key.  The secret keys stay in
 * host memory (client side); the bootstrapping key is converted to the NTT
 * domain and, with the keyswitching key, uploaded to `device` (-1 = no
 * device: host-side calls only).  On success *out owns all of it. */
FSQL_API int fsql_ctx_create(const fsql_params* params, uint64_t seed, int device, fsql_ctx** out);
/* As fsql_ctx_create with an explicit NTT engine (FSQL_ENGINE_*). */
FSQL_API int fsql_ctx_create_engine(const fsql_params* params, uint64_t seed, int device, int engine,
                                    fsql_ctx** out);
FSQL_API int fsql_ctx_engine(const fsql_ctx* ctx, int* engine);
/* Launch shape of the blind rotation for batches of at least two gates per
 * SM (smaller batches always run one gate per CTA).  Results never depend
 * on it.  Shapes (index: kernel, gates per CTA, gadget rows per step, slots
 * of the key-staging ring):
 *   0-3: packed kernel (each 128-thread group holds both primes' residues of
 *        a gate, or the 64-bit prime's), 1-4 gates per CTA, 2 rows per step
 *        (two-prime engine) or 1 (Goldilocks engine, which offers 0, 1, 3);
 *   4: prime-split kernel (two-prime engine: a gate is 256 threads, the two
 *      primes' transforms on separate warps), 2 gates, 2 rows, 2 slots;
 *   5: prime-split, 2 gates, 2 rows, 3 slots;
 *   6: prime-split, 3 gates, 2 rows, 2 slots;
 *   7: prime-split, 2 gates, 3 rows, 2 slots;
 *   8: packed kernel, 3 gates, 2 rows, one key slot per gate group (the
 *      groups of a CTA then run without a CTA-wide barrier per step).
 * fsql_ctx_set_br_gates(g) selects the packed shape g - 1 (g = 1..4). */
#define FSQL_BR_SHAPES 9
FSQL_API int fsql_ctx_set_br_shape(fsql_ctx* ctx, int shape);
FSQL_API int fsql_ctx_br_shape(const fsql_ctx* ctx, int* shape);
FSQL_API int fsql_br_shape_info(int shape, int* kind, int* gates_per_cta, int* rows_per_step, int* stages);
FSQL_API int fsql_ctx_set_br_gates(fsql_ctx* ctx, int gates_per_cta);
FSQL_API int fsql_ctx_br_gates(const fsql_ctx* ctx, int* gates_per_cta);
/* Latency mode for batches smaller than two gates per SM (two-prime
 * engine).  0: one gate per 128-thread CTA.  1: one gate per CTA of three
 * 128-thread groups that run the three gadget-row steps of every CMux side
 * by side.  2 (default): one gate per thread-block cluster of six CTAs on six
 * SMs (each one prime and two gadget rows; partial sums and residues pushed
 * into the other CTAs' shared memory, two cluster barriers per CMux), used
 * while every gate of the batch gets a cluster of its own at once, mode 1
 * above that.  In modes 1 and 2, batches of more than one and at most two
 * gates per SM run as one wave of two-gate CTAs of the packed kernel.  The
 * output words are the same in every mode.  FSQL_ERR_ARG for other values. */
FSQL_API int fsql_ctx_set_latency_mode(fsql_ctx* ctx, int on);

/* Device level walker for batched scans (two-prime engine, packed launch
 * shapes with 2 or 3 gates per CTA; off by default).  When on, a scan whose every
 * circuit level holds at least two gates per SM runs as ONE cooperative
 * launch (one CTA per SM) that walks the levels on the device: per level,
 * the CTAs bootstrap its gates, meet at a grid barrier, keyswitch them, and
 * meet again (Alg. 2 evaluates each row's tree level by level).  Each
 * barrier wait gives up after timeout_ms of device time (default 2000): the
 * kernel then raises an error word and every CTA returns, leaving the
 * context usable; fsql_walk_status reports it.  Results are bit-identical
 * to the per-level launches.  Errors: FSQL_ERR_ARG (timeout not in
 * (0, 600000]). */
FSQL_API int fsql_ctx_set_walk(fsql_ctx* ctx, int on, double timeout_ms);
/* Synchronises `stream`, then FSQL_ERR_TIMEOUT if a walker launch on this
 * context since its last scan started timed out at a grid barrier
 * (*barrier = its index, may be NULL), else FSQL_OK. */
FSQL_API int fsql_walk_status(fsql_ctx* ctx, void* stream, unsigned int* barrier);
/* Test hook: CTA `block` of later walker launches never arrives at a grid
 * barrier (-1: off), so the waits of the others run out of time. */
FSQL_API int fsql_debug_walk_skip_block(fsql_ctx* ctx, int block);

/* Autotuner: times the blind rotation of `probe_gates` synthetic gates
 * (0 = 48 x SMs, a whole number of waves of every shape; at least 2 x SMs,
 * at most 2^20) for every launch shape the
 * context's engine offers (kernel, gates per CTA, gadget rows per step,
 * staging depth), keeps the fastest in the context and in a per-process
 * table keyed by (device, engine), and returns the chosen shape index and
 * the timings (ms per shape index, -1 where not offered) in
 * ms_out[FSQL_BR_SHAPES] (may be NULL).  Synchronises `stream`; allocates
 * its probe buffers for the duration of the call.  A later context on the
 * same device and engine starts from the tuned shape. */
FSQL_API int fsql_autotune(fsql_ctx* ctx, size_t probe_gates, void* stream, int* best_shape, double* ms_out);
FSQL_API void fsql_ctx_destroy(fsql_ctx* ctx);
FSQL_API int fsql_ctx_params(const fsql_ctx* ctx, fsql_params* out);
/* Device bytes held by the context for keys (bootstrapping key in the NTT
 * domain + keyswitching key) and for scratch currently allocated. */
FSQL_API int fsql_ctx_device_bytes(const fsql_ctx* ctx, size_t* key_bytes, size_t* scratch_bytes);

/* Copy keys out to host buffers (any may be NULL): lwe_key [n] bits,
 * glwe_key [N] bits, bk [n][2l][2][N] standard domain (row u*l+j-1 holds
 * GLWE(0) + s_i * 2^(32-bg*j) on polynomial u: 0 = mask, 1 = body),
 * ksk [N][ks_t][2^ks_base_bits - 1][n+1] = LWE_s(v * S_i * 2^(32-kb*(j+1))). */
FSQL_API int fsql_export_keys(const fsql_ctx* ctx, uint8_t* lwe_key, uint8_t* glwe_key, uint32_t* bk, uint32_t* ksk);

/* ---------------- client side (host memory; Alg. 1 EncryptQuery / Decrypt) ---------------- */

/* Encrypt `count` torus messages.  Ciphertext c draws SplitMix64 words
 * (first_index + c) * (n + 2) .. + n + 1 of `stream` (mask, then two for
 * Box-Muller noise), so chunks encrypt identically to one big call. */
FSQL_API int fsql_encrypt(const fsql_ctx* ctx, const uint32_t* mu, size_t count, uint64_t stream, uint64_t first_index,
                 uint32_t* out);
/* Encrypt bits (0/1 bytes) as -q/8 / +q/8. */
FSQL_API int fsql_encrypt_bits(const fsql_ctx* ctx, const uint8_t* bits, size_t count, uint64_t stream,
                      uint64_t first_index, uint32_t* out);
/* Encrypt `rows` unsigned values of `width` bits (1..64) into [rows][width][n+1];
 * ciphertext index of (row, bit) is first_index + row*width + bit. */
FSQL_API int fsql_encrypt_uint(const fsql_ctx* ctx, const uint64_t* values, size_t rows, uint32_t width, uint64_t stream,
                      uint64_t first_index, uint32_t* out);
/* Phases b - <a, s> of `count` ciphertexts. */
FSQL_API int fsql_phase(const fsql_ctx* ctx, const uint32_t* ct, size_t count, uint32_t* out);
/* Decrypt bits: 1 when the phase read as int32 is positive. */
FSQL_API int fsql_decrypt_bits(const fsql_ctx* ctx, const uint32_t* ct, size_t count, uint8_t* out);
/* Decrypt [rows][width][n+1] into unsigned values. */
FSQL_API int fsql_decrypt_uint(const fsql_ctx* ctx, const uint32_t* ct, size_t rows, uint32_t width, uint64_t* out);

/* Keyswitch-first order (the order of TFHE-rs, which the paper uses, §2.2):
 * ciphertexts of N + 1 words under the N-bit key (the GLWE key read as an
 * LWE key), fresh ones with the GLWE noise; ciphertext c of a stream draws
 * words c (N + 2) .. c (N + 2) + N + 1.  Layouts as fsql_encrypt_bits /
 * fsql_decrypt_bits with N + 1 words per ciphertext. */
FSQL_API int fsql_encrypt_big_bits(const fsql_ctx* ctx, const uint8_t* bits, size_t count, uint64_t stream,
                                   uint64_t first_index, uint32_t* out);
FSQL_API int fsql_decrypt_big_bits(const fsql_ctx* ctx, const uint32_t* ct, size_t count, uint8_t* out);

/* ---------------- server side (device memory, asynchronous on `stream`) ---------------- */

/* Gate bootstraps of `count` independent gates: out[g] = gate types[g] of
 * (a[g], b[g]).  d_types: uint8 [count]; d_a, d_b, d_out: [count][n+1].
 * Steps: linear combination, modulus switch, blind rotation (n CMux external
 * products through an exact negacyclic NTT: by default over two primes
 * below 2^28 with a CRT lift, or over p = 2^64 - 2^32 + 1 with the
 * Goldilocks engine), sample extraction, keyswitch.  d_out may alias neither input.  Types must be FSQL_NAND ..
 * FSQL_ORYN (a device array is not checked: other values compute ORYN). */
FSQL_API int fsql_gate_batch(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a, const uint32_t* d_b,
                    uint32_t* d_out, size_t count, void* stream);

/* fsql_gate_batch for callers that must not allocate device memory.  The
 * paper has no counterpart: this exists for host programs that hand the whole
 * GPU to their own allocator (for example a caching allocator that reserved
 * it up front) or that cannot afford the device-wide synchronisation and
 * possible failure of a cudaMalloc in the middle of a query, and so cannot
 * let fsql_gate_batch grow the context's scratch.  Same arguments and result
 * as fsql_gate_batch (bit-identical outputs), at most 1024 gates per call
 * (FSQL_ERR_ARG above that).  Its scratch is a fixed 4 MiB array compiled
 * into the library, which every GPU that loads the library keeps until the
 * process exits; the call allocates nothing.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture.  All calls on one GPU share the
 * array: calls that can overlap on the GPU (other streams, other contexts on
 * the same device) race and must be ordered by the caller.  Its launches are
 * timed by fsql_profile_begin/end like fsql_gate_batch's; it always uses the
 * single-pass keyswitch (small batches of fsql_gate_batch split theirs over
 * more CTAs for latency; the words are the same). */
FSQL_API int fsql_gate_batch_noalloc(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a, const uint32_t* d_b,
                                     uint32_t* d_out, size_t count, void* stream);

/* The two halves of fsql_gate_batch, exposed for tests and profiling.
 * fsql_blind_rotate_extract writes, per gate, the extracted sample of
 * dimension N under the GLWE key: d_big [count][N+1]. */
FSQL_API int fsql_blind_rotate_extract(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a, const uint32_t* d_b,
                              uint32_t* d_big, size_t count, void* stream);
/* LWE keyswitch N -> n: d_big [count][N+1] -> d_out [count][n+1]. */
FSQL_API int fsql_keyswitch(fsql_ctx* ctx, const uint32_t* d_big, uint32_t* d_out, size_t count, void* stream);

/* Exact negacyclic product through the device NTT, for tests: out = d * a in
 * Z[X]/(X^N+1) mod 2^32, where d_digits holds N signed values in
 * [-2^(bg-1), 2^(bg-1)) and d_poly N uint32 coefficients. */
FSQL_API int fsql_debug_ntt_mul(fsql_ctx* ctx, const int32_t* d_digits, const uint32_t* d_poly, uint32_t* d_out,
                       void* stream);

/* Number of gate bootstraps per row and the level widths of the predicate
 * netlist (the circuit scheduler's lowering): *gates_per_row, *levels, and,
 * if level_widths is non-NULL, up to max_levels per-row gate counts. */
FSQL_API int fsql_plan_info(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width,
                   uint32_t* gates_per_row, uint32_t* levels, uint32_t* level_widths, uint32_t max_levels);

/* Oblivious scan-select (Alg. 2 ProcessQuery over all rows; §4.2).
 * d_column: [rows][width][n+1] encrypted column; d_const: the encrypted
 * constant bits ([width][n+1] for EQ/LT/LT_MAJ, lo then hi [2*width][n+1]
 * for RANGE/RANGE_MAJ); d_payloads: host array of n_payloads device pointers, each
 * [rows][payload_width][n+1].  Outputs: d_match [rows][n+1] the encrypted
 * predicate bit of each row; d_out_payloads: host array of n_payloads device
 * pointers [rows][payload_width][n+1] = AND(match, payload bit), i.e. the
 * payload where the row matches and an encryption of 0 elsewhere.  Every row
 * runs the same gates: the work depends only on the sizes.  Outputs may not
 * alias inputs.  per_gate != 0 launches one gate per kernel launch (the plain
 * baseline); otherwise each circuit level runs as batched launches, and
 * the launch sequence of a scan is captured once as a CUDA graph (on a
 * stream of the context) and replayed on `stream` by later calls with the
 * same buffers and shape (plain launches while fsql_profile is recording). */
FSQL_API int fsql_scan_select(fsql_ctx* ctx, const uint32_t* d_column, size_t rows, uint32_t width, uint32_t pred,
                     const uint32_t* d_const, uint32_t n_payloads, const uint32_t* const* d_payloads,
                     uint32_t payload_width, uint32_t* d_match, uint32_t* const* d_out_payloads, int per_gate,
                     void* stream);

/* Oblivious scan-select with plaintext query constants (§4.2 lets an
 * operand of the comparison be a plaintext; §6.1 D times trivially
 * encrypted operands).  consts: HOST array, consts[0] = k for EQ/LT/LT_MAJ,
 * consts[0] = lo and consts[1] = hi for RANGE/RANGE_MAJ; each must fit in
 * width bits (else FSQL_ERR_ARG).  The server then knows every constant bit
 * and reduces the circuit: XNOR with a known bit is the column bit or its
 * negation (no bootstrap), so EQ takes width-1 AND gates per row; a
 * comparator step with known k_i is one AND or OR gate, or none while the
 * running result is a known bit (LT and LT_MAJ give the same circuit).
 * Outputs that no gate writes are copies or negations (every word negated)
 * of input ciphertexts, or the trivial ciphertext (0, .., 0, +-q/8) of a
 * known bit.  The gates, hence the work, depend on the constant's bits: the
 * constant is not hidden from the server in this variant.  Other arguments,
 * layouts and the graph replay are those of fsql_scan_select. */
FSQL_API int fsql_scan_select_plain(fsql_ctx* ctx, const uint32_t* d_column, size_t rows, uint32_t width,
                                    uint32_t pred, const uint64_t* consts, uint32_t n_payloads,
                                    const uint32_t* const* d_payloads, uint32_t payload_width, uint32_t* d_match,
                                    uint32_t* const* d_out_payloads, int per_gate, void* stream);

/* fsql_plan_info for the plaintext-constant circuit of consts (host array as
 * in fsql_scan_select_plain); *literal_outputs (if non-null) receives the
 * outputs per row that no gate writes. */
FSQL_API int fsql_plan_info_plain(uint32_t pred, uint32_t width, uint32_t n_payloads, uint32_t payload_width,
                                  const uint64_t* consts, uint32_t* gates_per_row, uint32_t* levels,
                                  uint32_t* level_widths, uint32_t max_levels, uint32_t* literal_outputs);

/* SUM aggregation of selected rows (§6.1 D: the masked values of a scan
 * summed homomorphically into one value; rows that do not match were masked
 * to zero).  d_values: [rows][width][n+1] encrypted unsigned values (LSB
 * first), e.g. one d_out_payloads column of fsql_scan_select; d_out:
 * [out_width][n+1] receives the encrypted sum mod 2^out_width (out_width >=
 * width + ceil(log2 rows) keeps it exact).  Circuit: a carry-save tree of
 * full adders (XOR3 sum, MAJ carry; one bootstrap each) reduces every bit
 * column to at most two wires, then one ripple-carry adder; per layer, each
 * column's wires are taken in order in groups of three, sums stay in the
 * column and carries move to the next (dropped above out_width), with the
 * 0-2 leftover wires after them.  About 2 rows x width bootstraps; depth
 * about log_1.5(rows) + out_width levels.  Outputs that are inputs or known
 * zeros (one row, high bits) are copies or trivial ciphertexts.  The
 * context keeps the circuit's scratch (intermediate wires, descriptors) per
 * argument set and replays its launches as a CUDA graph.  Limits: rows <=
 * 2^22, rows x width <= 2^24, 1 <= width, out_width <= 64.  d_out may not
 * alias d_values. */
FSQL_API int fsql_aggregate_sum(fsql_ctx* ctx, const uint32_t* d_values, size_t rows, uint32_t width,
                                uint32_t out_width, uint32_t* d_out, void* stream);

/* MAX and MIN of selected rows (§4.2 B lists max(a, b) and min(a, b)
 * among the operators of the homomorphic expression tree).  d_values:
 * [rows][width][n+1] unsigned values (LSB first); d_out: [width][n+1].
 * MAX takes masked values as they are (an unselected row masked to 0 cannot
 * win); MIN also takes d_match [rows][n+1], the rows' encrypted match bits,
 * and first sets every bit of an unselected row to 1 (ORYN(v, m)).  Circuit:
 * a tournament pairing neighbours (an unpaired last value moves on); each
 * pair costs width gates of a majority comparator s = [a < b] and 3 width
 * gates of multiplexers OR(AND(s, x), ANDNY(s, y)).  MAX: 4 width (rows-1)
 * bootstraps; MIN: width more per row.  No rows: MAX = 0, MIN = 2^width - 1
 * as trivial ciphertexts.  Plans, scratch and graph replay as
 * fsql_aggregate_sum (one aggregation plan per context is kept).  Limits:
 * rows <= 2^22, rows x width <= 2^24, 1 <= width <= 64. */
FSQL_API int fsql_aggregate_max(fsql_ctx* ctx, const uint32_t* d_values, size_t rows, uint32_t width,
                                uint32_t* d_out, void* stream);
FSQL_API int fsql_aggregate_min(fsql_ctx* ctx, const uint32_t* d_values, const uint32_t* d_match, size_t rows,
                                uint32_t width, uint32_t* d_out, void* stream);
/* Gate and level counts of the MAX (is_min = 0) or MIN circuit. */
FSQL_API int fsql_extreme_plan_info(int is_min, size_t rows, uint32_t width, uint32_t* gates, uint32_t* levels);

/* Gate count and level count of the SUM circuit for (rows, width, out_width). */
FSQL_API int fsql_sum_plan_info(size_t rows, uint32_t width, uint32_t out_width, uint32_t* gates, uint32_t* levels,
                                uint32_t* literal_outputs);

/* Gates and scans in keyswitch-first order: every input and output is
 * N + 1 words under the N-bit key.  A gate forms its linear combination on
 * N + 1 words, keyswitches that one result to the n-bit key (the keyswitch
 * before the bootstrap instead of after it), bootstraps it and writes the
 * extracted sample.  Trades larger ciphertexts (4100 B instead of 2524 B per
 * bit) for keyswitching once per gate of the combination rather than once
 * per stored output.  Arguments otherwise as fsql_gate_batch and
 * fsql_scan_select (encrypted constants; d_const [width or 2 width][N+1]). */
FSQL_API int fsql_gate_batch_ks_first(fsql_ctx* ctx, const uint8_t* d_types, const uint32_t* d_a,
                                      const uint32_t* d_b, uint32_t* d_out, size_t count, void* stream);
FSQL_API int fsql_scan_select_ks_first(fsql_ctx* ctx, const uint32_t* d_column, size_t rows, uint32_t width,
                                       uint32_t pred, const uint32_t* d_const, uint32_t n_payloads,
                                       const uint32_t* const* d_payloads, uint32_t payload_width,
                                       uint32_t* d_match, uint32_t* const* d_out_payloads, int per_gate,
                                       void* stream);

/* The same scan from host buffers (layouts as above, h_payloads / h_out_payloads
 * are arrays of host pointers): copies inputs to the device, runs the batched
 * scan, copies the outputs back and synchronises `stream` before returning.
 * Device staging buffers are owned by the context and reused. */
FSQL_API int fsql_scan_select_host(fsql_ctx* ctx, const uint32_t* h_column, size_t rows, uint32_t width, uint32_t pred,
                          const uint32_t* h_const, uint32_t n_payloads, const uint32_t* const* h_payloads,
                          uint32_t payload_width, uint32_t* h_match, uint32_t* const* h_out_payloads, void* stream);

/* ---------------- serving: continuous batching of scan queries ---------------- */

/* One scan-select query for the server (the arguments of fsql_scan_select,
 * or of fsql_scan_select_plain when plain != 0; all pointers are device
 * pointers owned by the caller, which keeps them valid until the query is
 * done, failed or cancelled). */
#define FSQL_MAX_PAYLOADS 8
typedef struct fsql_query {
    const uint32_t* d_column;  /* [rows][width][n+1] */
    size_t rows;
    uint32_t width;
    uint32_t pred;             /* FSQL_EQ, FSQL_LT, FSQL_RANGE, FSQL_LT_MAJ, FSQL_RANGE_MAJ */
    const uint32_t* d_const;   /* [width or 2*width][n+1]; unused (may be null) when plain */
    uint32_t n_payloads;       /* <= FSQL_MAX_PAYLOADS */
    uint32_t payload_width;
    const uint32_t* d_payloads[FSQL_MAX_PAYLOADS];  /* each [rows][payload_width][n+1] */
    uint32_t* d_match;                              /* [rows][n+1] */
    uint32_t* d_out_payloads[FSQL_MAX_PAYLOADS];    /* each [rows][payload_width][n+1] */
    uint32_t plain;            /* nonzero: the constants are the plaintexts consts[] */
    uint32_t pad;
    uint64_t consts[2];        /* k, or lo and hi, each within width bits */
} fsql_query;

typedef struct fsql_server fsql_server;

/* Query states reported by fsql_server_status. */
#define FSQL_Q_WAITING 0   /* queued until its scratch fits the memory budget */
#define FSQL_Q_RUNNING 1   /* admitted: its gates join the server's launches */
#define FSQL_Q_DONE 2      /* outputs complete in device memory */
#define FSQL_Q_FAILED 3
#define FSQL_Q_CANCELLED 4

typedef struct fsql_server_stats {
    uint64_t completed;      /* queries done */
    uint64_t rounds;         /* launch rounds (one blind rotation + keyswitch pass each) */
    uint64_t gates;          /* gate bootstraps run */
    double busy_ms;          /* wall time spent in rounds */
    double p50_ms, p99_ms;   /* submit-to-done latency percentiles of completed queries */
    uint64_t waiting, running;
    size_t scratch_used;     /* bytes of the budget held by admitted queries */
} fsql_server_stats;

/* A server thread that runs the queries submitted to it (Alg. 2 for each,
 * §4.2 semantics) on the context's device.  Each round merges the
 * next circuit level of every admitted query into one launch pair of at
 * most max_batch_gates gate bootstraps (0 = 2^17).  A submitted query waits
 * until its device scratch (descriptors and intermediate wires, about
 * rows x gates_per_row x (32 + 2524) bytes) fits in scratch_budget_bytes,
 * which the server allocates once, and until the running queries' current
 * levels no longer fill an efficient round (64 gates per SM, or
 * max_batch_gates if smaller), so that under load queries finish closer to
 * arrival order instead of all sharing the GPU equally.  Results are bit-identical to
 * fsql_scan_select of the same query alone.  The context must not be
 * destroyed before the server. */
FSQL_API int fsql_server_create(fsql_ctx* ctx, size_t scratch_budget_bytes, size_t max_batch_gates,
                                fsql_server** out);
/* Queue a query; FSQL_ERR_ADMISSION if its scratch exceeds the whole budget.
 * The server runs on a stream of its own that does not wait for the
 * caller's streams: the query's inputs (and anything the caller still
 * writes into its output buffers) must be complete before this call, e.g.
 * by synchronising the stream that produced them. */
FSQL_API int fsql_server_submit(fsql_server* server, const fsql_query* query, uint64_t* id);
/* State (FSQL_Q_*) and, once done, the submit-to-done latency in ms (else -1). */
FSQL_API int fsql_server_status(fsql_server* server, uint64_t id, int* state, double* latency_ms);
/* Block until the query is done (FSQL_OK), failed (FSQL_ERR_CUDA) or
 * cancelled (FSQL_OK), or the timeout passes (FSQL_ERR_TIMEOUT). */
FSQL_API int fsql_server_wait(fsql_server* server, uint64_t id, double timeout_ms);
/* Drop a query: a waiting one is never run; a running one stops at the
 * next round boundary with its outputs incomplete. */
FSQL_API int fsql_server_cancel(fsql_server* server, uint64_t id);
FSQL_API int fsql_server_get_stats(fsql_server* server, fsql_server_stats* out);
/* Stops the server thread after its current round and frees its memory. */
FSQL_API void fsql_server_destroy(fsql_server* server);

/* Kernel timing with CUDA events, recorded on the launch stream around every
 * blind-rotation and keyswitch launch of this context between
 * fsql_profile_begin and fsql_profile_end (which waits for the recorded
 * events).  Durations are summed device times in milliseconds. */
typedef struct fsql_kernel_times {
    double blind_rotate_ms;
    double keyswitch_ms;
    uint64_t blind_rotate_launches;
    uint64_t keyswitch_launches;
    uint64_t gates;  /* gates bootstrapped by the recorded launches */
} fsql_kernel_times;
FSQL_API int fsql_profile_begin(fsql_ctx* ctx);
FSQL_API int fsql_profile_end(fsql_ctx* ctx, fsql_kernel_times* out);

/* Integer-ALU rates of this GPU, measured by short in-register
 * microkernels (no paper counterpart: the denominators of the blind
 * rotation's roofline).  Rates are operations per second over the whole GPU:
 * 32-bit multiply-add, high-half multiply-add, widening 32x32+64 multiply-add,
 * forward butterflies of the two-prime engine (one Shoup product by a twiddle
 * plus the lazy add and subtract; one 32-bit modular multiplication each) and
 * butterflies mod 2^64 - 2^32 + 1 (one 64-bit modular multiplication each).
 * Runs about half a second of kernels on `device` (the calling thread's
 * current device is changed to it); allocates 0.6 MB for the kernels'
 * outputs and frees it.  Errors: FSQL_ERR_ARG (null output, bad device),
 * FSQL_ERR_CUDA. */
typedef struct fsql_alu_peaks {
    double imad_per_s;
    double imad_hi_per_s;
    double imad_wide_per_s;
    double dual_prime_bfly_per_s;
    double goldilocks_bfly_per_s;
    double dual_prime_bfly_wide_per_s;    /* the quotient from a widening multiply's high word */
    double dual_prime_bfly_madwide_per_s; /* ... from a widening multiply-add */
    int sm_count;
    double clock_mhz;  /* the device's reported maximum SM clock */
} fsql_alu_peaks;
FSQL_API int fsql_measure_alu_peaks(int device, fsql_alu_peaks* out);

/* Message for the last failed call on this thread ("" if none). */
FSQL_API const char* fsql_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FHESQL_H */
