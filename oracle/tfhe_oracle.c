/*
 * tfhe_oracle.c -- plain, slow, CPU reference for the oblivious scan-select
 * of FHE-SQL (arXiv 2510.15413).  TEST INFRASTRUCTURE ONLY: it is linked by
 * the test-suite, by the package's smoke check and by the CPU-baseline leg of
 * the benchmark, never by the product path.  It shares no code, header or
 * table with the CUDA library; both sides only agree on the published
 * SplitMix64 generator, which each implements on its own.
 *
 * What it computes (every output word is a fixed function of seed and inputs):
 *   - the scan of Alg. 2 (ProcessQuery): per row, evaluate the WHERE
 *     predicate homomorphically into one encrypted mask bit, then apply the
 *     mask to the selected payload columns with If-Then-Else (§4.2, §6.1 D,
 *     eq. (1)-(3)); for one-bit payloads cmux(m, v, 0) is AND(m, v);
 *   - every binary gate is a TFHE gate bootstrap (the TFHE construction the
 *     paper cites in §1 and §2.2): linear combination, modulus switch, blind
 *     rotation of a GLWE accumulator by n CMux external products, sample
 *     extraction, LWE keyswitch;
 *   - polynomial products are exact negacyclic products over Z/2^32, by
 *     schoolbook or Karatsuba (no transform of any kind).
 *
 * Readings where the paper is silent (it delegates all of TFHE to a library):
 * bits are encoded as +-q/8, phase = b - <a,s>, gadget base 2^7 with 3 signed
 * digits in [-64,63], keyswitch base 4 with 8 unsigned digits, test vector
 * q/8 everywhere, rotation X^{-b} then X^{+a_i}, SplitMix64 randomness,
 * Box-Muller noise rounded half away from zero.  Each function below names the
 * reading it follows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

typedef struct {
    int32_t n;            /* LWE dimension */
    int32_t N;            /* GLWE polynomial size (power of two), k = 1 */
    int32_t bg_bits;      /* log2 of the bootstrap gadget base */
    int32_t l;            /* bootstrap gadget levels */
    int32_t ks_base_bits; /* log2 of the keyswitch base */
    int32_t ks_t;         /* keyswitch levels */
    double lwe_sigma;     /* LWE noise std-dev (fraction of the torus) */
    double glwe_sigma;    /* GLWE noise std-dev (fraction of the torus) */
} orc_params;

typedef struct {
    orc_params p;
    uint64_t seed;
    uint8_t *s;    /* LWE key, n bits */
    uint8_t *S;    /* GLWE key, N bits */
    uint32_t *bk;  /* [n][2l][2][N]: row r = u*l + (j-1), poly 0 = mask A, 1 = body B */
    uint32_t *ksk; /* [N][t][base-1][n+1]: LWE_s(v * S_i * 2^(32 - bb*(j+1))) */
} orc_ctx;

/* ------------------------------------------------------------------ */
/* Randomness: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).           */
/* The generator's state advances by the golden-ratio increment        */
/* gamma; each output is the state after k+1 increments, mixed.        */
/* word(seed, stream, ctr) = output #ctr of the generator whose start  */
/* state is output #stream of the generator started at seed.           */
/* ------------------------------------------------------------------ */
static uint64_t sm_output(uint64_t start, uint64_t k)
{
    uint64_t z = start + (k + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

ORC_API uint64_t orc_splitmix64(uint64_t start, uint64_t k) { return sm_output(start, k); }

static uint64_t rnd_word(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return sm_output(sm_output(seed, stream), ctr);
}

static uint32_t rnd_u32(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return (uint32_t)(rnd_word(seed, stream, ctr) >> 32);
}

/* Gaussian torus noise from two consecutive words: Box-Muller cosine branch,
 * then round half away from zero of sigma * z * 2^32, reduced mod 2^32. */
static uint32_t rnd_noise(uint64_t seed, uint64_t stream, uint64_t ctr, double sigma)
{
    uint64_t w1 = rnd_word(seed, stream, ctr);
    uint64_t w2 = rnd_word(seed, stream, ctr + 1);
    double u1 = (double)((w1 >> 11) + 1) * 0x1p-53; /* (0, 1] */
    double u2 = (double)(w2 >> 11) * 0x1p-53;       /* [0, 1) */
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    double t = sigma * z;
    long long e = llround(t * 4294967296.0);
    return (uint32_t)(uint64_t)e;
}

/* ------------------------------------------------------------------ */
/* Negacyclic polynomial products in Z[X]/(X^N + 1), coefficients      */
/* mod 2^32 (uint32 wrap-around is the ring Z/2^32).                   */
/* ------------------------------------------------------------------ */

/* Definition: c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j. */
ORC_API void orc_negacyclic_schoolbook(const uint32_t *a, const uint32_t *b, uint32_t *c, int N)
{
    for (int k = 0; k < N; k++) c[k] = 0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            uint32_t prod = a[i] * b[j];
            int k = i + j;
            if (k < N) c[k] += prod;
            else c[k - N] -= prod;
        }
}

/* Full product r[0..2m-2] (r[2m-1] = 0) of two length-m polys, schoolbook. */
static void full_school(const uint32_t *a, const uint32_t *b, uint32_t *r, int m)
{
    for (int k = 0; k < 2 * m; k++) r[k] = 0;
    for (int i = 0; i < m; i++) {
        uint32_t ai = a[i];
        for (int j = 0; j < m; j++) r[i + j] += ai * b[j];
    }
}

/* Full product by Karatsuba: a*b = z0 + (z1 - z0 - z2) X^h + z2 X^{2h},
 * z0 = a_lo b_lo, z2 = a_hi b_hi, z1 = (a_lo + a_hi)(b_lo + b_hi).
 * r has 2m slots, tmp has 8m slots. */
static void full_kara(const uint32_t *a, const uint32_t *b, uint32_t *r, int m, uint32_t *tmp)
{
    if (m <= 32) {
        full_school(a, b, r, m);
        return;
    }
    int h = m / 2;
    uint32_t *sa = tmp, *sb = tmp + h, *z1 = tmp + 2 * h, *rest = tmp + 4 * h;
    for (int i = 0; i < h; i++) {
        sa[i] = a[i] + a[i + h];
        sb[i] = b[i] + b[i + h];
    }
    full_kara(a, b, r, h, rest);                 /* z0 -> r[0 .. 2h-1]  */
    full_kara(a + h, b + h, r + 2 * h, h, rest); /* z2 -> r[2h .. 4h-1] */
    full_kara(sa, sb, z1, h, rest);              /* z1 -> z1[0 .. 2h-1] */
    for (int i = 0; i < 2 * h; i++) z1[i] -= r[i] + r[2 * h + i];
    for (int i = 0; i < 2 * h; i++) r[h + i] += z1[i];
}

/* Negacyclic product via Karatsuba, then fold X^N = -1. */
ORC_API void orc_negacyclic_karatsuba(const uint32_t *a, const uint32_t *b, uint32_t *c, int N)
{
    uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * 8 * N);
    full_kara(a, b, r, N, tmp);
    for (int k = 0; k < N; k++) c[k] = r[k] - r[k + N];
    free(r);
    free(tmp);
}

/* acc += a * b (negacyclic), using caller scratch r (2N) and tmp (8N). */
static void negacyclic_mac(const uint32_t *a, const uint32_t *b, uint32_t *acc, int N,
                           uint32_t *r, uint32_t *tmp)
{
    full_kara(a, b, r, N, tmp);
    for (int k = 0; k < N; k++) acc[k] += r[k] - r[k + N];
}

/* out = X^e * in in Z[X]/(X^N+1), e in [0, 2N): each coefficient moves up by e
 * places and changes sign every time it passes X^N. */
ORC_API void orc_monomial_mul(const uint32_t *in, uint32_t *out, int N, int e)
{
    for (int x = 0; x < N; x++) {
        int pos = x + e;
        uint32_t v = in[x];
        while (pos >= N) {
            pos -= N;
            v = (uint32_t)0 - v;
        }
        out[pos] = v;
    }
}

/* ------------------------------------------------------------------ */
/* Params and key generation                                            */
/* ------------------------------------------------------------------ */

ORC_API void orc_params_default(orc_params *p)
{
    p->n = 630;
    p->N = 1024;
    p->bg_bits = 7;
    p->l = 3;
    p->ks_base_bits = 2;
    p->ks_t = 8;
    p->lwe_sigma = 0x1p-15;
    p->glwe_sigma = 0x1p-25;
}

ORC_API void orc_params_toy(orc_params *p)
{
    p->n = 16;
    p->N = 64;
    p->bg_bits = 7;
    p->l = 3;
    p->ks_base_bits = 2;
    p->ks_t = 8;
    p->lwe_sigma = 0x1p-25;
    p->glwe_sigma = 0x1p-25;
}

static size_t bk_words(const orc_params *p) { return (size_t)p->n * 2 * p->l * 2 * p->N; }
static int ks_digits(const orc_params *p) { return (1 << p->ks_base_bits) - 1; }
static size_t ksk_words(const orc_params *p)
{
    return (size_t)p->N * p->ks_t * ks_digits(p) * (p->n + 1);
}

ORC_API size_t orc_bk_words(const orc_ctx *c) { return bk_words(&c->p); }
ORC_API size_t orc_ksk_words(const orc_ctx *c) { return ksk_words(&c->p); }
ORC_API const uint8_t *orc_lwe_key(const orc_ctx *c) { return c->s; }
ORC_API const uint8_t *orc_glwe_key(const orc_ctx *c) { return c->S; }
ORC_API const uint32_t *orc_bk(const orc_ctx *c) { return c->bk; }
ORC_API const uint32_t *orc_ksk(const orc_ctx *c) { return c->ksk; }

/* LWE encryption of torus message mu under key s (dimension n):
 * a_x uniform, e Gaussian, b = <a, s> + e + mu.  Randomness: words
 * [base, base+n) for the mask, [base+n, base+n+2) for the noise. */
static void lwe_encrypt(const uint8_t *s, int n, uint32_t mu, double sigma, uint64_t seed,
                        uint64_t stream, uint64_t base, uint32_t *ct)
{
    uint32_t dot = 0;
    for (int x = 0; x < n; x++) {
        ct[x] = rnd_u32(seed, stream, base + x);
        if (s[x]) dot += ct[x];
    }
    ct[n] = dot + rnd_noise(seed, stream, base + n, sigma) + mu;
}

/* Key generation.  Streams: 0 LWE key, 1 GLWE key, 2 bootstrapping key,
 * 3 keyswitching key.  Key bits are the top bit of one word each. */
ORC_API orc_ctx *orc_create(const orc_params *p, uint64_t seed)
{
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->p = *p;
    c->seed = seed;
    int n = p->n, N = p->N, l = p->l;
    c->s = (uint8_t *)malloc(n);
    c->S = (uint8_t *)malloc(N);
    for (int i = 0; i < n; i++) c->s[i] = (uint8_t)(rnd_word(seed, 0, i) >> 63);
    for (int j = 0; j < N; j++) c->S[j] = (uint8_t)(rnd_word(seed, 1, j) >> 63);

    /* Bootstrapping key: BK_i = GGSW_S(s_i).  Row r = (u, j): a GLWE
     * encryption of zero (A uniform, B = A*S + e), plus s_i * 2^(32 - bg*j)
     * on the constant coefficient of polynomial u (0 = A, 1 = B). */
    c->bk = (uint32_t *)malloc(sizeof(uint32_t) * bk_words(p));
#pragma omp parallel
    {
        uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
        uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * 8 * N);
        uint32_t *Spoly = (uint32_t *)malloc(sizeof(uint32_t) * N);
        for (int j = 0; j < N; j++) Spoly[j] = c->S[j];
#pragma omp for schedule(static)
        for (int R = 0; R < n * 2 * l; R++) {
            int i = R / (2 * l), row = R % (2 * l);
            int u = row / l, j = row % l + 1;
            uint64_t base = (uint64_t)R * 3 * N;
            uint32_t *A = c->bk + (size_t)R * 2 * N, *B = A + N;
            for (int x = 0; x < N; x++) A[x] = rnd_u32(seed, 2, base + x);
            for (int x = 0; x < N; x++) B[x] = rnd_noise(seed, 2, base + N + 2 * x, p->glwe_sigma);
            negacyclic_mac(A, Spoly, B, N, r, tmp);
            uint32_t g = (uint32_t)1u << (32 - p->bg_bits * j);
            if (c->s[i]) {
                if (u == 0) A[0] += g;
                else B[0] += g;
            }
        }
        free(r);
        free(tmp);
        free(Spoly);
    }

    /* Keyswitching key: KSK[i][j][v-1] = LWE_s(v * S_i * 2^(32 - kb*(j+1))),
     * v = 1 .. base-1, noise lwe_sigma. */
    int nd = ks_digits(p);
    c->ksk = (uint32_t *)malloc(sizeof(uint32_t) * ksk_words(p));
#pragma omp parallel for schedule(static)
    for (int idx = 0; idx < N * p->ks_t * nd; idx++) {
        int i = idx / (p->ks_t * nd);
        int j = (idx / nd) % p->ks_t;
        int v = idx % nd + 1;
        uint32_t mu = (uint32_t)v * (uint32_t)c->S[i] * ((uint32_t)1u << (32 - p->ks_base_bits * (j + 1)));
        lwe_encrypt(c->s, n, mu, p->lwe_sigma, seed, 3, (uint64_t)idx * (n + 2),
                    c->ksk + (size_t)idx * (n + 1));
    }
    return c;
}

ORC_API void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->s);
    free(c->S);
    free(c->bk);
    free(c->ksk);
    free(c);
}

/* Encrypt torus messages; ciphertext number first_index + c draws words
 * starting at (first_index + c) * (n + 2) of the given stream. */
ORC_API void orc_encrypt(const orc_ctx *c, const uint32_t *mu, size_t count, uint64_t stream,
                         uint64_t first_index, uint32_t *out)
{
    int n = c->p.n;
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)count; k++)
        lwe_encrypt(c->s, n, mu[k], c->p.lwe_sigma, c->seed, stream,
                    (first_index + (uint64_t)k) * (n + 2), out + (size_t)k * (n + 1));
}

/* Bit encoding: true -> +q/8, false -> -q/8. */
ORC_API void orc_encrypt_bits(const orc_ctx *c, const uint8_t *bits, size_t count, uint64_t stream,
                              uint64_t first_index, uint32_t *out)
{
    uint32_t *mu = (uint32_t *)malloc(sizeof(uint32_t) * (count ? count : 1));
    for (size_t k = 0; k < count; k++) mu[k] = bits[k] ? (1u << 29) : (uint32_t)(0u - (1u << 29));
    orc_encrypt(c, mu, count, stream, first_index, out);
    free(mu);
}

/* phase = b - <a, key> mod 2^32, for a ciphertext of dimension dim. */
static uint32_t lwe_phase(const uint32_t *ct, const uint8_t *key, int dim)
{
    uint32_t dot = 0;
    for (int x = 0; x < dim; x++)
        if (key[x]) dot += ct[x];
    return ct[dim] - dot;
}

ORC_API void orc_phase(const orc_ctx *c, const uint32_t *ct, size_t count, uint32_t *out)
{
    for (size_t k = 0; k < count; k++) out[k] = lwe_phase(ct + k * (c->p.n + 1), c->s, c->p.n);
}

/* Phase under the GLWE key read as an LWE key of dimension N (for extracted samples). */
ORC_API void orc_phase_big(const orc_ctx *c, const uint32_t *ct, size_t count, uint32_t *out)
{
    for (size_t k = 0; k < count; k++) out[k] = lwe_phase(ct + k * (c->p.N + 1), c->S, c->p.N);
}

/* Decryption: the bit is 1 when the phase, read as a signed 32-bit value, is positive. */
ORC_API void orc_decrypt_bits(const orc_ctx *c, const uint32_t *ct, size_t count, uint8_t *out)
{
    for (size_t k = 0; k < count; k++)
        out[k] = (int32_t)lwe_phase(ct + k * (c->p.n + 1), c->s, c->p.n) > 0;
}

/* ------------------------------------------------------------------ */
/* Gate bootstrap pieces                                                */
/* ------------------------------------------------------------------ */

/* Modulus switch q -> 2N: round(x * 2N / q) mod 2N, ties rounded up. */
ORC_API uint32_t orc_modswitch(uint32_t x, int N)
{
    uint64_t twoN = 2 * (uint64_t)N;
    return (uint32_t)((((uint64_t)x * twoN + (1ULL << 31)) >> 32) % twoN);
}

/* Signed gadget decomposition: round x to the nearest multiple of
 * 2^(32 - bg*l) (ties up), then write the rounded value, mod 2^(bg*l), in
 * balanced base 2^bg with digits in [-2^(bg-1), 2^(bg-1)), least significant
 * digit first, carrying into the next digit; the carry out of the top digit
 * wraps mod q.  digits[j-1] multiplies 2^(32 - bg*j). */
ORC_API void orc_decompose(uint32_t x, int bg_bits, int l, int32_t *digits)
{
    int drop = 32 - bg_bits * l;
    uint64_t v = (((uint64_t)x + (1ULL << (drop - 1))) >> drop) & ((1ULL << (bg_bits * l)) - 1);
    int64_t base = 1LL << bg_bits, half = base / 2;
    for (int j = l; j >= 1; j--) {
        int64_t d = (int64_t)(v % (uint64_t)base);
        v /= (uint64_t)base;
        if (d >= half) {
            d -= base;
            v += 1;
        }
        digits[j - 1] = (int32_t)d;
    }
}

/* Keyswitch digits: round x to its top kb*t bits (ties up), unsigned base-2^kb
 * digits, most significant first: x ~ sum_j d_j 2^(32 - kb*(j+1)). */
static void ks_decompose(uint32_t x, int kb, int t, int32_t *digits)
{
    int drop = 32 - kb * t;
    uint64_t v = (((uint64_t)x + (1ULL << (drop - 1))) >> drop) & ((1ULL << (kb * t)) - 1);
    for (int j = t - 1; j >= 0; j--) {
        digits[j] = (int32_t)(v & ((1u << kb) - 1));
        v >>= kb;
    }
}

/* External product BK_i [] (A, B): decompose both polynomials, then
 * out_c = sum over rows r = (u, j) of digitpoly(u, j) * BK_i[r][c]. */
static void external_product(const orc_ctx *c, const uint32_t *bki, const uint32_t *in,
                             uint32_t *out, uint32_t *scratch)
{
    int N = c->p.N, l = c->p.l;
    uint32_t *dig = scratch;                /* [2l][N] digit polys (two's complement) */
    uint32_t *r = dig + (size_t)2 * l * N;  /* 2N */
    uint32_t *tmp = r + 2 * N;              /* 8N */
    int32_t d[16];
    for (int u = 0; u < 2; u++)
        for (int x = 0; x < N; x++) {
            orc_decompose(in[u * N + x], c->p.bg_bits, l, d);
            for (int j = 0; j < l; j++) dig[(size_t)(u * l + j) * N + x] = (uint32_t)d[j];
        }
    memset(out, 0, sizeof(uint32_t) * 2 * N);
    for (int row = 0; row < 2 * l; row++)
        for (int cc = 0; cc < 2; cc++)
            negacyclic_mac(dig + (size_t)row * N, bki + ((size_t)row * 2 + cc) * N, out + cc * N, N, r, tmp);
}

static size_t ep_scratch_words(const orc_params *p) { return (size_t)2 * p->l * p->N + 10 * p->N; }

ORC_API void orc_external_product(const orc_ctx *c, int i, const uint32_t *in, uint32_t *out)
{
    uint32_t *scratch = (uint32_t *)malloc(sizeof(uint32_t) * ep_scratch_words(&c->p));
    external_product(c, c->bk + (size_t)i * 2 * c->p.l * 2 * c->p.N, in, out, scratch);
    free(scratch);
}

/* Blind rotation: ACC = X^{-b~} (0, v) with v_j = q/8 for every j, then for
 * each i: ACC <- ACC + BK_i [] (X^{a~_i} ACC - ACC).  Input is the LWE sample
 * of dimension n already linearly combined (mod q). */
ORC_API void orc_blind_rotate(const orc_ctx *c, const uint32_t *lwe, uint32_t *acc)
{
    int n = c->p.n, N = c->p.N;
    uint32_t *tv = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *rot = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
    uint32_t *prod = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
    uint32_t *scratch = (uint32_t *)malloc(sizeof(uint32_t) * ep_scratch_words(&c->p));
    for (int x = 0; x < N; x++) tv[x] = 1u << 29;
    uint32_t bbar = orc_modswitch(lwe[n], N);
    memset(acc, 0, sizeof(uint32_t) * N);
    orc_monomial_mul(tv, acc + N, N, (int)((2 * N - bbar) % (2 * N)));
    for (int i = 0; i < n; i++) {
        uint32_t abar = orc_modswitch(lwe[i], N);
        for (int u = 0; u < 2; u++) {
            orc_monomial_mul(acc + u * N, rot + u * N, N, (int)abar);
            for (int x = 0; x < N; x++) rot[u * N + x] -= acc[u * N + x];
        }
        external_product(c, c->bk + (size_t)i * 2 * c->p.l * 2 * N, rot, prod, scratch);
        for (int x = 0; x < 2 * N; x++) acc[x] += prod[x];
    }
    free(tv);
    free(rot);
    free(prod);
    free(scratch);
}

/* Sample extraction of coefficient 0: a'_0 = A_0, a'_j = -A_{N-j}, b' = B_0;
 * the result is an LWE sample of dimension N under the GLWE key's coefficients. */
ORC_API void orc_sample_extract(int N, const uint32_t *acc, uint32_t *out)
{
    out[0] = acc[0];
    for (int j = 1; j < N; j++) out[j] = (uint32_t)0 - acc[N - j];
    out[N] = acc[N];
}

/* Keyswitch from the N-bit key to the n-bit key:
 * out = (0, .., 0, b') - sum_{i, j} KSK[i][j][d_ij] (digit 0 contributes nothing). */
ORC_API void orc_keyswitch(const orc_ctx *c, const uint32_t *big, uint32_t *out)
{
    int n = c->p.n, N = c->p.N, t = c->p.ks_t, nd = ks_digits(&c->p);
    int32_t d[32];
    memset(out, 0, sizeof(uint32_t) * (n + 1));
    out[n] = big[N];
    for (int i = 0; i < N; i++) {
        ks_decompose(big[i], c->p.ks_base_bits, t, d);
        for (int j = 0; j < t; j++) {
            if (d[j] == 0) continue;
            const uint32_t *row = c->ksk + ((size_t)(i * t + j) * nd + (d[j] - 1)) * (n + 1);
            for (int x = 0; x <= n; x++) out[x] -= row[x];
        }
    }
}

/* Gate types (numbering fixed by the library's C interface). */
enum { G_NAND = 0, G_AND, G_OR, G_XOR, G_XNOR, G_NOR, G_ANDNY, G_ANDYN, G_ORNY, G_ORYN, G_MAJNYY, G_XOR3, G_MAJ,
       G_COUNT };

/* Linear combination before the bootstrap: constant (0, ..., 0, k) plus
 * ca * c1 + cb * c2, all mod q, with q/8 = 2^29.  The sign of the resulting
 * phase (about +-q/8 or +-q/4 away from zero) is the gate's truth value. */
ORC_API int orc_gate_lincomb(int type, int n, const uint32_t *c1, const uint32_t *c2, uint32_t *out)
{
    const uint32_t E = 1u << 29; /* q/8 */
    uint32_t k;
    int32_t ca, cb;
    switch (type) {
    case G_NAND:  k = E;         ca = -1; cb = -1; break;
    case G_AND:   k = 0u - E;    ca = 1;  cb = 1;  break;
    case G_OR:    k = E;         ca = 1;  cb = 1;  break;
    case G_XOR:   k = 2 * E;     ca = 2;  cb = 2;  break;
    case G_XNOR:  k = 0u - 2 * E; ca = -2; cb = -2; break;
    case G_NOR:   k = 0u - E;    ca = -1; cb = -1; break;
    case G_ANDNY: k = 0u - E;    ca = -1; cb = 1;  break;
    case G_ANDYN: k = 0u - E;    ca = 1;  cb = -1; break;
    case G_ORNY:  k = E;         ca = -1; cb = 1;  break;
    case G_ORYN:  k = E;         ca = 1;  cb = -1; break;
    default: return -1;
    }
    for (int x = 0; x <= n; x++) out[x] = (uint32_t)ca * c1[x] + (uint32_t)cb * c2[x];
    out[n] += k;
    return 0;
}

/* Three-input gates (no constant term).  With t of the three inputs true,
 * c1 + c2 + c3 has phase (2t - 3) q/8:
 *   MAJ     c1 + c2 + c3: +-q/8 or +-3q/8, positive iff t >= 2;
 *   MAJNYY  -c1 + c2 + c3: the same vote with the first input negated;
 *   XOR3    -2 (c1 + c2 + c3) = -(2t - 3) q/4, which is +q/4 for t = 1 and
 *           (as -3q/4 mod q) for t = 3, -q/4 for t = 0 and t = 2: positive
 *           iff t is odd (the sum bit of a full adder).
 * Two-input types ignore c3. */
ORC_API int orc_gate_lincomb3(int type, int n, const uint32_t *c1, const uint32_t *c2, const uint32_t *c3,
                              uint32_t *out)
{
    if (type == G_MAJNYY) {
        for (int x = 0; x <= n; x++) out[x] = c2[x] + c3[x] - c1[x];
    } else if (type == G_MAJ) {
        for (int x = 0; x <= n; x++) out[x] = c1[x] + c2[x] + c3[x];
    } else if (type == G_XOR3) {
        for (int x = 0; x <= n; x++) out[x] = (uint32_t)0 - 2u * (c1[x] + c2[x] + c3[x]);
    } else {
        return orc_gate_lincomb(type, n, c1, c2, out);
    }
    return 0;
}

static int gate_has_three_inputs(int type) { return type == G_MAJNYY || type == G_MAJ || type == G_XOR3; }

/* One gate bootstrap: lincomb -> blind rotation -> extract -> keyswitch. */
ORC_API int orc_gate3(const orc_ctx *c, int type, const uint32_t *c1, const uint32_t *c2, const uint32_t *c3,
                      uint32_t *out)
{
    int n = c->p.n, N = c->p.N;
    uint32_t *lin = (uint32_t *)malloc(sizeof(uint32_t) * (n + 1));
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
    uint32_t *big = (uint32_t *)malloc(sizeof(uint32_t) * (N + 1));
    int rc = (gate_has_three_inputs(type) && !c3) ? -1 : orc_gate_lincomb3(type, n, c1, c2, c3, lin);
    if (rc == 0) {
        orc_blind_rotate(c, lin, acc);
        orc_sample_extract(N, acc, big);
        orc_keyswitch(c, big, out);
    }
    free(lin);
    free(acc);
    free(big);
    return rc;
}

ORC_API int orc_gate(const orc_ctx *c, int type, const uint32_t *c1, const uint32_t *c2, uint32_t *out)
{
    return orc_gate3(c, type, c1, c2, NULL, out);
}

/* Independent gates, one per thread. */
ORC_API int orc_gate_batch(const orc_ctx *c, const int32_t *types, const uint32_t *a, const uint32_t *b,
                           uint32_t *out, size_t count)
{
    size_t w = (size_t)c->p.n + 1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (long long k = 0; k < (long long)count; k++)
        bad |= orc_gate(c, types[k], a + k * w, b + k * w, out + k * w) != 0;
    return bad ? -1 : 0;
}

/* NOT needs no bootstrap: negate every word. */
ORC_API void orc_not(int n, const uint32_t *in, uint32_t *out)
{
    for (int x = 0; x <= n; x++) out[x] = (uint32_t)0 - in[x];
}

/* ------------------------------------------------------------------ */
/* Predicate netlists (per row).  Wires: column bits 0..w-1 (LSB first),   */
/* then constant bits (w for EQ/LT: k; 2w for RANGE: lo then hi), then     */
/* payload bits (column-major, LSB first), then gate outputs in order.     */
/* ------------------------------------------------------------------ */

enum { P_EQ = 0, P_LT = 1, P_RANGE = 2, P_LT_MAJ = 3, P_RANGE_MAJ = 4 };

typedef struct {
    int32_t *type, *a, *b, *c; /* one entry per gate (c = -1: two inputs); gate g writes wire first_gate_wire + g */
    int count, cap, next_wire;
} netlist;

static int nl_add3(netlist *nl, int type, int a, int b, int c)
{
    if (nl->type) {
        nl->type[nl->count] = type;
        nl->a[nl->count] = a;
        nl->b[nl->count] = b;
        if (nl->c) nl->c[nl->count] = c;
    }
    nl->count++;
    return nl->next_wire++;
}

static int nl_add(netlist *nl, int type, int a, int b) { return nl_add3(nl, type, a, b, -1); }

/* x_i = XNOR(c_i, k_i); then a pairwise AND tree: each round pairs (2j, 2j+1)
 * in order and moves a trailing odd element to the end of the next round. */
static int nl_eq(netlist *nl, int cbase, int kbase, int w)
{
    int list[64], m = w;
    for (int i = 0; i < w; i++) list[i] = nl_add(nl, G_XNOR, cbase + i, kbase + i);
    while (m > 1) {
        int nm = 0;
        for (int j = 0; j + 1 < m; j += 2) list[nm++] = nl_add(nl, G_AND, list[j], list[j + 1]);
        if (m & 1) list[nm++] = list[m - 1];
        m = nm;
    }
    return list[0];
}

/* Unsigned c < k, ripple from the LSB:
 * lt_0 = (not c_0) and k_0;  lt_i = ((not c_i) and k_i) or (XNOR(c_i, k_i) and lt_{i-1}). */
static int nl_lt(netlist *nl, int cbase, int kbase, int w)
{
    int lt = nl_add(nl, G_ANDNY, cbase, kbase);
    for (int i = 1; i < w; i++) {
        int g = nl_add(nl, G_ANDNY, cbase + i, kbase + i);
        int e = nl_add(nl, G_XNOR, cbase + i, kbase + i);
        int t = nl_add(nl, G_AND, e, lt);
        lt = nl_add(nl, G_OR, g, t);
    }
    return lt;
}

/* Unsigned c < k as a majority chain (c < k over bits 0..i is "not c_i and
 * k_i", or, when c_i = k_i, the result over bits 0..i-1; with bits this is
 * the majority of not c_i, k_i and that result):
 * lt_0 = (not c_0) and k_0;  lt_i = MAJ(not c_i, k_i, lt_{i-1}). */
static int nl_lt_maj(netlist *nl, int cbase, int kbase, int w)
{
    int lt = nl_add(nl, G_ANDNY, cbase, kbase);
    for (int i = 1; i < w; i++) lt = nl_add3(nl, G_MAJNYY, cbase + i, kbase + i, lt);
    return lt;
}

/* Build the per-row netlist.  Returns the number of gates; fills the arrays
 * when non-null (each of capacity >= the count; c may be NULL for the
 * two-input predicates).  *match_wire receives the wire of the match bit;
 * mask gate outputs are the last n_payload*pw wires. */
ORC_API int orc_netlist3(int pred, int w, int n_payload, int pw, int32_t *type, int32_t *a, int32_t *b,
                         int32_t *c, int32_t *match_wire, int32_t *n_inputs)
{
    if (w < 1 || w > 64 || pw < 0 || n_payload < 0) return -1;
    int range = pred == P_RANGE || pred == P_RANGE_MAJ;
    int nconst = range ? 2 * w : w;
    int ninp = w + nconst + n_payload * pw;
    netlist nl = {type, a, b, c, 0, 0, ninp};
    int m;
    if (pred == P_EQ) m = nl_eq(&nl, 0, w, w);
    else if (pred == P_LT) m = nl_lt(&nl, 0, w, w);
    else if (pred == P_LT_MAJ) m = nl_lt_maj(&nl, 0, w, w);
    else if (range) {
        int ge_lo = pred == P_RANGE ? nl_lt(&nl, 0, w, w) : nl_lt_maj(&nl, 0, w, w);
        int lt_hi = pred == P_RANGE ? nl_lt(&nl, 0, 2 * w, w) : nl_lt_maj(&nl, 0, 2 * w, w);
        m = nl_add(&nl, G_ANDNY, ge_lo, lt_hi); /* not(c < lo) and (c < hi) */
    } else return -1;
    for (int p = 0; p < n_payload; p++)
        for (int bit = 0; bit < pw; bit++) nl_add(&nl, G_AND, m, w + nconst + p * pw + bit);
    if (match_wire) *match_wire = m;
    if (n_inputs) *n_inputs = ninp;
    return nl.count;
}

ORC_API int orc_netlist(int pred, int w, int n_payload, int pw, int32_t *type, int32_t *a, int32_t *b,
                        int32_t *match_wire, int32_t *n_inputs)
{
    return orc_netlist3(pred, w, n_payload, pw, type, a, b, NULL, match_wire, n_inputs);
}

/* Plaintext evaluation of a gate type on bits (truth-table reference). */
ORC_API int orc_gate_plain(int type, int x, int y)
{
    switch (type) {
    case G_NAND: return !(x && y);
    case G_AND: return x && y;
    case G_OR: return x || y;
    case G_XOR: return x != y;
    case G_XNOR: return x == y;
    case G_NOR: return !(x || y);
    case G_ANDNY: return !x && y;
    case G_ANDYN: return x && !y;
    case G_ORNY: return !x || y;
    case G_ORYN: return x || !y;
    }
    return -1;
}

ORC_API int orc_gate_plain3(int type, int x, int y, int z)
{
    if (type == G_MAJNYY) return ((!x) + y + z) >= 2;
    if (type == G_MAJ) return (x + y + z) >= 2;
    if (type == G_XOR3) return (x + y + z) & 1;
    return orc_gate_plain(type, x, y);
}

/* Plaintext evaluation of the netlist on one row's input bits. */
ORC_API int orc_netlist_eval_plain(int pred, int w, int n_payload, int pw, const uint8_t *inputs, uint8_t *wires_out)
{
    int32_t m, ninp;
    int g = orc_netlist3(pred, w, n_payload, pw, NULL, NULL, NULL, NULL, &m, &ninp);
    if (g < 0) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * g), *a = (int32_t *)malloc(sizeof(int32_t) * g),
            *b = (int32_t *)malloc(sizeof(int32_t) * g), *c3 = (int32_t *)malloc(sizeof(int32_t) * g);
    orc_netlist3(pred, w, n_payload, pw, t, a, b, c3, &m, &ninp);
    for (int i = 0; i < ninp; i++) wires_out[i] = inputs[i];
    for (int k = 0; k < g; k++)
        wires_out[ninp + k] = (uint8_t)orc_gate_plain3(t[k], wires_out[a[k]], wires_out[b[k]],
                                                       c3[k] >= 0 ? wires_out[c3[k]] : 0);
    free(t);
    free(a);
    free(b);
    free(c3);
    return m;
}

/* ------------------------------------------------------------------ */
/* The scan (Alg. 2): every row of a table.                               */
/* column: [rows][w][n+1]; consts: [w or 2w][n+1]; payload p: [rows][pw][n+1]; */
/* match: [rows][n+1]; out p: [rows][pw][n+1].  Rows are independent; the  */
/* gates of a row run in netlist order, except that gates whose inputs are */
/* all ready (same depth) run side by side, over all rows at once.         */
/* ------------------------------------------------------------------ */
ORC_API int orc_scan(const orc_ctx *c, int pred, int w, const uint32_t *column, const uint32_t *consts,
                     int n_payload, int pw, const uint32_t *const *payloads, uint32_t *match,
                     uint32_t *const *out_payloads, long long rows)
{
    int32_t m, ninp;
    int g = orc_netlist3(pred, w, n_payload, pw, NULL, NULL, NULL, NULL, &m, &ninp);
    if (g < 0) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * g), *a = (int32_t *)malloc(sizeof(int32_t) * g),
            *b = (int32_t *)malloc(sizeof(int32_t) * g), *c3 = (int32_t *)malloc(sizeof(int32_t) * g),
            *depth = (int32_t *)malloc(sizeof(int32_t) * (ninp + g));
    orc_netlist3(pred, w, n_payload, pw, t, a, b, c3, &m, &ninp);
    int maxd = 0;
    for (int i = 0; i < ninp; i++) depth[i] = 0;
    for (int k = 0; k < g; k++) {
        int d = depth[a[k]] > depth[b[k]] ? depth[a[k]] : depth[b[k]];
        if (c3[k] >= 0 && depth[c3[k]] > d) d = depth[c3[k]];
        depth[ninp + k] = 1 + d;
        if (depth[ninp + k] > maxd) maxd = depth[ninp + k];
    }
    size_t W = (size_t)c->p.n + 1, per_row = (size_t)(ninp + g) * W;
    int nconst = (pred == P_RANGE || pred == P_RANGE_MAJ) ? 2 * w : w;
    uint32_t *wires = (uint32_t *)malloc(sizeof(uint32_t) * per_row * (size_t)(rows > 0 ? rows : 1));
    for (long long row = 0; row < rows; row++) {
        uint32_t *wr = wires + (size_t)row * per_row;
        for (int i = 0; i < w; i++) memcpy(wr + i * W, column + ((size_t)row * w + i) * W, W * 4);
        for (int i = 0; i < nconst; i++) memcpy(wr + (w + i) * W, consts + (size_t)i * W, W * 4);
        for (int p = 0; p < n_payload; p++)
            for (int bit = 0; bit < pw; bit++)
                memcpy(wr + (size_t)(w + nconst + p * pw + bit) * W, payloads[p] + ((size_t)row * pw + bit) * W, W * 4);
    }
    int bad = 0;
    for (int d = 1; d <= maxd; d++) {
#pragma omp parallel for schedule(dynamic, 1) collapse(2) reduction(| : bad)
        for (long long row = 0; row < rows; row++)
            for (int k = 0; k < g; k++) {
                if (depth[ninp + k] != d) continue;
                uint32_t *wr = wires + (size_t)row * per_row;
                bad |= orc_gate3(c, t[k], wr + (size_t)a[k] * W, wr + (size_t)b[k] * W,
                                 c3[k] >= 0 ? wr + (size_t)c3[k] * W : NULL, wr + (size_t)(ninp + k) * W) != 0;
            }
    }
    int first_mask = ninp + g - n_payload * pw;
    for (long long row = 0; row < rows; row++) {
        uint32_t *wr = wires + (size_t)row * per_row;
        memcpy(match + (size_t)row * W, wr + (size_t)m * W, W * 4);
        for (int p = 0; p < n_payload; p++)
            for (int bit = 0; bit < pw; bit++)
                memcpy(out_payloads[p] + ((size_t)row * pw + bit) * W, wr + (size_t)(first_mask + p * pw + bit) * W, W * 4);
    }
    free(wires);
    free(t);
    free(a);
    free(b);
    free(c3);
    free(depth);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Plaintext query constants (§4.2 lets an operand of a comparison be a    */
/* plaintext; §6.1 D times trivially encrypted operands).  The server then */
/* knows every constant bit, so a gate with a known input reduces: XNOR    */
/* with a known bit is the column bit or its negation (no bootstrap), and  */
/* a comparator step with known k_i is one AND (k_i = 0) or one OR         */
/* (k_i = 1) of (not c_i) with the running result, or nothing when that    */
/* result is already a known bit.  Values are literals: 2*wire + negated,  */
/* or LIT_FALSE / LIT_TRUE for a known bit.  Every gate still writes a     */
/* plain (non-negated) wire; negation is folded into the gate type.        */
/* Wires: column bits 0..w-1, then payload bits, then gate outputs.        */
/* Outputs that are not gate outputs are materialised without bootstrap:   */
/* a copy or negation (every word negated) of an input ciphertext, or the  */
/* trivial ciphertext (0, .., 0, +-q/8) of a known bit.                    */
/* ------------------------------------------------------------------ */

#define LIT_FALSE (-1)
#define LIT_TRUE (-2)

static int lit_not(int u)
{
    if (u == LIT_FALSE) return LIT_TRUE;
    if (u == LIT_TRUE) return LIT_FALSE;
    return u ^ 1;
}

/* u and v; with two wires the gate type absorbs the negations */
static int lit_and(netlist *nl, int u, int v)
{
    static const int type[4] = {G_AND, G_ANDNY, G_ANDYN, G_NOR}; /* [neg u + 2 neg v] */
    if (u == LIT_FALSE || v == LIT_FALSE) return LIT_FALSE;
    if (u == LIT_TRUE) return v;
    if (v == LIT_TRUE) return u;
    return 2 * nl_add(nl, type[(u & 1) + 2 * (v & 1)], u >> 1, v >> 1);
}

/* u or v */
static int lit_or(netlist *nl, int u, int v)
{
    static const int type[4] = {G_OR, G_ORNY, G_ORYN, G_NAND}; /* [neg u + 2 neg v] */
    if (u == LIT_TRUE || v == LIT_TRUE) return LIT_TRUE;
    if (u == LIT_FALSE) return v;
    if (v == LIT_FALSE) return u;
    return 2 * nl_add(nl, type[(u & 1) + 2 * (v & 1)], u >> 1, v >> 1);
}

/* c == k: the literal c_i (k_i = 1) or not c_i (k_i = 0) per bit, then the
 * same pairwise AND tree as the encrypted-constant netlist. */
static int nlp_eq(netlist *nl, int cbase, int w, uint64_t k)
{
    int list[64], m = w;
    for (int i = 0; i < w; i++) list[i] = 2 * (cbase + i) + (int)(((k >> i) & 1) ^ 1);
    while (m > 1) {
        int nm = 0;
        for (int j = 0; j + 1 < m; j += 2) list[nm++] = lit_and(nl, list[j], list[j + 1]);
        if (m & 1) list[nm++] = list[m - 1];
        m = nm;
    }
    return list[0];
}

/* c < k: lt_0 = (not c_0) and k_0; lt_i = MAJ(not c_i, k_i, lt_{i-1}), which
 * is (not c_i) or lt_{i-1} for k_i = 1 and (not c_i) and lt_{i-1} for k_i = 0
 * (the ripple form reduces to the same two cases). */
static int nlp_lt(netlist *nl, int cbase, int w, uint64_t k)
{
    int lt = (k & 1) ? 2 * cbase + 1 : LIT_FALSE;
    for (int i = 1; i < w; i++) {
        int nc = 2 * (cbase + i) + 1;
        lt = ((k >> i) & 1) ? lit_or(nl, nc, lt) : lit_and(nl, nc, lt);
    }
    return lt;
}

/* Netlist for plaintext constants k0 (EQ, LT) or lo = k0, hi = k1 (RANGE).
 * pred: P_EQ, P_LT or P_RANGE (the majority forms are the same here).
 * Returns the gate count; *match_lit gets the match literal and out_lits
 * (capacity n_payload*pw, may be NULL) the literal of every masked payload
 * bit; when the match is a wire, the mask gates are the last n_payload*pw
 * gates. */
ORC_API int orc_netlist_plain(int pred, int w, int n_payload, int pw, uint64_t k0, uint64_t k1, int32_t *type,
                              int32_t *a, int32_t *b, int32_t *match_lit, int32_t *out_lits, int32_t *n_inputs)
{
    if (w < 1 || w > 64 || pw < 0 || n_payload < 0) return -1;
    int ninp = w + n_payload * pw;
    netlist nl = {type, a, b, NULL, 0, 0, ninp};
    int m;
    if (pred == P_EQ) m = nlp_eq(&nl, 0, w, k0);
    else if (pred == P_LT || pred == P_LT_MAJ) m = nlp_lt(&nl, 0, w, k0);
    else if (pred == P_RANGE || pred == P_RANGE_MAJ) {
        int below_lo = nlp_lt(&nl, 0, w, k0);
        int below_hi = nlp_lt(&nl, 0, w, k1);
        m = lit_and(&nl, lit_not(below_lo), below_hi);
    } else return -1;
    for (int p = 0; p < n_payload; p++)
        for (int bit = 0; bit < pw; bit++) {
            int o = lit_and(&nl, m, 2 * (w + p * pw + bit));
            if (out_lits) out_lits[p * pw + bit] = o;
        }
    if (match_lit) *match_lit = m;
    if (n_inputs) *n_inputs = ninp;
    return nl.count;
}

static int lit_value(const uint8_t *wires, int lit)
{
    if (lit == LIT_FALSE) return 0;
    if (lit == LIT_TRUE) return 1;
    return wires[lit >> 1] ^ (lit & 1);
}

/* Plaintext evaluation: inputs = column bits then payload bits of one row;
 * outputs = match bit then the masked payload bits. */
ORC_API int orc_netlist_plain_eval(int pred, int w, int n_payload, int pw, uint64_t k0, uint64_t k1,
                                   const uint8_t *inputs, uint8_t *outputs)
{
    int32_t m, ninp;
    int g = orc_netlist_plain(pred, w, n_payload, pw, k0, k1, NULL, NULL, NULL, &m, NULL, &ninp);
    if (g < 0) return -1;
    int np = n_payload * pw;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *a = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *b = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *ol = (int32_t *)malloc(sizeof(int32_t) * (np + 1));
    uint8_t *wires = (uint8_t *)malloc((size_t)(ninp + g + 1));
    orc_netlist_plain(pred, w, n_payload, pw, k0, k1, t, a, b, &m, ol, &ninp);
    for (int i = 0; i < ninp; i++) wires[i] = inputs[i];
    for (int k = 0; k < g; k++) wires[ninp + k] = (uint8_t)orc_gate_plain(t[k], wires[a[k]], wires[b[k]]);
    outputs[0] = (uint8_t)lit_value(wires, m);
    for (int i = 0; i < np; i++) outputs[1 + i] = (uint8_t)lit_value(wires, ol[i]);
    free(t);
    free(a);
    free(b);
    free(ol);
    free(wires);
    return g;
}

/* ciphertext of a literal: copy, negation, or trivial encryption */
static void lit_materialise(int n, const uint32_t *wr, size_t W, int lit, uint32_t *out)
{
    if (lit == LIT_FALSE || lit == LIT_TRUE) {
        memset(out, 0, (size_t)n * 4);
        out[n] = lit == LIT_TRUE ? (uint32_t)1 << 29 : (uint32_t)0 - ((uint32_t)1 << 29);
    } else if (lit & 1) {
        orc_not(n, wr + (size_t)(lit >> 1) * W, out);
    } else {
        memcpy(out, wr + (size_t)(lit >> 1) * W, W * 4);
    }
}

/* The scan with plaintext constants: layouts as orc_scan, without consts. */
ORC_API int orc_scan_plain(const orc_ctx *c, int pred, int w, const uint32_t *column, uint64_t k0, uint64_t k1,
                           int n_payload, int pw, const uint32_t *const *payloads, uint32_t *match,
                           uint32_t *const *out_payloads, long long rows)
{
    int32_t m, ninp;
    int g = orc_netlist_plain(pred, w, n_payload, pw, k0, k1, NULL, NULL, NULL, &m, NULL, &ninp);
    if (g < 0) return -1;
    int np = n_payload * pw;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *a = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *b = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *ol = (int32_t *)malloc(sizeof(int32_t) * (np + 1)),
            *depth = (int32_t *)malloc(sizeof(int32_t) * (ninp + g + 1));
    orc_netlist_plain(pred, w, n_payload, pw, k0, k1, t, a, b, &m, ol, &ninp);
    int maxd = 0;
    for (int i = 0; i < ninp; i++) depth[i] = 0;
    for (int k = 0; k < g; k++) {
        depth[ninp + k] = 1 + (depth[a[k]] > depth[b[k]] ? depth[a[k]] : depth[b[k]]);
        if (depth[ninp + k] > maxd) maxd = depth[ninp + k];
    }
    size_t W = (size_t)c->p.n + 1, per_row = (size_t)(ninp + g) * W;
    uint32_t *wires = (uint32_t *)malloc(sizeof(uint32_t) * per_row * (size_t)(rows > 0 ? rows : 1));
    for (long long row = 0; row < rows; row++) {
        uint32_t *wr = wires + (size_t)row * per_row;
        for (int i = 0; i < w; i++) memcpy(wr + i * W, column + ((size_t)row * w + i) * W, W * 4);
        for (int p = 0; p < n_payload; p++)
            for (int bit = 0; bit < pw; bit++)
                memcpy(wr + (size_t)(w + p * pw + bit) * W, payloads[p] + ((size_t)row * pw + bit) * W, W * 4);
    }
    int bad = 0;
    for (int d = 1; d <= maxd; d++) {
#pragma omp parallel for schedule(dynamic, 1) collapse(2) reduction(| : bad)
        for (long long row = 0; row < rows; row++)
            for (int k = 0; k < g; k++) {
                if (depth[ninp + k] != d) continue;
                uint32_t *wr = wires + (size_t)row * per_row;
                bad |= orc_gate(c, t[k], wr + (size_t)a[k] * W, wr + (size_t)b[k] * W,
                                wr + (size_t)(ninp + k) * W) != 0;
            }
    }
    for (long long row = 0; row < rows; row++) {
        const uint32_t *wr = wires + (size_t)row * per_row;
        lit_materialise(c->p.n, wr, W, m, match + (size_t)row * W);
        for (int p = 0; p < n_payload; p++)
            for (int bit = 0; bit < pw; bit++)
                lit_materialise(c->p.n, wr, W, ol[p * pw + bit], out_payloads[p] + ((size_t)row * pw + bit) * W);
    }
    free(wires);
    free(t);
    free(a);
    free(b);
    free(ol);
    free(depth);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* SUM aggregation of the selected rows (§6.1 D, the result_k / result_v  */
/* sums: the masked values of all rows added homomorphically; rows that  */
/* do not match contribute zero).                                         */
/* Each value is rows x pw encrypted bits, LSB first; the sum is taken     */
/* mod 2^ow.  The circuit is a carry-save (Wallace) tree of full adders:   */
/* sum bit XOR3(x, y, z) and carry MAJ(x, y, z), one bootstrap each, then  */
/* one ripple-carry adder.  Canonical form (every choice fixes the words):  */
/*  - column j (weight 2^j, j < ow) starts as the bits j of rows 0..R-1;  */
/*  - while some column holds more than 2 wires, one layer: for j = 0..ow-1 */
/*    take its wires in order in groups of three; each group appends its    */
/*    XOR3 to the next layer's column j and (if j + 1 < ow) its MAJ to the   */
/*    next layer's column j + 1; the 0-2 wires left over follow;            */
/*  - ripple: carry = none; for j = 0..ow-1 the operands are column j's      */
/*    wires then the carry: none -> output 0; one -> that wire; two ->      */
/*    XOR and carry AND; three -> XOR3 and carry MAJ (no carry out of the   */
/*    top column).                                                          */
/* Wires: input bit (r, j) is r*pw + j; gate outputs follow.  Output j is a */
/* literal (2*wire, or LIT_FALSE).                                          */
/* ------------------------------------------------------------------ */

ORC_API int orc_sum_netlist(int rows, int pw, int ow, int32_t *type, int32_t *a, int32_t *b, int32_t *c,
                            int32_t *out_lits, int32_t *n_inputs)
{
    if (rows < 1 || pw < 1 || pw > 64 || ow < 1 || ow > 64) return -1;
    int ninp = rows * pw, cap = rows + 4;
    netlist nl = {type, a, b, c, 0, 0, ninp};
    int *cur = (int *)malloc(sizeof(int) * (size_t)ow * cap), *nxt = (int *)malloc(sizeof(int) * (size_t)ow * cap);
    int *cn = (int *)calloc((size_t)ow, sizeof(int)), *nn = (int *)calloc((size_t)ow, sizeof(int));
    for (int j = 0; j < ow && j < pw; j++) {
        for (int r = 0; r < rows; r++) cur[(size_t)j * cap + r] = r * pw + j;
        cn[j] = rows;
    }
    for (;;) {
        int widest = 0;
        for (int j = 0; j < ow; j++)
            if (cn[j] > widest) widest = cn[j];
        if (widest <= 2) break;
        for (int j = 0; j < ow; j++) nn[j] = 0;
        for (int j = 0; j < ow; j++) {
            const int *L = cur + (size_t)j * cap;
            int i = 0;
            for (; cn[j] - i >= 3; i += 3) {
                nxt[(size_t)j * cap + nn[j]++] = nl_add3(&nl, G_XOR3, L[i], L[i + 1], L[i + 2]);
                if (j + 1 < ow) nxt[(size_t)(j + 1) * cap + nn[j + 1]++] = nl_add3(&nl, G_MAJ, L[i], L[i + 1], L[i + 2]);
            }
            for (; i < cn[j]; i++) nxt[(size_t)j * cap + nn[j]++] = L[i];
        }
        int *t = cur; cur = nxt; nxt = t;
        int *tn = cn; cn = nn; nn = tn;
    }
    int carry = -1;
    for (int j = 0; j < ow; j++) {
        int ops[3], k = 0;
        for (int i = 0; i < cn[j]; i++) ops[k++] = cur[(size_t)j * cap + i];
        if (carry >= 0) ops[k++] = carry;
        int lit, top = j + 1 == ow;
        if (k == 0) {
            lit = LIT_FALSE;
            carry = -1;
        } else if (k == 1) {
            lit = 2 * ops[0];
            carry = -1;
        } else if (k == 2) {
            lit = 2 * nl_add(&nl, G_XOR, ops[0], ops[1]);
            carry = top ? -1 : nl_add(&nl, G_AND, ops[0], ops[1]);
        } else {
            lit = 2 * nl_add3(&nl, G_XOR3, ops[0], ops[1], ops[2]);
            carry = top ? -1 : nl_add3(&nl, G_MAJ, ops[0], ops[1], ops[2]);
        }
        if (out_lits) out_lits[j] = lit;
    }
    free(cur);
    free(nxt);
    free(cn);
    free(nn);
    if (n_inputs) *n_inputs = ninp;
    return nl.count;
}

/* Plaintext evaluation of the SUM circuit: in_bits [rows][pw] -> out_bits [ow]. */
ORC_API int orc_sum_eval_plain(int rows, int pw, int ow, const uint8_t *in_bits, uint8_t *out_bits)
{
    int32_t ninp;
    int g = orc_sum_netlist(rows, pw, ow, NULL, NULL, NULL, NULL, NULL, &ninp);
    if (g < 0) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *a = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *b = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *c3 = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *ol = (int32_t *)malloc(sizeof(int32_t) * ow);
    uint8_t *wires = (uint8_t *)malloc((size_t)(ninp + g + 1));
    orc_sum_netlist(rows, pw, ow, t, a, b, c3, ol, &ninp);
    for (int i = 0; i < ninp; i++) wires[i] = in_bits[i];
    for (int k = 0; k < g; k++)
        wires[ninp + k] = (uint8_t)orc_gate_plain3(t[k], wires[a[k]], wires[b[k]], c3[k] >= 0 ? wires[c3[k]] : 0);
    for (int j = 0; j < ow; j++) out_bits[j] = (uint8_t)lit_value(wires, ol[j]);
    free(t);
    free(a);
    free(b);
    free(c3);
    free(ol);
    free(wires);
    return g;
}

/* Encrypted SUM: in [rows][pw][n+1] -> out [ow][n+1]; gates run level by
 * level (a gate's level is one more than its deepest input), side by side. */
ORC_API int orc_aggregate_sum(const orc_ctx *c, const uint32_t *in, int rows, int pw, int ow, uint32_t *out)
{
    int32_t ninp;
    int g = orc_sum_netlist(rows, pw, ow, NULL, NULL, NULL, NULL, NULL, &ninp);
    if (g < 0) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *a = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *b = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *c3 = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *ol = (int32_t *)malloc(sizeof(int32_t) * ow), *depth = (int32_t *)malloc(sizeof(int32_t) * (ninp + g + 1));
    orc_sum_netlist(rows, pw, ow, t, a, b, c3, ol, &ninp);
    int maxd = 0;
    for (int i = 0; i < ninp; i++) depth[i] = 0;
    for (int k = 0; k < g; k++) {
        int d = depth[a[k]] > depth[b[k]] ? depth[a[k]] : depth[b[k]];
        if (c3[k] >= 0 && depth[c3[k]] > d) d = depth[c3[k]];
        depth[ninp + k] = 1 + d;
        if (depth[ninp + k] > maxd) maxd = depth[ninp + k];
    }
    size_t W = (size_t)c->p.n + 1;
    uint32_t *wires = (uint32_t *)malloc(sizeof(uint32_t) * W * (size_t)(ninp + g + 1));
    memcpy(wires, in, sizeof(uint32_t) * W * (size_t)ninp);
    int bad = 0;
    for (int d = 1; d <= maxd; d++) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
        for (int k = 0; k < g; k++) {
            if (depth[ninp + k] != d) continue;
            bad |= orc_gate3(c, t[k], wires + (size_t)a[k] * W, wires + (size_t)b[k] * W,
                             c3[k] >= 0 ? wires + (size_t)c3[k] * W : NULL, wires + (size_t)(ninp + k) * W) != 0;
        }
    }
    for (int j = 0; j < ow; j++) lit_materialise(c->p.n, wires, W, ol[j], out + (size_t)j * W);
    free(wires);
    free(t);
    free(a);
    free(b);
    free(c3);
    free(ol);
    free(depth);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* MAX and MIN of the selected rows (§4.2 B lists max(a, b) and min(a, b) */
/* among the operators of the homomorphic expression tree).  Unsigned      */
/* values of w bits, LSB first.  Pairwise: s = [a < b] by the majority     */
/* comparator (s_0 = ANDNY(a_0, b_0), s_i = MAJNYY(a_i, b_i, s_{i-1})), then */
/* per bit a multiplexer OR(AND(s, x), ANDNY(s, y)) = s ? x : y, with      */
/* (x, y) = (b, a) for max and (a, b) for min.  Rows reduce as a tournament */
/* in the order of the equality AND tree: each round pairs (2i, 2i+1) and   */
/* moves an unpaired last value to the end of the next round.  MAX takes    */
/* the masked values as they are (a row that does not match is 0, the      */
/* identity of max over unsigned values); MIN first replaces every bit of  */
/* a row that does not match by 1, u_j = ORYN(v_j, m) = v_j or not m, so   */
/* such rows become 2^w - 1, the identity of min.  No rows: MAX is 0, MIN  */
/* is 2^w - 1 (known bits).  Wires: value bit (r, j) is r*w + j; for MIN    */
/* the match bit of row r is rows*w + r; gate outputs follow.              */
/* ------------------------------------------------------------------ */

static void nl_extreme_pair(netlist *nl, int is_min, const int *a, const int *b, int w, int *out)
{
    int s = nl_add(nl, G_ANDNY, a[0], b[0]); /* s = [a < b] */
    for (int i = 1; i < w; i++) s = nl_add3(nl, G_MAJNYY, a[i], b[i], s);
    for (int j = 0; j < w; j++) {
        int x = is_min ? a[j] : b[j], y = is_min ? b[j] : a[j];
        int tx = nl_add(nl, G_AND, s, x);
        int ty = nl_add(nl, G_ANDNY, s, y);
        out[j] = nl_add(nl, G_OR, tx, ty);
    }
}

ORC_API int orc_extreme_netlist(int is_min, int rows, int w, int32_t *type, int32_t *a, int32_t *b, int32_t *c,
                                int32_t *out_lits, int32_t *n_inputs)
{
    if (rows < 0 || w < 1 || w > 64) return -1;
    int ninp = rows * w + (is_min ? rows : 0);
    netlist nl = {type, a, b, c, 0, 0, ninp};
    int *cur = (int *)malloc(sizeof(int) * (size_t)(rows > 0 ? rows : 1) * w);
    int *nxt = (int *)malloc(sizeof(int) * (size_t)(rows > 0 ? rows : 1) * w);
    for (int r = 0; r < rows; r++)
        for (int j = 0; j < w; j++)
            cur[(size_t)r * w + j] = is_min ? nl_add(&nl, G_ORYN, r * w + j, rows * w + r) : r * w + j;
    int m = rows;
    while (m > 1) {
        int nm = 0;
        for (int i = 0; i + 1 < m; i += 2, nm++)
            nl_extreme_pair(&nl, is_min, cur + (size_t)i * w, cur + (size_t)(i + 1) * w, w, nxt + (size_t)nm * w);
        if (m & 1) {
            memcpy(nxt + (size_t)nm * w, cur + (size_t)(m - 1) * w, sizeof(int) * w);
            nm++;
        }
        int *t = cur; cur = nxt; nxt = t;
        m = nm;
    }
    if (out_lits)
        for (int j = 0; j < w; j++) out_lits[j] = rows > 0 ? 2 * cur[j] : (is_min ? LIT_TRUE : LIT_FALSE);
    free(cur);
    free(nxt);
    if (n_inputs) *n_inputs = ninp;
    return nl.count;
}

/* Plaintext evaluation: values [rows] (w bits each), match bits [rows] (MIN only). */
ORC_API int orc_extreme_eval_plain(int is_min, int rows, int w, const uint8_t *in_bits, uint8_t *out_bits)
{
    int32_t ninp;
    int g = orc_extreme_netlist(is_min, rows, w, NULL, NULL, NULL, NULL, NULL, &ninp);
    if (g < 0) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *a = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *b = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *c3 = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *ol = (int32_t *)malloc(sizeof(int32_t) * w);
    uint8_t *wires = (uint8_t *)malloc((size_t)(ninp + g + 1));
    orc_extreme_netlist(is_min, rows, w, t, a, b, c3, ol, &ninp);
    for (int i = 0; i < ninp; i++) wires[i] = in_bits[i];
    for (int k = 0; k < g; k++)
        wires[ninp + k] = (uint8_t)orc_gate_plain3(t[k], wires[a[k]], wires[b[k]], c3[k] >= 0 ? wires[c3[k]] : 0);
    for (int j = 0; j < w; j++) out_bits[j] = (uint8_t)lit_value(wires, ol[j]);
    free(t);
    free(a);
    free(b);
    free(c3);
    free(ol);
    free(wires);
    return g;
}

/* Encrypted MAX / MIN: values [rows][w][n+1], match [rows][n+1] (MIN only,
 * else NULL) -> out [w][n+1]; gates level by level as orc_aggregate_sum. */
ORC_API int orc_aggregate_extreme(const orc_ctx *c, int is_min, const uint32_t *values, const uint32_t *match,
                                  int rows, int w, uint32_t *out)
{
    int32_t ninp;
    int g = orc_extreme_netlist(is_min, rows, w, NULL, NULL, NULL, NULL, NULL, &ninp);
    if (g < 0 || (is_min && rows > 0 && !match)) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *a = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *b = (int32_t *)malloc(sizeof(int32_t) * (g + 1)), *c3 = (int32_t *)malloc(sizeof(int32_t) * (g + 1)),
            *ol = (int32_t *)malloc(sizeof(int32_t) * w), *depth = (int32_t *)malloc(sizeof(int32_t) * (ninp + g + 1));
    orc_extreme_netlist(is_min, rows, w, t, a, b, c3, ol, &ninp);
    int maxd = 0;
    for (int i = 0; i < ninp; i++) depth[i] = 0;
    for (int k = 0; k < g; k++) {
        int d = depth[a[k]] > depth[b[k]] ? depth[a[k]] : depth[b[k]];
        if (c3[k] >= 0 && depth[c3[k]] > d) d = depth[c3[k]];
        depth[ninp + k] = 1 + d;
        if (depth[ninp + k] > maxd) maxd = depth[ninp + k];
    }
    size_t W = (size_t)c->p.n + 1;
    uint32_t *wires = (uint32_t *)malloc(sizeof(uint32_t) * W * (size_t)(ninp + g + 1));
    memcpy(wires, values, sizeof(uint32_t) * W * (size_t)rows * w);
    if (is_min && rows > 0) memcpy(wires + W * (size_t)rows * w, match, sizeof(uint32_t) * W * (size_t)rows);
    int bad = 0;
    for (int d = 1; d <= maxd; d++) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
        for (int k = 0; k < g; k++) {
            if (depth[ninp + k] != d) continue;
            bad |= orc_gate3(c, t[k], wires + (size_t)a[k] * W, wires + (size_t)b[k] * W,
                             c3[k] >= 0 ? wires + (size_t)c3[k] * W : NULL, wires + (size_t)(ninp + k) * W) != 0;
        }
    }
    for (int j = 0; j < w; j++) lit_materialise(c->p.n, wires, W, ol[j], out + (size_t)j * W);
    free(wires);
    free(t);
    free(a);
    free(b);
    free(c3);
    free(ol);
    free(depth);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Keyswitch-first order (the order of TFHE-rs, which the paper uses,     */
/* §2.2): ciphertexts live under the N-bit key (the GLWE key read as an   */
/* LWE key), each gate forms its linear combination on N + 1 words,       */
/* keyswitches that single result to the n-bit key, and bootstraps it; the */
/* extracted sample is the gate's output, under the N-bit key again.      */
/* Fresh ciphertexts under the N-bit key use the GLWE noise; ciphertext c */
/* of a stream draws words c (N + 2) .. c (N + 2) + N + 1.                */
/* ------------------------------------------------------------------ */

ORC_API void orc_encrypt_big_bits(const orc_ctx *c, const uint8_t *bits, size_t count, uint64_t stream,
                                  uint64_t first_index, uint32_t *out)
{
    int N = c->p.N;
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)count; k++)
        lwe_encrypt(c->S, N, bits[k] ? (1u << 29) : (uint32_t)(0u - (1u << 29)), c->p.glwe_sigma, c->seed, stream,
                    (first_index + (uint64_t)k) * (N + 2), out + (size_t)k * (N + 1));
}

ORC_API void orc_decrypt_big_bits(const orc_ctx *c, const uint32_t *ct, size_t count, uint8_t *out)
{
    for (size_t k = 0; k < count; k++)
        out[k] = (int32_t)lwe_phase(ct + k * (c->p.N + 1), c->S, c->p.N) > 0;
}

/* One keyswitch-first gate: lincomb on N + 1 words -> keyswitch -> blind
 * rotation (which modulus-switches its input) -> sample extraction. */
ORC_API int orc_gate3_ks_first(const orc_ctx *c, int type, const uint32_t *c1, const uint32_t *c2,
                               const uint32_t *c3, uint32_t *out)
{
    int n = c->p.n, N = c->p.N;
    uint32_t *lin = (uint32_t *)malloc(sizeof(uint32_t) * (N + 1));
    uint32_t *small = (uint32_t *)malloc(sizeof(uint32_t) * (n + 1));
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
    int rc = (gate_has_three_inputs(type) && !c3) ? -1 : orc_gate_lincomb3(type, N, c1, c2, c3, lin);
    if (rc == 0) {
        orc_keyswitch(c, lin, small);
        orc_blind_rotate(c, small, acc);
        orc_sample_extract(N, acc, out);
    }
    free(lin);
    free(small);
    free(acc);
    return rc;
}

/* The scan in keyswitch-first order: orc_scan's netlists and layouts with
 * every ciphertext N + 1 words (column, constants, payloads, outputs). */
ORC_API int orc_scan_ks_first(const orc_ctx *c, int pred, int w, const uint32_t *column, const uint32_t *consts,
                              int n_payload, int pw, const uint32_t *const *payloads, uint32_t *match,
                              uint32_t *const *out_payloads, long long rows)
{
    int32_t m, ninp;
    int g = orc_netlist3(pred, w, n_payload, pw, NULL, NULL, NULL, NULL, &m, &ninp);
    if (g < 0) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * g), *a = (int32_t *)malloc(sizeof(int32_t) * g),
            *b = (int32_t *)malloc(sizeof(int32_t) * g), *c3 = (int32_t *)malloc(sizeof(int32_t) * g),
            *depth = (int32_t *)malloc(sizeof(int32_t) * (ninp + g));
    orc_netlist3(pred, w, n_payload, pw, t, a, b, c3, &m, &ninp);
    int maxd = 0;
    for (int i = 0; i < ninp; i++) depth[i] = 0;
    for (int k = 0; k < g; k++) {
        int d = depth[a[k]] > depth[b[k]] ? depth[a[k]] : depth[b[k]];
        if (c3[k] >= 0 && depth[c3[k]] > d) d = depth[c3[k]];
        depth[ninp + k] = 1 + d;
        if (depth[ninp + k] > maxd) maxd = depth[ninp + k];
    }
    size_t W = (size_t)c->p.N + 1, per_row = (size_t)(ninp + g) * W;
    int nconst = (pred == P_RANGE || pred == P_RANGE_MAJ) ? 2 * w : w;
    uint32_t *wires = (uint32_t *)malloc(sizeof(uint32_t) * per_row * (size_t)(rows > 0 ? rows : 1));
    for (long long row = 0; row < rows; row++) {
        uint32_t *wr = wires + (size_t)row * per_row;
        for (int i = 0; i < w; i++) memcpy(wr + i * W, column + ((size_t)row * w + i) * W, W * 4);
        for (int i = 0; i < nconst; i++) memcpy(wr + (w + i) * W, consts + (size_t)i * W, W * 4);
        for (int p = 0; p < n_payload; p++)
            for (int bit = 0; bit < pw; bit++)
                memcpy(wr + (size_t)(w + nconst + p * pw + bit) * W, payloads[p] + ((size_t)row * pw + bit) * W, W * 4);
    }
    int bad = 0;
    for (int d = 1; d <= maxd; d++) {
#pragma omp parallel for schedule(dynamic, 1) collapse(2) reduction(| : bad)
        for (long long row = 0; row < rows; row++)
            for (int k = 0; k < g; k++) {
                if (depth[ninp + k] != d) continue;
                uint32_t *wr = wires + (size_t)row * per_row;
                bad |= orc_gate3_ks_first(c, t[k], wr + (size_t)a[k] * W, wr + (size_t)b[k] * W,
                                          c3[k] >= 0 ? wr + (size_t)c3[k] * W : NULL,
                                          wr + (size_t)(ninp + k) * W) != 0;
            }
    }
    int first_mask = ninp + g - n_payload * pw;
    for (long long row = 0; row < rows; row++) {
        uint32_t *wr = wires + (size_t)row * per_row;
        memcpy(match + (size_t)row * W, wr + (size_t)m * W, W * 4);
        for (int p = 0; p < n_payload; p++)
            for (int bit = 0; bit < pw; bit++)
                memcpy(out_payloads[p] + ((size_t)row * pw + bit) * W, wr + (size_t)(first_mask + p * pw + bit) * W,
                       W * 4);
    }
    free(wires);
    free(t);
    free(a);
    free(b);
    free(c3);
    free(depth);
    return bad ? -1 : 0;
}

ORC_API void orc_set_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

ORC_API int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
