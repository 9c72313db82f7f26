"""Pins for the CPU oracle: each check ties it to something other than itself
(a published test vector, a closed form, an invariant of the TFHE
construction the paper cites, brute force on tiny inputs), so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
Q = 1 << 32
E8 = 1 << 29


def centered(x):
    x = np.asarray(x, dtype=np.int64) & 0xFFFFFFFF
    return np.where(x >= (1 << 31), x - Q, x)


def read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# randomness
# --------------------------------------------------------------------------
def test_splitmix64_published_vector():
    for idx, hexval in read_golden("splitmix64_seed0.txt"):
        assert O.splitmix64(0, int(idx)) == int(hexval, 16)


def test_key_bits_balanced_and_seeded(real_oracle):
    s, S = real_oracle.lwe_key(), real_oracle.glwe_key()
    assert set(np.unique(s)) <= {0, 1} and set(np.unique(S)) <= {0, 1}
    assert 250 < s.sum() < 380 and 430 < S.sum() < 600
    other = O.Oracle(12)
    assert not np.array_equal(other.lwe_key(), s)
    again = O.Oracle(11)
    assert np.array_equal(again.lwe_key(), s) and np.array_equal(again.bk(), real_oracle.bk())


# --------------------------------------------------------------------------
# negacyclic products
# --------------------------------------------------------------------------
def test_negacyclic_hand_example():
    # (1 + X)(1 + X^3) = 1 + X + X^3 + X^4 = X + X^3 in Z[X]/(X^4 + 1)
    a = np.array([1, 1, 0, 0], np.uint32)
    b = np.array([1, 0, 0, 1], np.uint32)
    for f in (O.negacyclic_schoolbook, O.negacyclic_karatsuba):
        assert list(f(a, b)) == [0, 1, 0, 1]


def test_negacyclic_x_to_the_n_is_minus_one():
    for N in (8, 64, 1024):
        xn1 = np.zeros(N, np.uint32)
        xn1[N - 1] = 1
        x = np.zeros(N, np.uint32)
        x[1] = 1
        want = np.zeros(N, np.uint32)
        want[0] = 0xFFFFFFFF
        assert np.array_equal(O.negacyclic_karatsuba(xn1, x), want)
        assert np.array_equal(O.negacyclic_schoolbook(xn1, x), want)


@pytest.mark.parametrize("N", [4, 8, 64, 256, 1024])
def test_schoolbook_equals_karatsuba(N):
    rng = np.random.default_rng(N)
    a = rng.integers(0, Q, N, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, Q, N, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(O.negacyclic_schoolbook(a, b), O.negacyclic_karatsuba(a, b))


def test_negacyclic_against_numpy_convolution():
    # small coefficients: the integer convolution (a library routine) is exact in int64
    rng = np.random.default_rng(5)
    N = 64
    a = rng.integers(-64, 64, N)
    b = rng.integers(0, 1 << 20, N)
    full = np.convolve(a, b)  # length 2N-1
    full = np.concatenate([full, [0]])
    want = (full[:N] - full[N:]) % Q
    got = O.negacyclic_karatsuba((a % Q).astype(np.uint32), b.astype(np.uint32))
    assert np.array_equal(got.astype(np.int64), want)


def test_monomial_mul_is_product_with_monomial():
    rng = np.random.default_rng(9)
    N = 16
    a = rng.integers(0, Q, N, dtype=np.uint64).astype(np.uint32)
    for e in range(2 * N):
        mono = np.zeros(N, np.uint32)
        if e < N:
            mono[e] = 1
        else:
            mono[e - N] = 0xFFFFFFFF
        assert np.array_equal(O.monomial_mul(a, e), O.negacyclic_schoolbook(mono, a)), e


# --------------------------------------------------------------------------
# modulus switch and decompositions
# --------------------------------------------------------------------------
def test_modswitch_closed_form():
    rng = np.random.default_rng(1)
    xs = list(rng.integers(0, Q, 2000)) + [0, 1, Q - 1, 1 << 20, (1 << 20) - 1, (1 << 21) + (1 << 20), Q - (1 << 20)]
    for N in (64, 1024):
        twoN = 2 * N
        for x in xs:
            x = int(x)
            # nearest integer to x*2N/q, ties up, computed with exact rationals
            num = x * twoN
            want = ((2 * num + Q) // (2 * Q)) % twoN
            assert O.modswitch(x, N) == want


def test_gadget_decomposition_reconstructs_and_matches_offset_form():
    rng = np.random.default_rng(2)
    xs = np.concatenate([np.arange(1 << 12, dtype=np.uint64),
                         rng.integers(0, Q, 20000, dtype=np.uint64),
                         Q - 1 - np.arange(1 << 12, dtype=np.uint64)]).astype(np.uint64)
    bg, l = 7, 3
    off = sum(64 << (32 - bg * j) for j in range(1, l + 1)) + (1 << (32 - bg * l - 1))
    for x in xs[::7]:
        x = int(x)
        d = O.decompose(x, bg, l)
        assert all(-64 <= v < 64 for v in d)
        recon = sum(int(d[j - 1]) << (32 - bg * j) for j in range(1, l + 1))
        err = (x - recon) % Q
        err = err - Q if err >= Q // 2 else err
        assert -(1 << 10) <= err < (1 << 10)  # ties round up
        # the offset form of the same balanced decomposition
        y = (x + off) % Q
        alt = [((y >> (32 - bg * j)) & 127) - 64 for j in range(1, l + 1)]
        assert list(d) == alt


# --------------------------------------------------------------------------
# keys
# --------------------------------------------------------------------------
def test_bootstrapping_key_rows_encrypt_gadget_times_key_bit(real_oracle):
    o = real_oracle
    s, S = o.lwe_key(), o.glwe_key().astype(np.uint32)
    bk = o.bk()
    l, N = o.params.l, o.N
    for i in (0, 1, 2, 317, o.n - 1):
        for row in range(2 * l):
            u, j = row // l, row % l + 1
            A, B = bk[i, row, 0], bk[i, row, 1]
            phase = (B.astype(np.int64) - O.negacyclic_schoolbook(A, S).astype(np.int64)) % Q
            g = 1 << (32 - 7 * j)
            want = np.zeros(N, np.int64)
            if s[i]:
                if u == 1:
                    want[0] = g
                else:
                    want = (-(g * S.astype(np.int64))) % Q
            err = centered((phase - want) % Q)
            assert np.abs(err).max() < (1 << 10), (i, row)


def test_keyswitching_key_rows(real_oracle):
    o = real_oracle
    S = o.glwe_key()
    ksk = o.ksk()
    for i in (0, 5, 1023):
        for j in range(8):
            for v in (1, 2, 3):
                ph = int(o.phase(ksk[i, j, v - 1])[0])
                want = (v * int(S[i]) << (30 - 2 * j)) % Q
                assert abs(int(centered((ph - want) % Q))) < (1 << 21)


def test_encryption_noise_statistics(real_oracle):
    o = real_oracle
    mu = np.full(20000, 12345, np.uint32)
    ct = o.encrypt(mu, stream=5)
    err = centered(o.phase(ct).astype(np.int64) - 12345).astype(np.float64)
    sigma = o.params.lwe_sigma * Q
    assert abs(err.mean()) < 0.05 * sigma
    assert 0.95 < err.std() / sigma < 1.05
    # encryption is deterministic in (seed, stream, index) and differs across streams
    assert np.array_equal(o.encrypt(mu[:3], stream=5), ct[:3])
    assert np.array_equal(o.encrypt(mu[:3], stream=5, first_index=10), ct[10:13])
    assert not np.array_equal(o.encrypt(mu[:3], stream=6), ct[:3])


def test_bit_encoding_decrypts(real_oracle):
    bits = np.array([0, 1, 1, 0, 1], np.uint8)
    ct = real_oracle.encrypt_bits(bits, stream=7)
    assert list(real_oracle.decrypt_bits(ct)) == list(bits)
    ph = centered(real_oracle.phase(ct))
    assert np.all(np.abs(ph - np.where(bits == 1, E8, -E8)) < (1 << 20))


# --------------------------------------------------------------------------
# bootstrap pieces
# --------------------------------------------------------------------------
def glwe_encrypt_manual(o, msg, rng):
    """(A, B) with B = A*S + msg + e, built in the test from the oracle's key."""
    N = o.N
    S = o.glwe_key().astype(np.uint32)
    A = rng.integers(0, Q, N, dtype=np.uint64).astype(np.uint32)
    e = rng.integers(-8, 9, N)
    B = (O.negacyclic_schoolbook(A, S).astype(np.int64) + msg + e) % Q
    return np.concatenate([A, B.astype(np.uint32)])


def test_sample_extract_identity(toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(3)
    S = o.glwe_key().astype(np.uint32)
    acc = rng.integers(0, Q, 2 * o.N, dtype=np.uint64).astype(np.uint32)
    big = o.sample_extract(acc)
    phase_poly = (acc[o.N:].astype(np.int64) - O.negacyclic_schoolbook(acc[:o.N], S).astype(np.int64)) % Q
    assert int(o.phase_big(big)[0]) == int(phase_poly[0])


@pytest.mark.parametrize("which", ["toy", "real"])
def test_external_product_multiplies_phase_by_key_bit(which, toy_oracle, real_oracle):
    o = toy_oracle if which == "toy" else real_oracle
    rng = np.random.default_rng(4)
    N = o.N
    S = o.glwe_key().astype(np.uint32)
    msg = rng.integers(0, Q, N).astype(np.int64)
    ct = glwe_encrypt_manual(o, msg, rng)
    s = o.lwe_key()
    for i in [int(np.argmax(s == 0)), int(np.argmax(s == 1))]:
        out = o.external_product(i, ct)
        phase = (out[N:].astype(np.int64) - O.negacyclic_schoolbook(out[:N], S).astype(np.int64)) % Q
        want = msg * int(s[i]) % Q
        err = centered((phase - want) % Q)
        # decomposition error N * 2^10 at most, plus key noise times digits
        assert np.abs(err).max() < (1 << 22), (which, i, int(np.abs(err).max()))


@pytest.mark.parametrize("which", ["toy", "real"])
def test_blind_rotation_sign_follows_rounded_phase(which, toy_oracle, real_oracle):
    o = toy_oracle if which == "toy" else real_oracle
    rng = np.random.default_rng(6)
    s = o.lwe_key().astype(np.int64)
    N = o.N
    trials = 12 if which == "toy" else 2
    for _ in range(trials):
        lwe = rng.integers(0, Q, o.n + 1, dtype=np.uint64).astype(np.uint32)
        bar = np.array([O.modswitch(int(x), N) for x in lwe], np.int64)
        phi = (bar[-1] - (bar[:-1] * s).sum()) % (2 * N)
        acc = o.blind_rotate(lwe)
        big = o.sample_extract(acc)
        ph = int(centered(o.phase_big(big))[0])
        want = E8 if phi < N else -E8
        assert abs(ph - want) < (1 << 26), (phi, ph)


def test_keyswitch_preserves_phase(real_oracle):
    o = real_oracle
    rng = np.random.default_rng(8)
    S = o.glwe_key().astype(np.int64)
    for mu in (E8, Q - E8, 12345678):
        a = rng.integers(0, Q, o.N).astype(np.int64)
        b = ((a * S).sum() + mu + 3) % Q
        big = np.concatenate([a, [b]]).astype(np.uint32)
        out = o.keyswitch(big)
        err = int(centered((int(o.phase(out)[0]) - mu) % Q))
        assert abs(err) < (1 << 26), err


def ks_digits_closed_form(x):
    """Keyswitch digits of the word x, from the definition of rounding to the
    nearest multiple of 2^16 with ties up: v = floor((x + 2^15) / 2^16) mod
    2^16, written in base 4, most significant digit first (weights 2^30,
    2^28, ..., 2^16)."""
    v = ((int(x) + (1 << 15)) // (1 << 16)) % (1 << 16)
    return [(v >> (14 - 2 * j)) & 3 for j in range(8)]


# words whose low 16 bits sit on, just below and just above the rounding tie
# (truncation and ties-down give other digits there), the wrap to zero at the
# top, and random words
KS_PIN_WORDS = [0x00008000, 0x00007FFF, 0x00008001, 0x12348000, 0x1234FFFF, 0xFFFF8000, 0xFFFF7FFF,
                0x7FFF8000, 0x55558000, 0xAAAA7FFF, 0x00000000, 0xFFFFFFFF, 0xC0DE1234, 0x3FFFC000]


def test_keyswitch_rounding_digits_exact(real_oracle):
    """One nonzero mask word: the keyswitch must return exactly (0, .., 0, b)
    minus the key rows KSK[i][j][d_j - 1] selected by the closed-form digits
    (a row per nonzero digit).  Plain truncation, ties-down rounding, a
    reversed digit order or a wrong row index gives other words."""
    o = real_oracle
    ksk = o.ksk().astype(np.int64)
    rng = np.random.default_rng(31)
    body = 0x0BADF00D
    words = KS_PIN_WORDS + [int(w) for w in rng.integers(0, Q, 10)]
    for k, x in enumerate(words):
        i = [0, 1, 511, 1023][k % 4]
        big = np.zeros(o.N + 1, np.uint32)
        big[i] = x
        big[o.N] = body
        want = np.zeros(o.n + 1, np.int64)
        want[o.n] = body
        for j, d in enumerate(ks_digits_closed_form(x)):
            if d:
                want -= ksk[i, j, d - 1]
        assert np.array_equal(o.keyswitch(big), (want % Q).astype(np.uint32)), hex(x)
    # ties: the digits of 2^15 are those of 2^16 (rounded up), not of 0
    assert ks_digits_closed_form(0x8000) == [0] * 7 + [1]
    assert ks_digits_closed_form(0xFFFF8000) == [0] * 8


def test_keyswitch_exact_phase_relation(real_oracle):
    """For any input, phase(KS(c)) = b - sum_i S_i round16(a_i) - (sum of the
    noise of the selected key rows), exactly mod q, where round16 is the
    closed-form rounding above and each row's noise is its phase minus
    d S_i 2^(30 - 2j).  The mean of the rounding part over many inputs is
    about zero; truncation would shift it by about 2^24."""
    o = real_oracle
    S = o.glwe_key().astype(np.int64)
    ksk = o.ksk()
    nd = ksk.shape[2]
    rows = ksk.reshape(-1, o.n + 1)
    row_phase = o.phase(rows).astype(np.int64).reshape(o.N, 8, nd)
    dv = np.arange(1, nd + 1, dtype=np.int64)
    weight = np.array([1 << (30 - 2 * j) for j in range(8)], np.int64)
    row_noise = (row_phase - (dv[None, None, :] * S[:, None, None] * weight[None, :, None])) % Q
    rng = np.random.default_rng(77)
    rounding_parts = []
    for _ in range(24):
        a = rng.integers(0, Q, o.N).astype(np.int64)
        b = int(rng.integers(0, Q))
        big = np.concatenate([a, [b]]).astype(np.uint32)
        got = int(o.phase(o.keyswitch(big))[0])
        rounded = np.array([((int(x) + (1 << 15)) >> 16) % (1 << 16) for x in a], np.int64) << 16
        noise = 0
        for i in range(o.N):
            for j, d in enumerate(ks_digits_closed_form(a[i])):
                if d:
                    noise += int(row_noise[i, j, d - 1])
        want = (b - int((S * rounded).sum()) - noise) % Q
        assert got == want
        rounding_parts.append(int(centered(int((S * ((a - rounded) % Q)).sum()) % Q)))
    assert abs(np.mean(rounding_parts)) < (1 << 21), np.mean(rounding_parts)


# --------------------------------------------------------------------------
# gates: full truth tables
# --------------------------------------------------------------------------
TRUTH = {"NAND": [1, 1, 1, 0], "AND": [0, 0, 0, 1], "OR": [0, 1, 1, 1], "XOR": [0, 1, 1, 0],
         "XNOR": [1, 0, 0, 1], "NOR": [1, 0, 0, 0], "ANDNY": [0, 1, 0, 0], "ANDYN": [0, 0, 1, 0],
         "ORNY": [1, 1, 0, 1], "ORYN": [1, 0, 1, 1]}  # index = 2*x + y


def test_gate_plain_truth_tables():
    for name, tt in TRUTH.items():
        for x in (0, 1):
            for y in (0, 1):
                assert O.gate_plain(O.GATES[name], x, y) == tt[2 * x + y], name


def test_all_gates_truth_tables_toy(toy_oracle):
    o = toy_oracle
    xs = np.array([0, 0, 1, 1], np.uint8)
    ys = np.array([0, 1, 0, 1], np.uint8)
    for rep in range(3):
        cx = o.encrypt_bits(xs, stream=20 + rep)
        cy = o.encrypt_bits(ys, stream=40 + rep)
        for name, tt in TRUTH.items():
            gates = np.full(4, O.GATES[name], np.int32)
            out = o.gate_batch(gates, cx, cy)
            assert list(o.decrypt_bits(out)) == tt, name
            # fresh-looking output: phase within q/16 of +-q/8
            ph = centered(o.phase(out))
            assert np.all(np.abs(np.abs(ph) - E8) < (1 << 27))


def test_chained_gates_toy(toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(10)
    bits = rng.integers(0, 2, 64).astype(np.uint8)
    ct = o.encrypt_bits(bits, stream=60)
    val, cval = bits[0], ct[0]
    names = list(TRUTH)
    for k in range(1, 64):
        name = names[k % len(names)]
        cval = o.gate(O.GATES[name], cval, ct[k])
        val = TRUTH[name][2 * int(val) + int(bits[k])]
        assert o.decrypt_bits(cval)[0] == val


def test_not_is_free_negation(toy_oracle):
    o = toy_oracle
    ct = o.encrypt_bits(np.array([1, 0], np.uint8), stream=3)
    assert list(o.decrypt_bits(np.stack([o.not_(ct[0]), o.not_(ct[1])]))) == [0, 1]


def test_gates_real_params(real_oracle):
    o = real_oracle
    cx = o.encrypt_bits(np.array([0, 1, 1, 1], np.uint8), stream=21)
    cy = o.encrypt_bits(np.array([1, 1, 0, 1], np.uint8), stream=22)
    gates = np.array([O.GATES[g] for g in ("AND", "XNOR", "ANDNY", "OR")], np.int32)
    out = o.gate_batch(gates, cx, cy)
    assert list(o.decrypt_bits(out)) == [0, 1, 0, 1]
    # different keys, same inputs: different words (the words depend on the keys)
    assert not np.array_equal(out[0], cx[0])


# --------------------------------------------------------------------------
# netlists
# --------------------------------------------------------------------------
def test_netlist_gate_counts_match_workload_definitions():
    preds = {"EQ": O.P_EQ, "LT": O.P_LT, "RANGE": O.P_RANGE}
    for pred, w, npay, pw, rows, per_row, total, nx, nand, _ in read_golden("netlist_gate_counts.txt"):
        t, a, b, m, ninp = O.netlist(preds[pred], int(w), int(npay), int(pw))
        assert t.size == int(per_row) and t.size * int(rows) == int(total)
        if nx != "-":
            assert int((t == O.GATES["XNOR"]).sum()) == int(nx)
            assert int((t == O.GATES["AND"]).sum()) == int(nand)


def test_majority_gate_plain_and_counts():
    for x in (0, 1):
        for y in (0, 1):
            for z in (0, 1):
                assert O.gate_plain3(O.GATES["MAJNYY"], x, y, z) == int((1 - x) + y + z >= 2)
    # a w-bit majority comparator is w gates (one ANDNY, w-1 majorities) instead of 4w-3
    t, a, b, c, m, ninp = O.netlist3(O.P_LT_MAJ, 16)
    assert t.size == 16 and (t == O.GATES["MAJNYY"]).sum() == 15 and (c >= 0).sum() == 15
    t, *_ = O.netlist3(O.P_RANGE_MAJ, 16, 2, 16)
    assert t.size == 16 + 16 + 1 + 32  # vs 155 with ripple comparators


@pytest.mark.parametrize("which", ["toy", "real"])
def test_majority_gate_truth_table_encrypted(which, toy_oracle, real_oracle):
    o = toy_oracle if which == "toy" else real_oracle
    combos = [(x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)]
    if which == "real":
        combos = combos[::3]
    cts = o.encrypt_bits(np.array([v for cmb in combos for v in cmb], np.uint8), stream=33).reshape(-1, 3, o.n + 1)
    for (x, y, z), ct in zip(combos, cts):
        out = o.gate3(O.GATES["MAJNYY"], ct[0], ct[1], ct[2])
        assert o.decrypt_bits(out)[0] == int((1 - x) + y + z >= 2)
        assert abs(abs(int(centered(o.phase(out))[0])) - E8) < (1 << 27)


@pytest.mark.parametrize("pred", [O.P_EQ, O.P_LT, O.P_RANGE, O.P_LT_MAJ, O.P_RANGE_MAJ])
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_netlist_brute_force(pred, w):
    rng = pred in (O.P_RANGE, O.P_RANGE_MAJ)
    for c in range(1 << w):
        for k in range(1 << w):
            for k2 in (range(1 << w) if rng else [None]):
                pay = (c * 5 + 3) % (1 << w)
                inp = [(c >> i) & 1 for i in range(w)] + [(k >> i) & 1 for i in range(w)]
                if rng:
                    inp += [(k2 >> i) & 1 for i in range(w)]
                inp += [(pay >> i) & 1 for i in range(w)]
                wires, m = O.netlist_eval_plain(pred, w, 1, w, np.array(inp, np.uint8))
                want = {O.P_EQ: c == k, O.P_LT: c < k, O.P_LT_MAJ: c < k,
                        O.P_RANGE: rng and k <= c < (k2 or 0), O.P_RANGE_MAJ: rng and k <= c < (k2 or 0)}[pred]
                assert wires[m] == int(want)
                out = wires[-w:]
                assert int(sum(int(out[i]) << i for i in range(w))) == (pay if want else 0)


# --------------------------------------------------------------------------
# the scan end to end (toy parameters) against the plaintext SQL answer
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pred", [O.P_EQ, O.P_LT, O.P_RANGE, O.P_LT_MAJ, O.P_RANGE_MAJ])
def test_scan_toy_matches_plaintext_sql(pred, toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(100 + pred)
    w, rows = 4, 16
    c = rng.integers(0, 16, rows)
    pay = rng.integers(0, 16, rows)
    if pred in (O.P_RANGE, O.P_RANGE_MAJ):
        lo, hi = 3, 11
        kbits = [(lo >> i) & 1 for i in range(w)] + [(hi >> i) & 1 for i in range(w)]
    else:
        k = int(c[5])
        kbits = [(k >> i) & 1 for i in range(w)]
    col = o.encrypt_bits(np.array([(v >> i) & 1 for v in c for i in range(w)], np.uint8), stream=5)
    pct = o.encrypt_bits(np.array([(v >> i) & 1 for v in pay for i in range(w)], np.uint8), stream=9)
    kct = o.encrypt_bits(np.array(kbits, np.uint8), stream=7)
    match, (outp,) = o.scan(pred, w, col, kct, [pct], w)
    mbits = o.decrypt_bits(match)
    obits = o.decrypt_bits(outp.reshape(-1, o.n + 1)).reshape(rows, w)
    for r in range(rows):
        if pred in (O.P_RANGE, O.P_RANGE_MAJ):
            want = lo <= c[r] < hi
        else:
            want = c[r] == k if pred == O.P_EQ else c[r] < k
        assert mbits[r] == int(want)
        got = int(sum(int(obits[r, i]) << i for i in range(w)))
        assert got == (int(pay[r]) if want else 0)


# --------------------------------------------------------------------------
# plaintext query constants: reduced netlists, copies and trivial outputs
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pred", [O.P_EQ, O.P_LT, O.P_RANGE])
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_plain_constant_netlist_brute_force(pred, w):
    """Every column value x every constant (every lo, hi pair for RANGE):
    the reduced netlist computes the SQL predicate and the masked payload."""
    rng = pred == O.P_RANGE
    for k in range(1 << w):
        for k2 in (range(1 << w) if rng else [0]):
            consts = (k, k2) if rng else (k,)
            for c in range(1 << w):
                pay = (c * 5 + 3) % (1 << w)
                inp = [(c >> i) & 1 for i in range(w)] + [(pay >> i) & 1 for i in range(w)]
                m, out = O.netlist_plain_eval(pred, w, 1, w, consts, np.array(inp, np.uint8))
                want = {O.P_EQ: c == k, O.P_LT: c < k, O.P_RANGE: k <= c < k2}[pred]
                assert m == int(want), (consts, c)
                assert int(sum(int(out[i]) << i for i in range(w))) == (pay if want else 0)


def test_plain_constant_gate_counts_closed_form():
    """EQ: w - 1 ANDs; LT: one gate per bit above the lowest set bit of k
    (none for k = 0, the predicate is then false); masks add one gate per
    payload bit unless the match is a known bit."""
    for w in (1, 5, 16, 32):
        for k in sorted({0, 1, 2, 6, (1 << w) - 1, 1 << (w - 1)}):
            if k >= 1 << w:
                continue
            t, _, _, m, ol, _ = O.netlist_plain(O.P_EQ, w, 1, w, (k,))
            assert t.size == (w - 1) + w
            t, _, _, m, ol, _ = O.netlist_plain(O.P_LT, w, 0, 0, (k,))
            low = (k & -k).bit_length() - 1
            assert t.size == (0 if k == 0 else w - 1 - low)
            assert (m == O.LIT_FALSE) == (k == 0)
    # k = 0: no gate at all, every output a known bit
    t, _, _, m, ol, _ = O.netlist_plain(O.P_LT, 8, 2, 8, (0,))
    assert t.size == 0 and m == O.LIT_FALSE and np.all(ol == O.LIT_FALSE)
    # RANGE with lo = 0: not(c < 0) is true, so match = (c < hi)
    t, _, _, m, _, _ = O.netlist_plain(O.P_RANGE, 16, 0, 0, (0, 6554))
    t2, _, _, m2, _, _ = O.netlist_plain(O.P_LT, 16, 0, 0, (6554,))
    assert t.size == t2.size and m == m2


@pytest.mark.parametrize("pred,consts", [(O.P_EQ, (9,)), (O.P_LT, (11,)), (O.P_RANGE, (3, 12)),
                                         (O.P_LT, (0,)), (O.P_LT, (8,)), (O.P_RANGE, (0, 16 - 1)),
                                         (O.P_EQ, (0,))])
def test_scan_plain_toy_matches_plaintext_sql(pred, consts, toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(200 + pred + sum(consts))
    w, rows = 4, 16
    c = rng.integers(0, 16, rows)
    pay = rng.integers(0, 16, rows)
    col = o.encrypt_bits(np.array([(v >> i) & 1 for v in c for i in range(w)], np.uint8), stream=5)
    pct = o.encrypt_bits(np.array([(v >> i) & 1 for v in pay for i in range(w)], np.uint8), stream=9)
    match, (outp,) = o.scan_plain(pred, w, col, consts, [pct], w)
    mbits = o.decrypt_bits(match)
    obits = o.decrypt_bits(outp.reshape(-1, o.n + 1)).reshape(rows, w)
    for r in range(rows):
        want = {O.P_EQ: c[r] == consts[0], O.P_LT: c[r] < consts[0],
                O.P_RANGE: consts[0] <= c[r] < consts[-1]}[pred]
        assert mbits[r] == int(want)
        assert int(sum(int(obits[r, i]) << i for i in range(w))) == (int(pay[r]) if want else 0)
    # outputs that are not gate outputs are exact copies, negations or trivial ciphertexts
    _, _, _, m, ol, _ = O.netlist_plain(pred, w, 1, w, consts)
    col3 = col.reshape(rows, w, o.n + 1).astype(np.int64)
    if m == O.LIT_FALSE:
        assert np.all(match[:, :o.n] == 0) and np.all(match[:, o.n] == np.uint32((Q - E8) % Q))
        assert np.all(outp[:, :, :o.n] == 0) and np.all(outp[:, :, o.n] == np.uint32((Q - E8) % Q))
    elif m >= 0 and (m >> 1) < w:
        src = col3[:, m >> 1]
        want = (-src) % Q if m & 1 else src
        assert np.array_equal(match.astype(np.int64), want)


def test_scan_plain_equality_at_real_params(real_oracle):
    """One 3-bit row at the real parameters, a match and a miss."""
    o = real_oracle
    w = 3
    col = o.encrypt_bits(np.array([1, 0, 1, 0, 1, 1], np.uint8), stream=5)  # rows 5, 6
    pct = o.encrypt_bits(np.array([1, 1, 0, 0, 1, 1], np.uint8), stream=9)  # payloads 3, 6
    match, (outp,) = o.scan_plain(O.P_EQ, w, col, (5,), [pct], w)
    assert list(o.decrypt_bits(match)) == [1, 0]
    assert list(o.decrypt_bits(outp.reshape(-1, o.n + 1))) == [1, 1, 0, 0, 0, 0]


# --------------------------------------------------------------------------
# SUM aggregation: full-adder gates and the carry-save tree
# --------------------------------------------------------------------------
def test_full_adder_gates_plain():
    for x in (0, 1):
        for y in (0, 1):
            for z in (0, 1):
                assert O.gate_plain3(O.GATES["XOR3"], x, y, z) == (x + y + z) % 2
                assert O.gate_plain3(O.GATES["MAJ"], x, y, z) == int(x + y + z >= 2)


@pytest.mark.parametrize("which", ["toy", "real"])
@pytest.mark.parametrize("gate", ["XOR3", "MAJ"])
def test_full_adder_gates_encrypted(which, gate, toy_oracle, real_oracle):
    """Every input triple (toy) or a spread of them (real parameters): the
    bootstrapped output decrypts to the truth table at +-q/8."""
    o = toy_oracle if which == "toy" else real_oracle
    combos = [(x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)]
    if which == "real":
        combos = combos[1::2]
    cts = o.encrypt_bits(np.array([v for cmb in combos for v in cmb], np.uint8), stream=34).reshape(-1, 3, o.n + 1)
    for (x, y, z), ct in zip(combos, cts):
        out = o.gate3(O.GATES[gate], ct[0], ct[1], ct[2])
        want = (x + y + z) % 2 if gate == "XOR3" else int(x + y + z >= 2)
        assert o.decrypt_bits(out)[0] == want
        assert abs(abs(int(centered(o.phase(out))[0])) - E8) < (1 << 27)


def test_full_adder_lincomb_phases_closed_form():
    """Before the bootstrap, the three-input forms put t true inputs at
    (2t - 3) q/8 (MAJ) and -(2t - 3) q/4 (XOR3), exactly, on noiseless
    trivial ciphertexts."""
    n = 4
    enc = lambda v: np.array([0] * n + [E8 if v else (Q - E8)], np.uint32)
    for x in (0, 1):
        for y in (0, 1):
            for z in (0, 1):
                t = x + y + z
                c = [enc(x), enc(y), enc(z)]
                maj = O.gate_lincomb3(O.GATES["MAJ"], n, *c)
                xor3 = O.gate_lincomb3(O.GATES["XOR3"], n, *c)
                assert int(maj[n]) == ((2 * t - 3) * E8) % Q
                assert int(xor3[n]) == (-(2 * t - 3) * 2 * E8) % Q


def test_sum_circuit_exhaustive_small():
    """Every value combination for tiny tables: the circuit's plaintext
    evaluation equals the integer sum mod 2^ow."""
    import itertools

    for rows in (1, 2, 3, 4):
        for pw in (1, 2):
            for ow in sorted({1, pw, pw + 1, pw + 3}):
                for vals in itertools.product(range(1 << pw), repeat=rows):
                    assert O.sum_eval_plain(rows, pw, ow, vals) == sum(vals) % (1 << ow), (rows, pw, ow, vals)


def test_sum_circuit_random_larger():
    rng = np.random.default_rng(9)
    for rows, pw, ow in [(5, 3, 6), (7, 4, 7), (16, 8, 12), (33, 5, 11), (100, 16, 23), (9, 4, 3)]:
        for _ in range(20):
            vals = [int(v) for v in rng.integers(0, 1 << pw, rows)]
            assert O.sum_eval_plain(rows, pw, ow, vals) == sum(vals) % (1 << ow)
    # extreme values: every bit set
    for rows, pw in [(64, 8), (17, 16)]:
        ow = pw + 7
        assert O.sum_eval_plain(rows, pw, ow, [(1 << pw) - 1] * rows) == rows * ((1 << pw) - 1) % (1 << ow)


def test_sum_circuit_shape():
    """Only full adders (XOR3 with MAJ) and half adders (XOR with AND) appear,
    paired except in the top column, which drops its carry; a single row
    needs no gate at all (outputs are its bits and known zeros)."""
    t, a, b, c, ol, ninp = O.sum_netlist(1, 8, 10)
    assert t.size == 0 and list(ol[:8]) == [2 * j for j in range(8)] and all(ol[8:] == O.LIT_FALSE)
    t, a, b, c, ol, ninp = O.sum_netlist(4096, 32, 44)
    kinds = {int(k) for k in np.unique(t)}
    assert kinds <= {O.GATES["XOR3"], O.GATES["MAJ"], O.GATES["XOR"], O.GATES["AND"]}
    n_xor3, n_maj = int((t == O.GATES["XOR3"]).sum()), int((t == O.GATES["MAJ"]).sum())
    n_xor, n_and = int((t == O.GATES["XOR"]).sum()), int((t == O.GATES["AND"]).sum())
    assert 0 <= n_xor3 - n_maj and 0 <= n_xor - n_and <= 1
    assert np.all(c[(t == O.GATES["XOR3"]) | (t == O.GATES["MAJ"])] >= 0)


def test_aggregate_sum_toy_decrypts_to_sum(toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(12)
    for rows, pw, ow in [(6, 3, 6), (1, 4, 6), (9, 2, 3)]:
        vals = rng.integers(0, 1 << pw, rows)
        bits = np.array([(int(v) >> j) & 1 for v in vals for j in range(pw)], np.uint8)
        ct = o.encrypt_bits(bits, stream=40 + rows)
        out = o.aggregate_sum(ct, rows, pw, ow)
        got = o.decrypt_bits(out)
        assert int(sum(int(got[j]) << j for j in range(ow))) == int(vals.sum()) % (1 << ow)
        if rows == 1:  # no gate: copies of the input bits and trivial zeros
            assert np.array_equal(out[:pw], ct.reshape(pw, -1))
            assert np.all(out[pw:, :o.n] == 0) and np.all(out[pw:, o.n] == np.uint32(Q - E8))


# --------------------------------------------------------------------------
# MAX / MIN of the selected rows: comparator + multiplexer tournament
# --------------------------------------------------------------------------
def test_extreme_circuits_exhaustive_small():
    """Every value (and match) combination for tiny tables: MAX is the
    largest masked value (0 for no rows), MIN the smallest selected value
    (2^w - 1 when nothing is selected)."""
    import itertools

    for w in (1, 2, 3):
        for rows in range(0, 5):
            for vals in itertools.product(range(1 << w), repeat=rows):
                assert O.extreme_eval_plain(False, w, vals) == (max(vals) if vals else 0)
                for m in itertools.product((0, 1), repeat=rows):
                    sel = [v for v, mm in zip(vals, m) if mm]
                    assert O.extreme_eval_plain(True, w, vals, m) == (min(sel) if sel else (1 << w) - 1)


def test_extreme_circuits_random_and_counts():
    rng = np.random.default_rng(21)
    for rows, w in [(7, 8), (33, 5), (100, 16), (64, 32)]:
        for _ in range(10):
            vals = [int(v) for v in rng.integers(0, 1 << w, rows, dtype=np.uint64)]
            m = [int(v) for v in rng.integers(0, 2, rows)]
            sel = [v for v, mm in zip(vals, m) if mm]
            assert O.extreme_eval_plain(False, w, vals) == max(vals)
            assert O.extreme_eval_plain(True, w, vals, m) == (min(sel) if sel else (1 << w) - 1)
        # (rows - 1) pairwise steps of w comparator gates and 3w multiplexer gates; MIN adds w per row
        assert O.extreme_netlist(False, rows, w)[0].size == 4 * w * (rows - 1)
        assert O.extreme_netlist(True, rows, w)[0].size == 4 * w * (rows - 1) + w * rows


def test_aggregate_extreme_toy_decrypts(toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(22)
    rows, w = 5, 3
    vals = rng.integers(0, 8, rows)
    m = np.array([1, 0, 1, 1, 0], np.uint8)
    ct = o.encrypt_bits(np.array([(int(v) >> j) & 1 for v in vals for j in range(w)], np.uint8), stream=50)
    mct = o.encrypt_bits(m, stream=51)
    dec = lambda out: int(sum(int(b) << j for j, b in enumerate(o.decrypt_bits(out))))
    assert dec(o.aggregate_extreme(False, ct, rows, w)) == int(vals.max())
    assert dec(o.aggregate_extreme(True, ct, rows, w, mct)) == int(vals[m == 1].min())
    one = o.aggregate_extreme(False, ct[:w], 1, w)  # one row: its own ciphertexts
    assert np.array_equal(one, ct[:w].reshape(w, -1))


# --------------------------------------------------------------------------
# keyswitch-first order: ciphertexts under the N-bit key
# --------------------------------------------------------------------------
def test_big_key_encryption_noise_and_phase(real_oracle):
    """Fresh N-bit-key ciphertexts: phase = +-q/8 + e with e of the GLWE
    noise (sigma 2^-25, i.e. 2^7 in torus units), exactly b - <a, S>."""
    o = real_oracle
    rng = np.random.default_rng(31)
    bits = rng.integers(0, 2, 2000).astype(np.uint8)
    ct = o.encrypt_big_bits(bits, 70)
    assert ct.shape == (2000, o.N + 1)
    S = o.glwe_key().astype(np.int64)
    ph = (ct[:, o.N].astype(np.int64) - (ct[:, :o.N].astype(np.int64) * S).sum(axis=1)) % Q
    assert np.array_equal(ph.astype(np.uint32), o.phase_big(ct))
    e = centered(ph - np.where(bits == 1, E8, Q - E8))
    assert abs(e.mean()) < 10 and 110 < e.std() < 146
    assert np.array_equal(o.decrypt_big_bits(ct), bits)
    # the same (stream, index) gives the same ciphertext
    assert np.array_equal(o.encrypt_big_bits(bits[5:9], 70, 5), ct[5:9])


@pytest.mark.parametrize("which", ["toy", "real"])
def test_ks_first_gates_truth_tables(which, toy_oracle, real_oracle):
    """Every two-input gate on every input pair and the three-input gates on
    every triple (a spread of them at real parameters): the keyswitch-first
    gate decrypts to the truth table with phase near +-q/8."""
    o = toy_oracle if which == "toy" else real_oracle
    pairs = [(x, y) for x in (0, 1) for y in (0, 1)]
    cts = o.encrypt_big_bits(np.array([1, 0, 1, 1, 0], np.uint8), 71)
    bit_ct = {0: cts[1], 1: cts[0]}
    bit_ct2 = {0: cts[4], 1: cts[2]}
    gates2 = [g for g in range(10)] if which == "toy" else [0, 3, 4, 6, 9]
    for g in gates2:
        for x, y in pairs:
            out = o.gate3_ks_first(g, bit_ct[x], bit_ct2[y])
            assert o.decrypt_big_bits(out)[0] == O.gate_plain(g, x, y), (g, x, y)
            assert abs(abs(int(centered(o.phase_big(out))[0])) - E8) < (1 << 27)
    triples = [(x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)]
    if which == "real":
        triples = triples[::3]
    third = {0: o.encrypt_big_bits(np.array([0], np.uint8), 72)[0], 1: o.encrypt_big_bits(np.array([1], np.uint8), 72, 1)[0]}
    for g in (O.GATES["MAJNYY"], O.GATES["XOR3"], O.GATES["MAJ"]):
        for x, y, z in triples:
            out = o.gate3_ks_first(g, bit_ct[x], bit_ct2[y], third[z])
            assert o.decrypt_big_bits(out)[0] == O.gate_plain3(g, x, y, z), (g, x, y, z)


def test_ks_first_identity_gate_is_bootstrap_of_keyswitch(real_oracle):
    """AND with a noiseless trivial true input is the identity on the linear
    combination, so the keyswitch-first gate must equal keyswitch, blind
    rotation and extraction of the input itself."""
    o = real_oracle
    x = o.encrypt_big_bits(np.array([1, 0], np.uint8), 73)
    T = np.zeros(o.N + 1, np.uint32)
    T[o.N] = E8
    for k in range(2):
        got = o.gate3_ks_first(O.GATES["AND"], x[k], T)
        want = o.sample_extract(o.blind_rotate(o.keyswitch(x[k])))
        assert np.array_equal(got, want)


@pytest.mark.parametrize("pred", [O.P_EQ, O.P_RANGE_MAJ])
def test_scan_ks_first_toy_matches_plaintext_sql(pred, toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(300 + pred)
    w, rows = 4, 12
    c = rng.integers(0, 16, rows)
    pay = rng.integers(0, 16, rows)
    if pred == O.P_RANGE_MAJ:
        lo, hi = 3, 11
        kbits = [(lo >> i) & 1 for i in range(w)] + [(hi >> i) & 1 for i in range(w)]
    else:
        k = int(c[3])
        kbits = [(k >> i) & 1 for i in range(w)]
    col = o.encrypt_big_bits(np.array([(v >> i) & 1 for v in c for i in range(w)], np.uint8), 5)
    pct = o.encrypt_big_bits(np.array([(v >> i) & 1 for v in pay for i in range(w)], np.uint8), 6)
    kct = o.encrypt_big_bits(np.array(kbits, np.uint8), 7)
    match, (outp,) = o.scan_ks_first(pred, w, col, kct, [pct], w)
    mbits = o.decrypt_big_bits(match)
    obits = o.decrypt_big_bits(outp.reshape(-1, o.N + 1)).reshape(rows, w)
    for r in range(rows):
        want = (lo <= c[r] < hi) if pred == O.P_RANGE_MAJ else c[r] == k
        assert mbits[r] == int(want)
        assert int(sum(int(obits[r, i]) << i for i in range(w))) == (int(pay[r]) if want else 0)
