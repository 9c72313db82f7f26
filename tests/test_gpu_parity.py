"""GPU parity: the CUDA path against the CPU oracle, bit-exact on every output
word (this is integer cryptographic work; nothing is rounded), through the
C-ABI library.  Inputs: both sides encrypt the same seeded plaintexts with
their own code (their ciphertexts are asserted equal first)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_15413_b300 import fhesql as F
from paper_2510_15413_b300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 2510


@pytest.fixture(scope="module")
def oracle_ctx():
    O.set_threads(os.cpu_count() or 1)
    o = O.Oracle(SEED)
    yield o
    o.close()


@pytest.fixture(scope="module", params=["dual_prime", "goldilocks"])
def env(request, oracle_ctx):
    """Every parity test runs on both exact NTT engines."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = F.Context(SEED, device=0, engine=request.param)
    yield ctx, oracle_ctx
    ctx.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def both_encrypt_bits(ctx, o, bits, stream, first=0):
    a = ctx.encrypt_bits(bits, stream, first)
    b = o.encrypt_bits(bits, stream, first)
    assert np.array_equal(a, b)
    return a


# ---------------------------------------------------------------- NTT
def test_ntt_product_matches_schoolbook(env):
    ctx, _ = env
    rng = np.random.default_rng(1)
    cases = [
        (rng.integers(-64, 64, 1024), rng.integers(0, 1 << 32, 1024, dtype=np.uint64)),
        (np.full(1024, -64), np.full(1024, 0xFFFFFFFF, np.uint64)),  # largest |integer coefficient|
        (np.full(1024, 63), np.full(1024, 0xFFFFFFFF, np.uint64)),
        (np.eye(1, 1024, 1023, dtype=np.int64)[0], np.eye(1, 1024, 1, dtype=np.uint64)[0]),  # X^1023 * X = -1
    ]
    for d, a in cases:
        d = d.astype(np.int32)
        a = a.astype(np.uint32)
        out = torch.zeros(1024, dtype=torch.int32, device="cuda")
        ctx.debug_ntt_mul(dev(d), dev(a.view(np.int32)), out)
        got = host(out).view(np.uint32)
        want = O.negacyclic_schoolbook(d.astype(np.int64).astype(np.uint32), a)
        assert np.array_equal(got, want)


# ---------------------------------------------------------------- pieces of one bootstrap
def test_blind_rotate_extract_matches_oracle(env):
    ctx, o = env
    rng = np.random.default_rng(2)
    count = 11  # several CTAs of the small-batch kernel, the last one partly idle
    types = rng.integers(0, 10, count).astype(np.uint8)
    x = both_encrypt_bits(ctx, o, rng.integers(0, 2, count).astype(np.uint8), 30)
    y = both_encrypt_bits(ctx, o, rng.integers(0, 2, count).astype(np.uint8), 31)
    big = torch.zeros((count, 1025), dtype=torch.int32, device="cuda")
    ctx.blind_rotate_extract(dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), big)
    got = host(big).view(np.uint32)
    for g in [0, 5, 8, 10]:
        lin = o.lincomb(int(types[g]), x[g], y[g])
        want = o.sample_extract(o.blind_rotate(lin))
        assert np.array_equal(got[g], want), g


def test_keyswitch_matches_oracle(env):
    ctx, o = env
    rng = np.random.default_rng(3)
    count = 37  # two full 16-gate groups and a ragged one
    big = rng.integers(0, 1 << 32, (count, 1025), dtype=np.uint64).astype(np.uint32)
    big[0, :1024] = 0
    big[1, :1024] = 0xFFFFFFFF
    big[2, :1024] = 1 << 15  # rounding ties
    out = torch.zeros((count, 631), dtype=torch.int32, device="cuda")
    ctx.keyswitch(dev(big.view(np.int32)), out, count)
    got = host(out).view(np.uint32)
    for g in range(count):
        assert np.array_equal(got[g], o.keyswitch(big[g])), g


# ---------------------------------------------------------------- whole gates
def test_gate_batch_every_type_and_input_pair(env):
    ctx, o = env
    types = np.repeat(np.arange(10, dtype=np.uint8), 4)
    xb = np.tile(np.array([0, 0, 1, 1], np.uint8), 10)
    yb = np.tile(np.array([0, 1, 0, 1], np.uint8), 10)
    x = both_encrypt_bits(ctx, o, xb, 40)
    y = both_encrypt_bits(ctx, o, yb, 41)
    out = torch.zeros((40, 631), dtype=torch.int32, device="cuda")
    ctx.gate_batch(dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), out)
    got = host(out).view(np.uint32)
    want = o.gate_batch(types.astype(np.int32), x, y)
    assert np.array_equal(got, want)
    truth = np.array([O.gate_plain(int(t), int(a), int(b)) for t, a, b in zip(types, xb, yb)], np.uint8)
    assert np.array_equal(ctx.decrypt_bits(got), truth)


def test_gate_batch_random_microbench_inputs(env):
    ctx, o = env
    B = 150  # about one gate per SM: the small-batch kernels, a partial last wave
    types, xb, yb = WL.gates(B, seed=5)
    x = both_encrypt_bits(ctx, o, xb, WL.STREAM_GATES, 0)
    y = both_encrypt_bits(ctx, o, yb, WL.STREAM_GATES, B)
    out = torch.zeros((B, 631), dtype=torch.int32, device="cuda")
    ctx.gate_batch(dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), out)
    got = host(out).view(np.uint32)
    sample = np.random.default_rng(6).choice(B, 24, replace=False)
    want = o.gate_batch(types[sample].astype(np.int32), x[sample], y[sample])
    assert np.array_equal(got[sample], want)
    truth = np.array([O.gate_plain(int(t), int(a), int(b)) for t, a, b in zip(types, xb, yb)], np.uint8)
    assert np.array_equal(ctx.decrypt_bits(got), truth)


def test_empty_batches_are_no_ops(env):
    ctx, _ = env
    e = torch.zeros(0, dtype=torch.uint8, device="cuda")
    ctx.gate_batch(e, 0, 0, 0)
    ctx.keyswitch(0, 0, 0)


# ---------------------------------------------------------------- scans
def run_scan(ctx, t, col, cst, pays, per_gate=False):
    W = ctx.words
    dcol, dcst = dev(col.view(np.int32)), dev(cst.view(np.int32))
    dp = [dev(p.view(np.int32)) for p in pays]
    match = torch.zeros((t.rows, W), dtype=torch.int32, device="cuda")
    outs = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda") for _ in pays]
    ctx.scan_select(dcol, t.rows, t.width, t.pred, dcst, dp, t.payload_width, match, outs, per_gate=per_gate)
    return host(match).view(np.uint32), [host(x).view(np.uint32) for x in outs]


def check_plaintext(ctx, t, match, outs):
    m_want, p_want = t.expected()
    assert np.array_equal(ctx.decrypt_bits(match), m_want)
    for q, o_ in enumerate(outs):
        assert np.array_equal(ctx.decrypt_uint(o_, t.payload_width), p_want[q])


def encrypt_both(ctx, o, t):
    lib_ct = WL.encrypt_table(ctx, t)
    orc_ct = WL.encrypt_table(o, t)
    assert all(np.array_equal(a, b) for a, b in zip(lib_ct[:2], orc_ct[:2]))
    assert all(np.array_equal(a, b) for a, b in zip(lib_ct[2], orc_ct[2]))
    return lib_ct, orc_ct


@pytest.mark.parametrize("name,rows", [("eq4x16", 16), ("lt8x64", 5), ("range4x16", 6), ("lt8x64maj", 6),
                                       ("range4x16maj", 7)])
def test_scan_small_tables_bit_exact(env, name, rows):
    ctx, o = env
    t = WL.table(name, seed=3, rows=rows)
    (col, cst, pays), (ocol, ocst, opays) = encrypt_both(ctx, o, t)
    match, outs = run_scan(ctx, t, col, cst, pays)
    om, oouts = o.scan(t.pred, t.width, ocol, ocst, opays, t.payload_width)
    assert np.array_equal(match.reshape(om.shape), om)
    for a, b in zip(outs, oouts):
        assert np.array_equal(a.reshape(b.shape), b)
    check_plaintext(ctx, t, match, outs)


def test_scan_graph_replay_is_stable(env):
    """The second scan on the same buffers replays the captured launch graph."""
    ctx, _ = env
    t = WL.table("range4x16maj", seed=5, rows=4)
    col, cst, pays = WL.encrypt_table(ctx, t)
    dcol, dcst, dp = dev(col.view(np.int32)), dev(cst.view(np.int32)), [dev(p.view(np.int32)) for p in pays]
    match = torch.zeros((t.rows, ctx.words), dtype=torch.int32, device="cuda")
    outs = [torch.zeros((t.rows, t.payload_width, ctx.words), dtype=torch.int32, device="cuda") for _ in pays]
    results = []
    for _ in range(3):
        match.zero_()
        for o_ in outs:
            o_.zero_()
        ctx.scan_select(dcol, t.rows, t.width, t.pred, dcst, dp, t.payload_width, match, outs)
        results.append((host(match).copy(), [host(o_).copy() for o_ in outs]))
    for m, o in results[1:]:
        assert np.array_equal(m, results[0][0]) and all(np.array_equal(a, b) for a, b in zip(o, results[0][1]))
    check_plaintext(ctx, t, results[0][0].view(np.uint32), [x.view(np.uint32) for x in results[0][1]])


def test_scan_per_gate_and_host_paths_equal_batched(env):
    ctx, o = env
    t = WL.table("eq4x16", seed=4)
    col, cst, pays = WL.encrypt_table(ctx, t)
    m1, o1 = run_scan(ctx, t, col, cst, pays, per_gate=False)
    m2, o2 = run_scan(ctx, t, col, cst, pays, per_gate=True)
    assert np.array_equal(m1, m2) and all(np.array_equal(a, b) for a, b in zip(o1, o2))
    m3 = np.zeros_like(m1)
    o3 = [np.zeros_like(x) for x in o1]
    ctx.scan_select_host(col, t.rows, t.width, t.pred, cst, pays, t.payload_width, m3, o3)
    assert np.array_equal(m1, m3) and all(np.array_equal(a, b) for a, b in zip(o1, o3))


def run_scan_plain(ctx, t, col, pays, per_gate=False):
    W = ctx.words
    dcol = dev(col.view(np.int32))
    dp = [dev(p.view(np.int32)) for p in pays]
    match = torch.full((t.rows, W), 7, dtype=torch.int32, device="cuda")  # stale words must be overwritten
    outs = [torch.full((t.rows, t.payload_width, W), 7, dtype=torch.int32, device="cuda") for _ in pays]
    ctx.scan_select_plain(dcol, t.rows, t.width, t.pred, t.consts, dp, t.payload_width, match, outs,
                          per_gate=per_gate)
    return host(match).view(np.uint32), [host(x).view(np.uint32) for x in outs]


# plaintext constants: ordinary constants and the degenerate ones (no gate at
# all, a negated column bit as the match, lo = 0, the largest constants)
@pytest.mark.parametrize("name,rows,consts", [
    ("eq4x16plain", 16, None), ("lt8x64plain", 6, None), ("range4x16plain", 7, None),
    ("lt8x64plain", 5, (0,)), ("lt8x64plain", 5, (128,)), ("lt8x64plain", 5, (255,)),
    ("range4x16plain", 6, (0, 9)), ("range4x16plain", 6, (15, 3)), ("eq4x16plain", 5, (15,)),
])
def test_scan_plain_constants_bit_exact(env, name, rows, consts):
    ctx, o = env
    t = WL.table(name, seed=6, rows=rows)
    if consts is not None:
        t.consts = consts
    (col, _, pays), (ocol, _, opays) = encrypt_both(ctx, o, t)
    match, outs = run_scan_plain(ctx, t, col, pays)
    om, oouts = o.scan_plain(t.pred, t.width, ocol, t.consts, opays, t.payload_width)
    assert np.array_equal(match.reshape(om.shape), om)
    for a, b in zip(outs, oouts):
        assert np.array_equal(a.reshape(b.shape), b)
    check_plaintext(ctx, t, match, outs)


def test_scan_plain_per_gate_equals_batched_and_replays(env):
    ctx, _ = env
    t = WL.table("range4x16plain", seed=7, rows=5)
    col, _, pays = WL.encrypt_table(ctx, t)
    m1, o1 = run_scan_plain(ctx, t, col, pays)
    m2, o2 = run_scan_plain(ctx, t, col, pays, per_gate=True)
    m3, o3 = run_scan_plain(ctx, t, col, pays)
    for m, o_ in ((m2, o2), (m3, o3)):
        assert np.array_equal(m, m1) and all(np.array_equal(a, b) for a, b in zip(o_, o1))


def test_scan_plain_eq32x4096_full_size_sampled_rows(env):
    """Plaintext-constant equality at the benchmark size: every row decrypted
    against the SQL answer, the matching row and the last row recomputed by
    the oracle word for word."""
    ctx, o = env
    t = WL.table("eq32x4096plain", seed=1)
    col, _, pays = WL.encrypt_table(ctx, t)
    match, outs = run_scan_plain(ctx, t, col, pays)
    check_plaintext(ctx, t, match, outs)
    m_want, _ = t.expected()
    rows = sorted({int(np.argmax(m_want)), t.rows - 1})
    ocol = np.concatenate([o.encrypt_bits(t.column_bits().reshape(t.rows, t.width)[r], WL.STREAM_COLUMN,
                                          r * t.width) for r in rows])
    opay = np.concatenate([o.encrypt_bits(t.payload_bits(0).reshape(t.rows, t.payload_width)[r],
                                          WL.STREAM_PAYLOAD, r * t.payload_width) for r in rows])
    om, (oout,) = o.scan_plain(t.pred, t.width, ocol, t.consts, [opay], t.payload_width)
    assert np.array_equal(match.reshape(t.rows, -1)[rows], om)
    assert np.array_equal(outs[0].reshape(t.rows, t.payload_width, -1)[rows], oout)


def test_latency_mode_equals_group_mode_and_oracle(env):
    """Small batches: the latency-mode kernel (one gate per CTA of three
    groups) and the one-group-per-gate kernel give the oracle's words."""
    ctx, o = env
    rng = np.random.default_rng(17)
    for count in (1, 5, 150, 295):
        types = rng.integers(0, 10, count).astype(np.uint8)
        a = both_encrypt_bits(ctx, o, rng.integers(0, 2, count).astype(np.uint8), 60)
        b = both_encrypt_bits(ctx, o, rng.integers(0, 2, count).astype(np.uint8), 61)
        res = []
        for on in (True, False):
            ctx.set_latency_mode(on)
            out = torch.zeros((count, ctx.words), dtype=torch.int32, device="cuda")
            ctx.gate_batch(dev(types), dev(a.view(np.int32)), dev(b.view(np.int32)), out)
            res.append(host(out).view(np.uint32))
        ctx.set_latency_mode(2)
        assert np.array_equal(res[0], res[1]), count
        k = min(count, 4)
        assert np.array_equal(res[0][:k], o.gate_batch(types[:k].astype(np.int32), a[:k], b[:k]))


# ---------------------------------------------------------------- keyswitch-first order
def encrypt_table_big(enc, t):
    """WL.encrypt_table with N + 1-word ciphertexts under the N-bit key."""
    col = enc.encrypt_big_bits(t.column_bits(), WL.STREAM_COLUMN, 0)
    cst = enc.encrypt_big_bits(t.const_bits(), WL.STREAM_CONST, 0)
    pays = [enc.encrypt_big_bits(t.payload_bits(q), WL.STREAM_PAYLOAD, q * t.rows * t.payload_width)
            for q in range(len(t.payloads))]
    return col, cst, pays


def test_ks_first_gates_bit_exact(env):
    ctx, o = env
    rng = np.random.default_rng(23)
    count = 40  # all ten two-input types, four times
    types = (np.arange(count) % 10).astype(np.uint8)
    xb, yb = rng.integers(0, 2, count).astype(np.uint8), rng.integers(0, 2, count).astype(np.uint8)
    x, y = ctx.encrypt_big_bits(xb, 74), ctx.encrypt_big_bits(yb, 75)
    assert np.array_equal(x, o.encrypt_big_bits(xb, 74))
    out = torch.zeros((count, ctx.big_words), dtype=torch.int32, device="cuda")
    ctx.gate_batch_ks_first(dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), out)
    got = host(out).view(np.uint32)
    for g in range(0, count, 7):
        assert np.array_equal(got[g], o.gate3_ks_first(int(types[g]), x[g], y[g])), g
    truth = np.array([O.gate_plain(int(t), int(a), int(b)) for t, a, b in zip(types, xb, yb)], np.uint8)
    assert np.array_equal(ctx.decrypt_big_bits(got), truth)


@pytest.mark.parametrize("name,rows", [("eq4x16", 6), ("range4x16maj", 5), ("lt8x64", 3)])
def test_ks_first_scan_bit_exact(env, name, rows):
    ctx, o = env
    t = WL.table(name, seed=8, rows=rows)
    col, cst, pays = encrypt_table_big(ctx, t)
    ocol, ocst, opays = encrypt_table_big(o, t)
    assert np.array_equal(col, ocol) and np.array_equal(cst, ocst)
    W = ctx.big_words
    match = torch.zeros((t.rows, W), dtype=torch.int32, device="cuda")
    outs = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda") for _ in pays]
    ctx.scan_select_ks_first(dev(col.view(np.int32)), t.rows, t.width, t.pred, dev(cst.view(np.int32)),
                             [dev(p.view(np.int32)) for p in pays], t.payload_width, match, outs)
    om, oouts = o.scan_ks_first(t.pred, t.width, ocol, ocst, opays, t.payload_width)
    assert np.array_equal(host(match).view(np.uint32), om)
    for a, b in zip(outs, oouts):
        assert np.array_equal(host(a).view(np.uint32).reshape(b.shape), b)
    m_want, (p_want,) = t.expected()
    assert np.array_equal(ctx.decrypt_big_bits(om), m_want)
    got_p = ctx.decrypt_big_bits(oouts[0].reshape(-1, W)).reshape(t.rows, t.payload_width)
    assert np.array_equal((got_p.astype(np.uint64) << np.arange(t.payload_width, dtype=np.uint64)).sum(axis=1), p_want)
    # one gate per launch gives the same words
    m2 = torch.zeros_like(match)
    o2 = [torch.zeros_like(x) for x in outs]
    ctx.scan_select_ks_first(dev(col.view(np.int32)), t.rows, t.width, t.pred, dev(cst.view(np.int32)),
                             [dev(p.view(np.int32)) for p in pays], t.payload_width, m2, o2, per_gate=True)
    assert np.array_equal(host(m2), host(match)) and all(np.array_equal(host(a), host(b)) for a, b in zip(o2, outs))


def test_ks_first_scan_eq32x4096_full_size_sampled_rows(env):
    """The equality workload at full size in keyswitch-first order: every row
    decrypted against the SQL answer; the matching and last rows recomputed
    by the oracle word for word (default engine only, for time)."""
    ctx, o = env
    if ctx.engine != F.FSQL_ENGINE_DUAL_PRIME:
        pytest.skip("full-size keyswitch-first scan runs on the default engine")
    t = WL.table("eq32x4096", seed=1)
    col, cst, pays = encrypt_table_big(ctx, t)
    W = ctx.big_words
    match = torch.zeros((t.rows, W), dtype=torch.int32, device="cuda")
    outs = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda")]
    ctx.scan_select_ks_first(dev(col.view(np.int32)), t.rows, t.width, t.pred, dev(cst.view(np.int32)),
                             [dev(pays[0].view(np.int32))], t.payload_width, match, outs)
    gm, go = host(match).view(np.uint32), host(outs[0]).view(np.uint32)
    m_want, (p_want,) = t.expected()
    assert np.array_equal(ctx.decrypt_big_bits(gm), m_want)
    bits = ctx.decrypt_big_bits(go.reshape(-1, W)).reshape(t.rows, t.payload_width)
    assert np.array_equal((bits.astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(axis=1), p_want)
    rows = sorted({int(np.argmax(m_want)), t.rows - 1})
    ocol = np.concatenate([o.encrypt_big_bits(t.column_bits().reshape(t.rows, 32)[r], WL.STREAM_COLUMN, r * 32)
                           for r in rows])
    opay = np.concatenate([o.encrypt_big_bits(t.payload_bits(0).reshape(t.rows, 32)[r], WL.STREAM_PAYLOAD, r * 32)
                           for r in rows])
    ocst = o.encrypt_big_bits(t.const_bits(), WL.STREAM_CONST, 0)
    om, (oout,) = o.scan_ks_first(t.pred, 32, ocol, ocst, [opay], 32)
    assert np.array_equal(gm[rows], om)
    assert np.array_equal(go.reshape(t.rows, 32, W)[rows], oout)


# ---------------------------------------------------------------- SUM aggregation
@pytest.mark.parametrize("rows,width,out_width", [(6, 3, 6), (1, 4, 6), (24, 8, 13), (9, 4, 3)])
def test_aggregate_sum_bit_exact(env, rows, width, out_width):
    ctx, o = env
    rng = np.random.default_rng(rows * 7 + width)
    vals = rng.integers(0, 1 << width, rows)
    bits = np.array([(int(v) >> j) & 1 for v in vals for j in range(width)], np.uint8)
    ct = both_encrypt_bits(ctx, o, bits, 41)
    out = torch.full((out_width, ctx.words), 7, dtype=torch.int32, device="cuda")
    ctx.aggregate_sum(dev(ct.view(np.int32)), rows, width, out_width, out)
    got = host(out).view(np.uint32)
    assert np.array_equal(got, o.aggregate_sum(ct, rows, width, out_width))
    dec = ctx.decrypt_bits(got)
    assert int(sum(int(dec[j]) << j for j in range(out_width))) == int(vals.sum()) % (1 << out_width)


def test_aggregate_sum_empty_and_replay(env):
    ctx, _ = env
    out = torch.full((5, ctx.words), 7, dtype=torch.int32, device="cuda")
    ctx.aggregate_sum(None, 0, 8, 5, out)  # no rows: the sum is a known zero
    got = host(out).view(np.uint32)
    assert np.all(got[:, :-1] == 0) and np.all(got[:, -1] == np.uint32((1 << 32) - (1 << 29)))
    # the same arguments twice: the second call replays the plan and gives the same words
    rng = np.random.default_rng(3)
    vals = rng.integers(0, 16, 10)
    ct = ctx.encrypt_bits(np.array([(int(v) >> j) & 1 for v in vals for j in range(4)], np.uint8), 42, 0)
    dct = dev(ct.view(np.int32))
    res = []
    for _ in range(2):
        o_ = torch.zeros((8, ctx.words), dtype=torch.int32, device="cuda")
        ctx.aggregate_sum(dct, 10, 4, 8, o_)
        res.append(host(o_))
    assert np.array_equal(res[0], res[1])


def test_scan_then_sum_full_size(env):
    """SUM over the masked payload of the full-size equality scan (4096 rows,
    262,080 more bootstraps): the decrypted sum is the SQL answer, and the
    oracle's own evaluation of the same circuit on a 24-row slice of the
    masked column gives the same words as the library's."""
    ctx, o = env
    t = WL.table("eq32x4096", seed=1)
    col, cst, pays = WL.encrypt_table(ctx, t)
    match, outs = run_scan(ctx, t, col, cst, pays)
    masked = dev(outs[0].view(np.int32))
    ow = 44
    out = torch.zeros((ow, ctx.words), dtype=torch.int32, device="cuda")
    ctx.aggregate_sum(masked, t.rows, 32, ow, out)
    dec = ctx.decrypt_bits(host(out).view(np.uint32))
    _, (p_want,) = t.expected()
    assert int(sum(int(dec[j]) << j for j in range(ow))) == int(p_want.astype(object).sum()) % (1 << ow)
    # oracle on a slice: rows 0..23 of the masked column, an 8-bit slice of each value
    sl = outs[0].reshape(t.rows, 32, -1)[:24, :8].copy()
    out2 = torch.zeros((13, ctx.words), dtype=torch.int32, device="cuda")
    ctx.aggregate_sum(dev(sl.view(np.int32)), 24, 8, 13, out2)
    assert np.array_equal(host(out2).view(np.uint32), o.aggregate_sum(sl, 24, 8, 13))


# ---------------------------------------------------------------- MAX / MIN aggregation
@pytest.mark.parametrize("rows,width", [(5, 3), (1, 4), (8, 6), (0, 3)])
def test_aggregate_max_min_bit_exact(env, rows, width):
    ctx, o = env
    rng = np.random.default_rng(rows * 11 + width)
    vals = rng.integers(0, 1 << width, rows)
    m = (rng.integers(0, 2, rows) if rows else np.zeros(0, int)).astype(np.uint8)
    if rows > 1:
        m[0] = 1
    W = ctx.words
    bits = np.array([(int(v) >> j) & 1 for v in vals for j in range(width)], np.uint8)
    ct = both_encrypt_bits(ctx, o, bits, 43) if rows else np.zeros((0, W), np.uint32)
    mct = both_encrypt_bits(ctx, o, m, 44) if rows else np.zeros((0, W), np.uint32)
    dct = dev(ct.view(np.int32)) if rows else None
    dm = dev(mct.view(np.int32)) if rows else None
    for is_min in (False, True):
        out = torch.full((width, W), 7, dtype=torch.int32, device="cuda")
        if is_min:
            ctx.aggregate_min(dct, dm, rows, width, out)
        else:
            ctx.aggregate_max(dct, rows, width, out)
        got = host(out).view(np.uint32)
        want = o.aggregate_extreme(is_min, ct, rows, width, mct if is_min else None)
        assert np.array_equal(got, want), is_min
        dec = ctx.decrypt_bits(got)
        value = int(sum(int(dec[j]) << j for j in range(width)))
        sel = [int(v) for v, mm in zip(vals, m) if mm]
        assert value == ((min(sel) if sel else (1 << width) - 1) if is_min else (int(vals.max()) if rows else 0))


def test_scan_then_max_min_full_size(env):
    """MAX and MIN over the full-size equality scan's payload (4096 rows,
    524,160 and 655,232 bootstraps): decrypted results equal the SQL
    answers.  Default engine only: 1.2 M bootstraps take minutes on the
    64-bit-prime engine, whose gates the small-table tests cover."""
    ctx, _ = env
    if ctx.engine != F.FSQL_ENGINE_DUAL_PRIME:
        pytest.skip("full-size MAX/MIN runs on the default engine")
    t = WL.table("eq32x4096", seed=1)
    col, cst, pays = WL.encrypt_table(ctx, t)
    match, outs = run_scan(ctx, t, col, cst, pays)
    masked, dmatch = dev(outs[0].view(np.int32)), dev(match.view(np.int32))
    m_want, (p_want,) = t.expected()
    raw = t.payloads[0]
    dec = lambda out: int(sum(int(b) << j for j, b in enumerate(ctx.decrypt_bits(host(out).view(np.uint32)))))
    out = torch.zeros((32, ctx.words), dtype=torch.int32, device="cuda")
    ctx.aggregate_max(masked, t.rows, 32, out)
    assert dec(out) == int(p_want.max())
    ctx.aggregate_min(masked, dmatch, t.rows, 32, out)
    assert dec(out) == int(raw[m_want == 1].min())


def test_scan_eq32x4096_full_size_sampled_rows(env):
    """The benchmark workload at full size, in the benchmark's launch
    configuration; the oracle recomputes whole sampled rows (the matching row
    and the last row), every row is decrypted against the SQL answer."""
    ctx, o = env
    t = WL.table("eq32x4096", seed=1)
    col, cst, pays = WL.encrypt_table(ctx, t)
    match, outs = run_scan(ctx, t, col, cst, pays)
    check_plaintext(ctx, t, match, outs)
    m_want, _ = t.expected()
    rows = sorted({int(np.argmax(m_want)), t.rows - 1})
    sub = WL.Table(t.name, len(rows), t.width, t.pred, t.column[rows], [p[rows] for p in t.payloads],
                   t.payload_width, t.consts)
    # oracle encrypts the sampled rows at their own positions in the column stream
    ocol = np.concatenate([o.encrypt_bits(t.column_bits().reshape(t.rows, t.width)[r], WL.STREAM_COLUMN,
                                          r * t.width) for r in rows])
    opay = np.concatenate([o.encrypt_bits(t.payload_bits(0).reshape(t.rows, t.payload_width)[r],
                                          WL.STREAM_PAYLOAD, r * t.payload_width) for r in rows])
    ocst = o.encrypt_bits(t.const_bits(), WL.STREAM_CONST, 0)
    assert np.array_equal(ocol.reshape(len(rows), t.width, -1), col.reshape(t.rows, t.width, -1)[rows])
    om, (oout,) = o.scan(sub.pred, sub.width, ocol, ocst, [opay], sub.payload_width)
    assert np.array_equal(match.reshape(t.rows, -1)[rows], om)
    assert np.array_equal(outs[0].reshape(t.rows, t.payload_width, -1)[rows], oout)


def test_autotune_picks_a_shape_and_keeps_results(env):
    ctx, _ = env
    types, xb, yb = WL.gates(40, seed=9)
    x = ctx.encrypt_bits(xb, WL.STREAM_GATES, 0)
    y = ctx.encrypt_bits(yb, WL.STREAM_GATES, 40)
    a = torch.zeros((40, 631), dtype=torch.int32, device="cuda")
    b = torch.zeros((40, 631), dtype=torch.int32, device="cuda")
    ctx.gate_batch(dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), a)
    best, ms = ctx.autotune(probe_gates=1184)
    assert best in ms and ctx.br_shape == best and all(v > 0 for v in ms.values())
    assert set(ms) == ({0, 1, 3} if ctx.engine == F.FSQL_ENGINE_GOLDILOCKS else set(range(F.BR_SHAPES)))
    ctx.gate_batch(dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), b)
    assert np.array_equal(host(a), host(b))
