"""GPU parity at the sizes and launch shapes the benchmark times.

The small-table tests in test_gpu_parity.py mostly run the kernels for
small batches (the latency-mode blind rotation, the split keyswitch).  Here
the throughput kernels (several gates per CTA over a persistent grid, the
single-pass keyswitch) are compared word for word with the CPU oracle:
gate batches of 296, 4736 and 65,536 random microbenchmark gates (512
seeded samples each, every gate decrypted), the single-pass keyswitch on
edge-case inputs, 16 whole rows of the 4096-row equality scan, and a served
mix whose merged rounds are large enough for the throughput kernels.
Default (two-prime) engine: it is the engine the benchmark runs."""
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
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    O.set_threads(os.cpu_count() or 1)
    o = O.Oracle(SEED)
    ctx = F.Context(SEED, device=0)
    yield ctx, o
    ctx.close()
    o.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_rows(o, t, rows):
    """The oracle's scan of the given rows of table t, each row encrypted at
    its own position in the column and payload streams (the positions the
    library used for the whole table)."""
    w, pw = t.width, t.payload_width
    cb = t.column_bits().reshape(t.rows, w)
    ocol = np.concatenate([o.encrypt_bits(cb[r], WL.STREAM_COLUMN, r * w) for r in rows])
    opays = []
    for q in range(len(t.payloads)):
        pb = t.payload_bits(q).reshape(t.rows, pw)
        opays.append(np.concatenate([o.encrypt_bits(pb[r], WL.STREAM_PAYLOAD, q * t.rows * pw + r * pw)
                                     for r in rows]))
    ocst = o.encrypt_bits(t.const_bits(), WL.STREAM_CONST, 0)
    return o.scan(t.pred, w, ocol, ocst, opays, pw)


@pytest.mark.parametrize("B", [201, 256, 296, 4736, 65536])
def test_gate_batch_throughput_kernels_sampled(env, B):
    """B between one and two gates per SM (201: a ragged last CTA; 256: the
    sweep's point) and exactly two (one wave of two-gate CTAs), 32 per SM and
    65,536 (the sweep's large point): 512 seeded samples recomputed by the
    oracle, including the first and last gates (ragged tails of the
    persistent grid), every gate decrypted."""
    ctx, o = env
    types, xb, yb = WL.gates(B, seed=B)
    x = ctx.encrypt_bits(xb, WL.STREAM_GATES, 0)
    y = ctx.encrypt_bits(yb, WL.STREAM_GATES, B)
    out = torch.zeros((B, ctx.words), dtype=torch.int32, device="cuda")
    ctx.gate_batch(dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), out)
    got = host(out).view(np.uint32)
    truth = np.array([[1, 1, 1, 0], [0, 0, 0, 1], [0, 1, 1, 1], [0, 1, 1, 0], [1, 0, 0, 1]], np.uint8)[types, 2 * xb + yb]
    assert np.array_equal(ctx.decrypt_bits(got), truth)
    rng = np.random.default_rng(B + 1)
    sample = np.unique(np.concatenate([[0, 1, 2, B - 3, B - 2, B - 1], rng.choice(B, min(B, 506), replace=False)]))
    ox = o.encrypt_bits(xb, WL.STREAM_GATES, 0)
    oy = o.encrypt_bits(yb, WL.STREAM_GATES, B)
    assert np.array_equal(ox, x) and np.array_equal(oy, y)
    want = o.gate_batch(types[sample].astype(np.int32), ox[sample], oy[sample])
    assert np.array_equal(got[sample], want)


def test_keyswitch_single_pass_edge_cases(env):
    """200 samples (more than the split path's 128, so the single-pass
    kernel runs; 12 full groups of 16 and a ragged one of 8): all-zero,
    all-ones, every mask word on a rounding tie, just below and above it,
    the wrap to zero at the top, and random words; every output compared."""
    ctx, o = env
    count = 200
    rng = np.random.default_rng(3)
    big = rng.integers(0, 1 << 32, (count, 1025), dtype=np.uint64).astype(np.uint32)
    big[0, :1024] = 0
    big[1, :1024] = 0xFFFFFFFF
    big[2, :1024] = 1 << 15
    big[3, :1024] = (rng.integers(0, 1 << 16, 1024, dtype=np.uint64) << 16 | 0x8000).astype(np.uint32)
    big[4, :1024] = (rng.integers(0, 1 << 16, 1024, dtype=np.uint64) << 16 | 0x7FFF).astype(np.uint32)
    big[5, :1024] = 0xFFFF8000
    big[199, :1024] = (rng.integers(0, 1 << 16, 1024, dtype=np.uint64) << 16 | 0x8001).astype(np.uint32)
    out = torch.zeros((count, ctx.words), dtype=torch.int32, device="cuda")
    ctx.keyswitch(dev(big.view(np.int32)), out, count)
    got = host(out).view(np.uint32)
    for g in range(count):
        assert np.array_equal(got[g], o.keyswitch(big[g])), g


def test_scan_eq32x4096_sixteen_oracle_rows(env):
    """The benchmark's equality scan at full size (4096 rows, 389,120
    bootstraps, the launch configuration bench.py times): 16 whole rows
    recomputed by the oracle (the matching row, the first and last rows, 13
    seeded others), every row decrypted against the SQL answer."""
    ctx, o = env
    t = WL.table("eq32x4096", seed=1)
    col, cst, pays = WL.encrypt_table(ctx, t)
    W = ctx.words
    match = torch.zeros((t.rows, W), dtype=torch.int32, device="cuda")
    outs = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda")]
    ctx.scan_select(dev(col.view(np.int32)), t.rows, t.width, t.pred, dev(cst.view(np.int32)),
                    [dev(pays[0].view(np.int32))], t.payload_width, match, outs)
    gm, go = host(match).view(np.uint32), host(outs[0]).view(np.uint32)
    m_want, (p_want,) = t.expected()
    assert np.array_equal(ctx.decrypt_bits(gm), m_want)
    assert np.array_equal(ctx.decrypt_uint(go, 32), p_want)
    hit = int(np.argmax(m_want))
    others = np.random.default_rng(16).choice(np.setdiff1d(np.arange(1, t.rows - 1), [hit]), 13, replace=False)
    rows = sorted({hit, 0, t.rows - 1, *map(int, others)})
    assert len(rows) == 16
    om, (oout,) = oracle_rows(o, t, rows)
    assert np.array_equal(gm[rows], om)
    assert np.array_equal(go.reshape(t.rows, 32, W)[rows], oout.reshape(len(rows), 32, W))


def test_served_mix_large_rounds_match_oracle(env):
    """A served mix whose merged rounds reach thousands of gates (so they run
    on the multi-gate-per-CTA kernel and the single-pass keyswitch): two
    sampled rows of each query recomputed by the oracle word for word, match
    bits and masked payloads of every row decrypted against the SQL answer."""
    ctx, o = env
    tables = [WL.table("eq32x4096", seed=21, rows=96), WL.table("range16x65536", seed=22, rows=40),
              WL.table("eq4x16", seed=23), WL.table("range16x65536maj", seed=24, rows=64)]
    W = ctx.words
    ios = []
    for t in tables:
        col, cst, pays = WL.encrypt_table(ctx, t)
        ios.append({"column": dev(col.view(np.int32)), "const": dev(cst.view(np.int32)),
                    "payloads": [dev(p.view(np.int32)) for p in pays],
                    "match": torch.zeros((t.rows, W), dtype=torch.int32, device="cuda"),
                    "outs": [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda")
                             for _ in pays]})
    torch.cuda.synchronize()  # inputs and zeroed outputs complete before the server stream reads them
    srv = F.Server(ctx, scratch_budget_bytes=256 << 20, max_batch_gates=8192)
    ids = [srv.submit(io["column"], t.rows, t.width, t.pred, io["const"], io["payloads"], t.payload_width,
                      io["match"], io["outs"]) for t, io in zip(tables, ios)]
    for qid in ids:
        srv.wait(qid, 600000)
        assert srv.status(qid)[0] == F.Q_DONE
    st = srv.stats()
    srv.close()
    assert st["gates"] == sum(t.rows * t.gates_per_row for t in tables)
    assert st["gates"] / st["rounds"] > 2 * 148  # average round above two gates per SM
    for k, (t, io) in enumerate(zip(tables, ios)):
        gm = host(io["match"]).view(np.uint32)
        gouts = [host(x).view(np.uint32) for x in io["outs"]]
        m_want, p_want = t.expected()
        assert np.array_equal(ctx.decrypt_bits(gm), m_want)
        for q, g in enumerate(gouts):
            assert np.array_equal(ctx.decrypt_uint(g, t.payload_width), p_want[q])
        rows = sorted({int(np.argmax(m_want)), t.rows - 1 - k})
        om, oouts = oracle_rows(o, t, rows)
        assert np.array_equal(gm[rows], om), t.name
        for g, ob in zip(gouts, oouts):
            assert np.array_equal(g.reshape(t.rows, t.payload_width, W)[rows],
                                  ob.reshape(len(rows), t.payload_width, W)), t.name


def test_ks_first_graph_follows_scratch_growth(env):
    """Keyswitch-first scans capture their launches in a graph that reads the
    context's keyswitch-first scratch.  A larger plan in between reallocates
    that scratch; replaying the small plan afterwards must use the new
    buffers (checked word for word against the oracle)."""
    ctx, o = env
    W = ctx.big_words

    def run(t, col, cst, pays, match, outs):
        ctx.scan_select_ks_first(col, t.rows, t.width, t.pred, cst, pays, t.payload_width, match, outs)
        torch.cuda.synchronize()

    def make(t):
        col = ctx.encrypt_big_bits(t.column_bits(), WL.STREAM_COLUMN, 0)
        cst = ctx.encrypt_big_bits(t.const_bits(), WL.STREAM_CONST, 0)
        pays = [ctx.encrypt_big_bits(t.payload_bits(q), WL.STREAM_PAYLOAD, q * t.rows * t.payload_width)
                for q in range(len(t.payloads))]
        io = (dev(col.view(np.int32)), dev(cst.view(np.int32)), [dev(p.view(np.int32)) for p in pays],
              torch.zeros((t.rows, W), dtype=torch.int32, device="cuda"),
              [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda") for _ in pays])
        return (col, cst, pays), io

    small = WL.table("eq4x16", seed=31, rows=5)
    large = WL.table("eq32x4096", seed=32, rows=40)
    (scol, scst, spays), sio = make(small)
    _, lio = make(large)
    run(small, *sio)  # captures the small plan's graph
    first = host(sio[3]).copy()
    run(large, *lio)  # the large plan grows the keyswitch-first scratch (and replaces the plan)
    sio[3].zero_()
    for x in sio[4]:
        x.zero_()
    run(small, *sio)  # a new plan for the small scan, captured against the new scratch
    run(small, *sio)  # and its replay
    om, oouts = o.scan_ks_first(small.pred, small.width, scol, scst, spays, small.payload_width)
    assert np.array_equal(host(sio[3]).view(np.uint32), om)
    assert np.array_equal(first.view(np.uint32), om)
    assert np.array_equal(host(sio[4][0]).view(np.uint32).reshape(oouts[0].shape), oouts[0])


def test_every_launch_shape_gives_the_same_words(env):
    """Every blind-rotation launch shape of the engine (packed and
    prime-split kernels, 2 or 3 gates per CTA, 2 or 3 gadget rows per step,
    2 or 3 staging slots) on a 1184-gate batch (8 per SM, a ragged last wave
    for 3 gates per CTA): words equal to each other and, on 40 samples, to
    the oracle's."""
    ctx, o = env
    B = 1184
    types, xb, yb = WL.gates(B, seed=77)
    x = ctx.encrypt_bits(xb, WL.STREAM_GATES, 0)
    y = ctx.encrypt_bits(yb, WL.STREAM_GATES, B)
    dt, da, db = dev(types), dev(x.view(np.int32)), dev(y.view(np.int32))
    saved = ctx.br_shape
    words = {}
    try:
        for shape in range(F.BR_SHAPES):
            ctx.br_shape = shape
            out = torch.full((B, ctx.words), -1, dtype=torch.int32, device="cuda")
            ctx.gate_batch(dt, da, db, out)
            words[shape] = host(out).view(np.uint32)
    finally:
        ctx.br_shape = saved
    for shape in range(1, F.BR_SHAPES):
        assert np.array_equal(words[shape], words[0]), F.br_shape_info(shape)
    sample = np.unique(np.concatenate([[0, B - 1], np.random.default_rng(9).choice(B, 38, replace=False)]))
    want = o.gate_batch(types[sample].astype(np.int32), x[sample], y[sample])
    assert np.array_equal(words[0][sample], want)


def _scan(ctx, t, col, cst, pays):
    W = ctx.words
    match = torch.zeros((t.rows, W), dtype=torch.int32, device="cuda")
    outs = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda") for _ in pays]
    ctx.scan_select(col, t.rows, t.width, t.pred, cst, pays, t.payload_width, match, outs)
    return match, outs


def test_device_walker_equals_level_launches_and_oracle(env):
    """The device level walker (one cooperative launch for the whole scan)
    gives the words of the per-level launches, and two rows equal the
    oracle's; a replay of the captured walker graph gives them again."""
    ctx, o = env
    t = WL.table("eq32x4096", seed=41, rows=300)  # every level at least two gates per SM
    col, cst, pays = WL.encrypt_table(ctx, t)
    dcol, dcst, dp = dev(col.view(np.int32)), dev(cst.view(np.int32)), [dev(p.view(np.int32)) for p in pays]
    m_lv, o_lv = _scan(ctx, t, dcol, dcst, dp)
    ref_m, ref_o = host(m_lv).copy(), host(o_lv[0]).copy()
    try:
        ctx.set_walk(True)
        for _ in range(2):
            m_w, o_w = _scan(ctx, t, dcol, dcst, dp)
            ctx.walk_status()
            assert np.array_equal(host(m_w), ref_m) and np.array_equal(host(o_w[0]), ref_o)
    finally:
        ctx.set_walk(False)
    om, (oout,) = oracle_rows(o, t, [0, t.rows - 1])
    assert np.array_equal(ref_m.view(np.uint32)[[0, t.rows - 1]], om)
    assert np.array_equal(ref_o.view(np.uint32).reshape(t.rows, 32, -1)[[0, t.rows - 1]],
                          oout.reshape(2, 32, -1))


def test_device_walker_barrier_timeout_is_reported(env):
    """A CTA that never arrives at the walker's grid barriers (test hook):
    the other CTAs' waits run out after 200 ms, the kernel returns, the host
    reads FSQL_ERR_TIMEOUT, and the context keeps working (the next walked
    scan equals the per-level launches)."""
    ctx, _ = env
    t = WL.table("eq32x4096", seed=42, rows=300)
    col, cst, pays = WL.encrypt_table(ctx, t)
    dcol, dcst, dp = dev(col.view(np.int32)), dev(cst.view(np.int32)), [dev(p.view(np.int32)) for p in pays]
    m_lv, o_lv = _scan(ctx, t, dcol, dcst, dp)
    ref_m = host(m_lv).copy()
    try:
        ctx.set_walk(True, timeout_ms=200.0)
        ctx.debug_walk_skip_block(5)
        _scan(ctx, t, dcol, dcst, dp)
        with pytest.raises(F.FsqlError) as e:
            ctx.walk_status()
        assert e.value.code == F.FSQL_ERR_TIMEOUT
        ctx.debug_walk_skip_block(-1)
        m_w, _ = _scan(ctx, t, dcol, dcst, dp)
        ctx.walk_status()
        assert np.array_equal(host(m_w), ref_m)
    finally:
        ctx.debug_walk_skip_block(-1)
        ctx.set_walk(False)


def test_cluster_latency_mode_equals_other_modes_and_oracle(env):
    """Small batches on the cluster kernel (one gate per cluster of six CTAs
    exchanging through distributed shared memory): the words of the three-group
    latency kernel and of one gate per CTA, and the oracle's on samples, for
    one gate, one cluster wave and more gates than clusters."""
    ctx, o = env
    rng = np.random.default_rng(29)
    try:
        for count in (1, 7, 48):
            types = rng.integers(0, 10, count).astype(np.uint8)
            xb, yb = rng.integers(0, 2, count).astype(np.uint8), rng.integers(0, 2, count).astype(np.uint8)
            a = ctx.encrypt_bits(xb, 62, 0)
            b = ctx.encrypt_bits(yb, 63, 0)
            res = {}
            for mode in (2, 1, 0):
                ctx.set_latency_mode(mode)
                out = torch.full((count, ctx.words), -1, dtype=torch.int32, device="cuda")
                ctx.gate_batch(dev(types), dev(a.view(np.int32)), dev(b.view(np.int32)), out)
                res[mode] = host(out).view(np.uint32)
            assert np.array_equal(res[2], res[1]) and np.array_equal(res[2], res[0]), count
            k = min(count, 3)
            assert np.array_equal(res[2][:k], o.gate_batch(types[:k].astype(np.int32), a[:k], b[:k]))
            truth = np.array([O.gate_plain(int(t), int(x), int(y)) for t, x, y in zip(types, xb, yb)], np.uint8)
            assert np.array_equal(ctx.decrypt_bits(res[2]), truth)
    finally:
        ctx.set_latency_mode(2)
