"""Serving loop: queries of different shapes share launches (continuous
batching under a memory budget) and each one's output words are exactly the
words of the same scan run alone."""
import numpy as np
import pytest

from paper_2510_15413_b300 import fhesql as F
from paper_2510_15413_b300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = F.Context(77, device=0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).cuda()


def prepare(ctx, t):
    col, cst, pays = WL.encrypt_table(ctx, t)
    W = ctx.words
    io = {"column": dev(col), "const": dev(cst), "payloads": [dev(p) for p in pays],
          "match": torch.zeros((t.rows, W), dtype=torch.int32, device="cuda"),
          "outs": [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda") for _ in pays]}
    return io


def alone(ctx, t, io):
    W = ctx.words
    m = torch.zeros((t.rows, W), dtype=torch.int32, device="cuda")
    o = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda") for _ in io["payloads"]]
    ctx.scan_select(io["column"], t.rows, t.width, t.pred, io["const"], io["payloads"], t.payload_width, m, o)
    torch.cuda.synchronize()
    return m.cpu().numpy(), [x.cpu().numpy() for x in o]


def test_mixed_queries_equal_their_solo_runs(ctx):
    tables = [WL.table("eq4x16", seed=1), WL.table("lt8x64", seed=2, rows=6), WL.table("range4x16", seed=3, rows=5),
              WL.table("eq32x4096", seed=4, rows=9), WL.table("range16x65536", seed=5, rows=3)]
    ios = [prepare(ctx, t) for t in tables]
    # budget for about two queries at a time and small rounds: forces queueing, chunked levels and merging
    torch.cuda.synchronize()  # inputs and zeroed outputs complete before the server stream reads them
    srv = F.Server(ctx, scratch_budget_bytes=2 << 20, max_batch_gates=96)
    ids = [srv.submit(io["column"], t.rows, t.width, t.pred, io["const"], io["payloads"], t.payload_width,
                      io["match"], io["outs"]) for t, io in zip(tables, ios)]
    for qid in ids:
        srv.wait(qid, 300000)
        assert srv.status(qid)[0] == F.Q_DONE
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(tables) and st["p50_ms"] <= st["p99_ms"]
    assert st["gates"] == sum(t.rows * t.gates_per_row for t in tables)
    assert st["rounds"] < sum(F.plan_info(t.pred, t.width, len(t.payloads), t.payload_width)[0] for t in tables) * 8
    for t, io in zip(tables, ios):
        m_alone, o_alone = alone(ctx, t, io)
        assert np.array_equal(io["match"].cpu().numpy(), m_alone)
        for a, b in zip(io["outs"], o_alone):
            assert np.array_equal(a.cpu().numpy(), b)
        m_want, p_want = t.expected()
        assert np.array_equal(ctx.decrypt_bits(m_alone.view(np.uint32)), m_want)
        for q, b in enumerate(o_alone):
            assert np.array_equal(ctx.decrypt_uint(b.view(np.uint32), t.payload_width), p_want[q])


def test_admission_rejects_query_larger_than_budget(ctx):
    t = WL.table("eq32x4096", seed=6, rows=64)
    io = prepare(ctx, t)
    torch.cuda.synchronize()  # inputs and zeroed outputs complete before the server stream reads them
    srv = F.Server(ctx, scratch_budget_bytes=1 << 20)
    with pytest.raises(F.FsqlError) as e:
        srv.submit(io["column"], t.rows, t.width, t.pred, io["const"], io["payloads"], t.payload_width,
                   io["match"], io["outs"])
    assert e.value.code == F.FSQL_ERR_ADMISSION
    srv.close()


def test_cancel_waiting_query(ctx):
    t = WL.table("eq32x4096", seed=7, rows=32)
    io1, io2 = prepare(ctx, t), prepare(ctx, t)
    torch.cuda.synchronize()  # inputs and zeroed outputs complete before the server stream reads them
    srv = F.Server(ctx, scratch_budget_bytes=6 << 20)  # one such query at a time
    a = srv.submit(io1["column"], t.rows, t.width, t.pred, io1["const"], io1["payloads"], t.payload_width,
                   io1["match"], io1["outs"])
    b = srv.submit(io2["column"], t.rows, t.width, t.pred, io2["const"], io2["payloads"], t.payload_width,
                   io2["match"], io2["outs"])
    srv.cancel(b)
    srv.wait(a, 300000)
    srv.wait(b, 300000)
    assert srv.status(a)[0] == F.Q_DONE and srv.status(b)[0] == F.Q_CANCELLED
    srv.close()


def test_served_plain_constant_queries_equal_solo(ctx):
    """Plaintext-constant queries (including one with no gate at all and one
    whose match is a negated column bit) served next to an encrypted one."""
    specs = [("eq4x16plain", 1, None), ("lt8x64plain", 2, (0,)), ("lt8x64plain", 3, (128,)),
             ("range4x16plain", 4, None), ("eq4x16", 5, None)]
    tables = []
    for name, seed, consts in specs:
        t = WL.table(name, seed=seed, rows=6)
        if consts is not None:
            t.consts = consts
        tables.append(t)
    ios = [prepare(ctx, t) for t in tables]
    torch.cuda.synchronize()  # inputs and zeroed outputs complete before the server stream reads them
    srv = F.Server(ctx, scratch_budget_bytes=2 << 20, max_batch_gates=64)
    ids = [srv.submit(io["column"], t.rows, t.width, t.pred, None if t.plain else io["const"], io["payloads"],
                      t.payload_width, io["match"], io["outs"], plain_consts=t.consts if t.plain else None)
           for t, io in zip(tables, ios)]
    for qid in ids:
        srv.wait(qid, 300000)
        assert srv.status(qid)[0] == F.Q_DONE
    srv.close()
    W = ctx.words
    for t, io in zip(tables, ios):
        m = torch.zeros((t.rows, W), dtype=torch.int32, device="cuda")
        o = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device="cuda") for _ in io["payloads"]]
        if t.plain:
            ctx.scan_select_plain(io["column"], t.rows, t.width, t.pred, t.consts, io["payloads"], t.payload_width,
                                  m, o)
        else:
            ctx.scan_select(io["column"], t.rows, t.width, t.pred, io["const"], io["payloads"], t.payload_width, m, o)
        torch.cuda.synchronize()
        assert np.array_equal(io["match"].cpu().numpy(), m.cpu().numpy())
        for a, b in zip(io["outs"], o):
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
        m_want, p_want = t.expected()
        assert np.array_equal(ctx.decrypt_bits(m.cpu().numpy().view(np.uint32)), m_want)
        for q, b in enumerate(o):
            assert np.array_equal(ctx.decrypt_uint(b.cpu().numpy().view(np.uint32), t.payload_width), p_want[q])
