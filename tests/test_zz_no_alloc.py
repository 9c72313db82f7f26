"""The no-allocation gate entry point, checked against the ordinary one.

fsql_gate_batch_noalloc serves host programs that cannot let the library
call cudaMalloc (the device memory belongs to their own allocator, or a
mid-query allocation and its device-wide synchronisation are not
acceptable).  It must give the same words as fsql_gate_batch, through the
C interface, on consecutive calls that reuse its fixed scratch array.
This file sorts last so that a run stopping at the first failure has
already run every other test."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_15413_b300 import fhesql as F
from paper_2510_15413_b300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = F.Context(4242, device=0)
    yield c
    c.close()


def _batch(ctx, count, seed, with_host=False):
    types, xb, yb = WL.gates(count, seed=seed)
    x = ctx.encrypt_bits(xb, WL.STREAM_GATES, 0)
    y = ctx.encrypt_bits(yb, WL.STREAM_GATES, count)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    truth = np.array([[1, 1, 1, 0], [0, 0, 0, 1], [0, 1, 1, 1], [0, 1, 1, 0], [1, 0, 0, 1]], np.uint8)[types, 2 * xb + yb]
    if with_host:
        return dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), truth, (types, x, y)
    return dev(types), dev(x.view(np.int32)), dev(y.view(np.int32)), truth


def test_noalloc_matches_gate_batch_on_two_calls(ctx):
    for count, seed in [(37, 11), (9, 12)]:  # second call is smaller: stale scratch from the first must not leak
        types, a, b, truth = _batch(ctx, count, seed)
        want = torch.zeros((count, ctx.words), dtype=torch.int32, device="cuda")
        got = torch.full((count, ctx.words), -1, dtype=torch.int32, device="cuda")
        ctx.gate_batch(types, a, b, want)
        ctx.gate_batch_noalloc(types, a, b, got)
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.array_equal(g, w)  # bit-exact, the tolerance of every parity test here
        assert np.array_equal(ctx.decrypt_bits(g.view(np.uint32)), truth)


def test_noalloc_full_scratch_on_throughput_kernels(ctx):
    """1024 gates, the most one call takes: the batch is large enough for
    the several-gates-per-CTA blind rotation and the single-pass keyswitch,
    over the whole fixed array.  Words equal fsql_gate_batch's, a seeded
    sample equals the CPU oracle's, and a warm call changes the device's free
    memory by nothing."""
    count = 1024
    types, a, b, truth, (ht, hx, hy) = _batch(ctx, count, 14, with_host=True)
    want = torch.zeros((count, ctx.words), dtype=torch.int32, device="cuda")
    got = torch.full((count, ctx.words), -1, dtype=torch.int32, device="cuda")
    ctx.gate_batch(types, a, b, want)
    ctx.gate_batch_noalloc(types, a, b, got)  # warm: the scratch address lookup is done by now
    got2 = torch.full((count, ctx.words), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        ctx.gate_batch_noalloc(types, a, b, got2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    w, g, g2 = want.cpu().numpy(), got.cpu().numpy(), got2.cpu().numpy()
    assert np.array_equal(g, w) and np.array_equal(g2, w)
    assert np.array_equal(ctx.decrypt_bits(g.view(np.uint32)), truth)
    O.set_threads(os.cpu_count() or 1)
    o = O.Oracle(4242)
    try:
        assert np.array_equal(o.encrypt_bits(WL.gates(count, seed=14)[1], WL.STREAM_GATES, 0), hx)
        sample = np.unique(np.concatenate([[0, count - 1], np.random.default_rng(5).choice(count, 62, replace=False)]))
        oracle_words = o.gate_batch(ht[sample].astype(np.int32), hx[sample], hy[sample])
    finally:
        o.close()
    assert np.array_equal(g.view(np.uint32)[sample], oracle_words)


def test_noalloc_rejects_more_than_its_scratch_holds(ctx):
    types, a, b, _ = _batch(ctx, 1, 13)
    big = torch.zeros(1025, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FsqlError) as e:
        ctx.gate_batch_noalloc(big, a, b, a)
    assert e.value.code == F.FSQL_ERR_ARG and "1024" in str(e.value)
