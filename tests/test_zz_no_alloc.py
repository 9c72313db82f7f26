"""The no-allocation gate entry point, checked against the ordinary one.

fsql_gate_batch_noalloc serves host programs that cannot let the library
call cudaMalloc (the device memory belongs to their own allocator, or a
mid-query allocation and its device-wide synchronisation are not
acceptable).  It must give the same words as fsql_gate_batch, through the
C interface, on consecutive calls that reuse its fixed scratch array.
This file sorts last so that a run stopping at the first failure has
already run every other test."""
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
    c = F.Context(4242, device=0)
    yield c
    c.close()


def _batch(ctx, count, seed):
    types, xb, yb = WL.gates(count, seed=seed)
    x = ctx.encrypt_bits(xb, WL.STREAM_GATES, 0)
    y = ctx.encrypt_bits(yb, WL.STREAM_GATES, count)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    truth = np.array([[1, 1, 1, 0], [0, 0, 0, 1], [0, 1, 1, 1], [0, 1, 1, 0], [1, 0, 0, 1]], np.uint8)[types, 2 * xb + yb]
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


def test_noalloc_rejects_more_than_its_scratch_holds(ctx):
    types, a, b, _ = _batch(ctx, 1, 13)
    big = torch.zeros(1025, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FsqlError) as e:
        ctx.gate_batch_noalloc(big, a, b, a)
    assert e.value.code == F.FSQL_ERR_ARG and "1024" in str(e.value)
