"""Host-side checks of the C-ABI library (no GPU needed): every declared symbol
is exported, and its client-side half (key generation, encryption, decryption,
circuit scheduler) agrees with the independent CPU oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_15413_b300 import build as B
from paper_2510_15413_b300 import fhesql as F
from paper_2510_15413_b300 import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_symbols():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            names += re.findall(r"FSQL_API\s+[\w\s\*]*?\b(fsql_\w+)\s*\(", text)
    return names


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 20
    lib = ctypes.CDLL(F.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert set(F.API) <= set(names)


@pytest.mark.parametrize("which", ["default", "toy"])
def test_keys_equal_oracle_keys(which):
    seed = 11 if which == "default" else 7
    params = F.params_default() if which == "default" else F.params_toy()
    ctx = F.Context(seed, params, device=-1)
    o = O.Oracle(seed, O.default_params() if which == "default" else O.toy_params())
    s, S, bk, ksk = ctx.export_keys()
    assert np.array_equal(s, o.lwe_key())
    assert np.array_equal(S, o.glwe_key())
    assert np.array_equal(bk, o.bk())
    assert np.array_equal(ksk, o.ksk())


def test_encryption_equals_oracle_encryption():
    ctx = F.Context(11, device=-1)
    o = O.Oracle(11)
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2, 300).astype(np.uint8)
    full = ctx.encrypt_bits(bits, 5, 0)
    assert np.array_equal(full, o.encrypt_bits(bits, 5, 0))
    # chunked encryption with first_index reproduces the single call
    assert np.array_equal(ctx.encrypt_bits(bits[100:], 5, 100), full[100:])
    mu = rng.integers(0, 1 << 32, 50, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(ctx.encrypt(mu, 9, 4), o.encrypt(mu, 9, 4))
    vals = rng.integers(0, 1 << 32, 20, dtype=np.uint64)
    ct = ctx.encrypt_uint(vals, 32, 5, 0)
    assert ct.shape == (20, 32, 631)
    assert np.array_equal(ctx.decrypt_uint(ct, 32), vals)
    assert np.array_equal(ctx.decrypt_bits(full), bits)
    assert np.array_equal(ctx.phase(full[:10]), o.phase(full[:10]))


def _oracle_levels(pred, w, npay, pw):
    t, a, b, c, m, ninp = O.netlist3(pred, w, npay, pw)
    depth = [0] * ninp
    for k in range(t.size):
        depth.append(1 + max(depth[a[k]], depth[b[k]], depth[c[k]] if c[k] >= 0 else 0))
    d = np.array(depth[ninp:])
    return int(t.size), [int((d == L).sum()) for L in range(1, d.max() + 1)]


@pytest.mark.parametrize("shape", [(WL.PRED_EQ, 4, 1, 4), (WL.PRED_EQ, 32, 1, 32), (WL.PRED_LT, 8, 1, 8),
                                   (WL.PRED_RANGE, 16, 2, 16), (WL.PRED_EQ, 1, 0, 0), (WL.PRED_RANGE, 3, 3, 5),
                                   (WL.PRED_LT_MAJ, 8, 1, 8), (WL.PRED_RANGE_MAJ, 16, 2, 16),
                                   (WL.PRED_RANGE_MAJ, 1, 1, 1)])
def test_scheduler_levels_equal_oracle_netlist_depths(shape):
    assert F.plan_info(*shape) == _oracle_levels(*shape)


def test_scheduler_known_level_widths():
    # 16-row 4-bit equality scan: 64 XNOR, 32 + 16 AND, 64 mask gates
    g, widths = F.plan_info(WL.PRED_EQ, 4, 1, 4)
    assert g * 16 == 176 and [16 * x for x in widths] == [64, 32, 16, 64]
    g, widths = F.plan_info(WL.PRED_EQ, 32, 1, 32)
    assert g * 4096 == 389120 and [4096 * x for x in widths] == [131072, 65536, 32768, 16384, 8192, 4096, 131072]
    g, widths = F.plan_info(WL.PRED_RANGE, 16, 2, 16)
    assert g * 65536 == 10158080 and widths[0] * 65536 == 65536 * 62
    g, widths = F.plan_info(WL.PRED_RANGE_MAJ, 16, 2, 16)
    assert g == 65 and WL.table("range16x65536maj").gates_per_row == 65


def test_argument_errors_are_codes_not_crashes():
    p = F.params_default()
    p.N = 1000  # not a power of two
    with pytest.raises(F.FsqlError) as e:
        F.Context(1, p, device=-1)
    assert e.value.code == F.FSQL_ERR_ARG
    # the kernels implement N = 1024 only: a device context with toy params is refused before any CUDA call
    with pytest.raises(F.FsqlError) as e:
        F.Context(1, F.params_toy(), device=0)
    assert e.value.code == F.FSQL_ERR_UNSUPPORTED
    ctx = F.Context(1, F.params_toy(), device=-1)
    with pytest.raises(F.FsqlError):  # host-only context has no device keys
        ctx.gate_batch(np.zeros(1, np.uint8), 1, 2, 3)
    with pytest.raises(F.FsqlError):
        F.plan_info(7, 4, 1, 4)
    with pytest.raises(F.FsqlError):
        F.plan_info(WL.PRED_EQ, 0, 1, 4)


def test_workload_tables_plaintext_semantics():
    t = WL.table("eq32x4096")
    m, (p,) = t.expected()
    assert t.rows == 4096 and m.sum() >= 1 and t.gates_per_row == 95
    assert np.all(p[m == 0] == 0) and np.all(p[m == 1] == t.payloads[0][m == 1])
    r = WL.table("range16x65536")
    m, _ = r.expected()
    assert abs(m.mean() - 0.1) < 0.01 and r.gates_per_row == 155
    assert WL.table("eq4x16").gates_per_row * 16 == 176
    types, x, y = WL.gates(1000)
    assert set(np.unique(types)) == {0, 1, 2, 3, 4}


def _oracle_plain_plan(pred, w, npay, pw, consts):
    t, a, b, m, ol, ninp = O.netlist_plain(pred, w, npay, pw, consts)
    depth = [0] * ninp
    for k in range(t.size):
        depth.append(1 + max(depth[a[k]], depth[b[k]]))
    d = np.array(depth[ninp:], dtype=int)
    widths = [int((d == L).sum()) for L in range(1, (d.max() if d.size else 0) + 1)]
    # outputs that are not a gate's own plain output
    lits = [m] + list(ol)
    n_lit = sum(1 for x in lits if not (x >= 0 and (x >> 1) >= ninp and not x & 1))
    return int(t.size), widths, n_lit


@pytest.mark.parametrize("pred", [WL.PRED_EQ, WL.PRED_LT, WL.PRED_RANGE, WL.PRED_LT_MAJ])
@pytest.mark.parametrize("w", [1, 3, 4, 16])
def test_plain_scheduler_equals_oracle_netlist(pred, w):
    """The library's plaintext-constant circuits (gate count, level widths,
    outputs without a gate) equal the oracle's for many constants."""
    rng = np.random.default_rng(w * 10 + pred)
    top = 1 << w
    ks = sorted({0, 1, top - 1, top >> 1, *[int(v) for v in rng.integers(0, top, 6)]})
    for k in ks:
        for k2 in (ks if pred == WL.PRED_RANGE else [0]):
            consts = (k, k2) if pred == WL.PRED_RANGE else (k,)
            assert F.plan_info_plain(pred, w, 2, 3, consts) == _oracle_plain_plan(pred, w, 2, 3, consts), consts


def test_plain_scheduler_counts_and_errors():
    g, widths, lits = F.plan_info_plain(WL.PRED_EQ, 32, 1, 32, (123456789,))
    assert g == 31 + 32 and widths[-1] == 32 and lits == 0
    g, widths, lits = F.plan_info_plain(WL.PRED_LT, 8, 2, 8, (0,))
    assert g == 0 and widths == [] and lits == 1 + 16
    with pytest.raises(F.FsqlError):
        F.plan_info_plain(WL.PRED_LT, 8, 1, 8, (256,))  # wider than the column
    assert WL.table("eq32x4096plain").plain and WL.table("eq32x4096plain").consts == WL.table("eq32x4096").consts


@pytest.mark.parametrize("rows,width,out_width", [(1, 4, 6), (2, 1, 1), (3, 2, 4), (6, 3, 6), (16, 4, 8), (33, 5, 11),
                                                  (100, 16, 23), (4096, 32, 44), (9, 4, 3)])
def test_sum_circuit_equals_oracle_circuit(rows, width, out_width):
    """The library's SUM-aggregation circuit has the oracle's gate count,
    depth and number of outputs for every shape tried."""
    t, a, b, c, ol, ninp = O.sum_netlist(rows, width, out_width)
    depth = [0] * ninp
    for k in range(t.size):
        depth.append(1 + max(depth[a[k]], depth[b[k]], depth[c[k]] if c[k] >= 0 else 0))
    levels = max(depth[ninp:]) if t.size else 0
    assert F.sum_plan_info(rows, width, out_width) == (int(t.size), levels, out_width)


def test_sum_circuit_limits():
    assert F.sum_plan_info(0, 8, 5) == (0, 0, 5)  # empty table: every output bit a known zero
    for bad in [(4, 0, 4), (4, 8, 0), (4, 8, 65), (1 << 23, 1, 8)]:
        with pytest.raises(F.FsqlError):
            F.sum_plan_info(*bad)


@pytest.mark.parametrize("is_min", [False, True])
@pytest.mark.parametrize("rows,width", [(0, 4), (1, 4), (2, 3), (5, 3), (7, 8), (64, 32), (4096, 32)])
def test_extreme_circuits_equal_oracle_circuits(is_min, rows, width):
    t, a, b, c, ol, ninp = O.extreme_netlist(is_min, rows, width)
    depth = [0] * ninp
    for k in range(t.size):
        depth.append(1 + max(depth[a[k]], depth[b[k]], depth[c[k]] if c[k] >= 0 else 0))
    levels = max(depth[ninp:]) if t.size else 0
    assert F.extreme_plan_info(is_min, rows, width) == (int(t.size), levels)


def test_big_key_encryption_equals_oracle():
    """Keyswitch-first ciphertexts (N + 1 words under the N-bit key): the
    library's encryption equals the oracle's word for word and decrypts."""
    ctx = F.Context(11, device=-1)
    o = O.Oracle(11)
    bits = np.random.default_rng(8).integers(0, 2, 64).astype(np.uint8)
    a = ctx.encrypt_big_bits(bits, 5, 7)
    assert a.shape == (64, 1025)
    assert np.array_equal(a, o.encrypt_big_bits(bits, 5, 7))
    assert np.array_equal(ctx.decrypt_big_bits(a), bits)
    assert np.array_equal(o.decrypt_big_bits(a), bits)


def test_workload_range_bounds_fit_the_column_width():
    """Every RANGE query of the serving mix and of the named tables has
    lo <= hi < 2^width: an hi of 2^width would be encrypted as 0 (its w bits)
    while the SQL answer treats it as 2^width."""
    for seed in range(1, 6):
        for t in WL.serving_queries(300, seed=seed, min_log2=8, max_log2=16):
            if t.pred == WL.PRED_RANGE:
                assert t.consts[0] <= t.consts[1] < (1 << t.width), (seed, t.name, t.consts)
        for name in ("range16x65536", "range4x16"):
            t = WL.table(name, seed=seed)
            assert t.consts[0] <= t.consts[1] < (1 << t.width)
