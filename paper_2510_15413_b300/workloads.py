"""Seeded synthetic workloads (plaintext side only; no homomorphic arithmetic).

The paper measures on u32 key/value tables it does not publish (§6.1 D); these
generators stand in for them with the shapes of the benchmark workloads:

  eq4x16        16 rows, one 4-bit column c ~ U[0,16), one 4-bit payload,
                WHERE c = k with k ~ U[0,16)
  eq32x4096     4096 rows, one uint32 column (uniform), one uint32 payload,
                WHERE c = k with k drawn from the column (about one match)
  range16x65536 65536 rows, one uint16 column (uniform), two uint16 payloads,
                WHERE lo <= c < hi with hi - lo = 6554 (10% selectivity)
  <name>maj     the same table with the majority-chain comparator
  <name>plain   the same table with the query constants given as plaintexts
  <name>sum     the same scan followed by the SUM of each masked payload column
  <name>ksfirst the same scan in keyswitch-first order (N + 1-word ciphertexts)
  gates(B)      B independent gates: random bit pairs, gate type uniform in
                {NAND, AND, OR, XOR, XNOR}

Values come from numpy's PCG64 seeded with (seed, purpose); encryption
randomness is separate (SplitMix64 streams inside the library and oracle):
stream 5 encrypts the column, 6 the payloads, 7 the query constants,
8 gate inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

STREAM_COLUMN, STREAM_PAYLOAD, STREAM_CONST, STREAM_GATES = 5, 6, 7, 8
PRED_EQ, PRED_LT, PRED_RANGE, PRED_LT_MAJ, PRED_RANGE_MAJ = 0, 1, 2, 3, 4
MICRO_GATES = (0, 1, 2, 3, 4)  # NAND, AND, OR, XOR, XNOR


@dataclass
class Table:
    name: str
    rows: int
    width: int
    pred: int
    column: np.ndarray                 # uint64 [rows]
    payloads: list = field(default_factory=list)  # list of uint64 [rows]
    payload_width: int = 0
    consts: tuple = ()                 # (k,) or (lo, hi)
    plain: bool = False                # constants given to the server as plaintexts
    aggregate: bool = False            # SUM of each masked payload column after the scan
    ks_first: bool = False             # keyswitch-first order: ciphertexts under the N-bit key

    @property
    def sum_width(self) -> int:
        """Output bits of an exact SUM of one payload column over all rows."""
        return self.payload_width + max(1, (self.rows - 1).bit_length())

    def const_bits(self) -> np.ndarray:
        bits = []
        for v in self.consts:
            bits += [(int(v) >> i) & 1 for i in range(self.width)]
        return np.array(bits, np.uint8)

    def column_bits(self) -> np.ndarray:
        return ((self.column[:, None] >> np.arange(self.width, dtype=np.uint64)) & 1).astype(np.uint8).ravel()

    def payload_bits(self, q: int) -> np.ndarray:
        p = self.payloads[q]
        return ((p[:, None] >> np.arange(self.payload_width, dtype=np.uint64)) & 1).astype(np.uint8).ravel()

    def expected(self):
        """Plaintext SQL answer: (match [rows] 0/1, masked payloads list)."""
        c = self.column
        if self.pred == PRED_EQ:
            m = c == np.uint64(self.consts[0])
        elif self.pred in (PRED_LT, PRED_LT_MAJ):
            m = c < np.uint64(self.consts[0])
        else:
            m = (c >= np.uint64(self.consts[0])) & (c < np.uint64(self.consts[1]))
        return m.astype(np.uint8), [np.where(m, p, np.uint64(0)) for p in self.payloads]

    @property
    def gates_per_row(self) -> int:
        """Bootstraps per row with encrypted constants (with plaintext
        constants the count depends on the constant's bits; the library's
        plan_info_plain gives it)."""
        if self.plain:
            raise ValueError("gate count of a plaintext-constant scan depends on the constants")
        w = self.width
        pred = {PRED_EQ: 2 * w - 1, PRED_LT: 4 * w - 3, PRED_RANGE: 2 * (4 * w - 3) + 1,
                PRED_LT_MAJ: w, PRED_RANGE_MAJ: 2 * w + 1}[self.pred]
        return pred + len(self.payloads) * self.payload_width


def _rng(seed: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(purpose)]))


def table(name: str, seed: int = 1, rows: int | None = None) -> Table:
    """A named workload table; the suffix "maj" gives the same table with the
    majority-chain comparator (LT_MAJ / RANGE_MAJ) instead of the ripple one,
    the suffix "plain" the same table with plaintext query constants, the
    suffix "sum" the same scan followed by a SUM of its masked payloads."""
    if name.endswith("ksfirst"):
        t = table(name[:-7], seed, rows)
        t.ks_first = True
        t.name = name
        return t
    if name.endswith("sum"):
        t = table(name[:-3], seed, rows)
        t.aggregate = True
        t.name = name
        return t
    if name.endswith("plain"):
        t = table(name[:-5], seed, rows)
        t.plain = True
        t.name = name
        return t
    if name.endswith("maj"):
        t = table(name[:-3], seed, rows)
        t.pred = {PRED_LT: PRED_LT_MAJ, PRED_RANGE: PRED_RANGE_MAJ}[t.pred]
        t.name = name
        return t
    g = _rng(seed, 1)
    if name == "eq4x16":
        r = rows or 16
        c = g.integers(0, 16, r, dtype=np.uint64)
        p = g.integers(0, 16, r, dtype=np.uint64)
        k = int(g.integers(0, 16))
        return Table(name, r, 4, PRED_EQ, c, [p], 4, (k,))
    if name == "eq32x4096":
        r = rows or 4096
        c = g.integers(0, 1 << 32, r, dtype=np.uint64)
        p = g.integers(0, 1 << 32, r, dtype=np.uint64)
        k = int(c[int(g.integers(0, r))])
        return Table(name, r, 32, PRED_EQ, c, [p], 32, (k,))
    if name == "range16x65536":
        r = rows or 65536
        c = g.integers(0, 1 << 16, r, dtype=np.uint64)
        ps = [g.integers(0, 1 << 16, r, dtype=np.uint64) for _ in range(2)]
        span = 6554
        lo = int(g.integers(0, 65536 - span))  # hi = lo + span stays below 2^16
        return Table(name, r, 16, PRED_RANGE, c, ps, 16, (lo, lo + span))
    if name == "lt8x64":
        r = rows or 64
        c = g.integers(0, 256, r, dtype=np.uint64)
        p = g.integers(0, 256, r, dtype=np.uint64)
        return Table(name, r, 8, PRED_LT, c, [p], 8, (int(g.integers(0, 256)),))
    if name == "range4x16":
        r = rows or 16
        c = g.integers(0, 16, r, dtype=np.uint64)
        p = g.integers(0, 16, r, dtype=np.uint64)
        lo = int(g.integers(0, 12))
        return Table(name, r, 4, PRED_RANGE, c, [p], 4, (lo, lo + 4))
    raise KeyError(name)


def serving_queries(count: int, seed: int = 1, min_log2: float = 8.0, max_log2: float = 10.0):
    """Seeded query mix for the serving benchmark: rows = round(2^U[min, max]),
    width in {8, 16, 32}, EQ or RANGE (50/50), 1-2 payload columns of the same
    width; EQ constants come from the column, RANGE bounds cover about 10% of
    the value range."""
    g = _rng(seed, 3)
    out = []
    for i in range(count):
        rows = int(round(2 ** g.uniform(min_log2, max_log2)))
        w = int(g.choice([8, 16, 32]))
        npay = int(g.integers(1, 3))
        c = g.integers(0, 1 << w, rows, dtype=np.uint64)
        pays = [g.integers(0, 1 << w, rows, dtype=np.uint64) for _ in range(npay)]
        if g.integers(0, 2) == 0:
            out.append(Table(f"q{i}", rows, w, PRED_EQ, c, pays, w, (int(c[int(g.integers(0, rows))]),)))
        else:
            span = max(1, (1 << w) // 10)
            lo = int(g.integers(0, (1 << w) - span))  # hi = lo + span stays below 2^w
            out.append(Table(f"q{i}", rows, w, PRED_RANGE, c, pays, w, (lo, lo + span)))
    return out


def gates(batch: int, seed: int = 1):
    """(types uint8 [B], x bits [B], y bits [B]) for the gate microbenchmark."""
    g = _rng(seed, 2)
    types = np.array(MICRO_GATES, np.uint8)[g.integers(0, len(MICRO_GATES), batch)]
    x = g.integers(0, 2, batch).astype(np.uint8)
    y = g.integers(0, 2, batch).astype(np.uint8)
    return types, x, y


def encrypt_table(enc, t: Table):
    """Encrypt a table with any object exposing encrypt_bits(bits, stream, first_index)
    (the library context or the oracle) -> (column, const, [payloads]); a
    keyswitch-first table uses encrypt_big_bits (N + 1-word ciphertexts)."""
    fn = enc.encrypt_big_bits if t.ks_first else enc.encrypt_bits
    col = fn(t.column_bits(), STREAM_COLUMN, 0)
    cst = fn(t.const_bits(), STREAM_CONST, 0)
    pays = [fn(t.payload_bits(q), STREAM_PAYLOAD, q * t.rows * t.payload_width) for q in range(len(t.payloads))]
    return col, cst, pays
