"""ctypes wrapper around the CPU oracle (oracle/tfhe_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by the package smoke check and
by the benchmark's CPU-baseline leg; never by the product path.  It does not
import the product package and the product does not import it.

Everything is numpy uint32 arrays; ciphertexts are rows of n+1 words, body last.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

P_EQ, P_LT, P_RANGE, P_LT_MAJ, P_RANGE_MAJ = 0, 1, 2, 3, 4
GATES = {"NAND": 0, "AND": 1, "OR": 2, "XOR": 3, "XNOR": 4, "NOR": 5,
         "ANDNY": 6, "ANDYN": 7, "ORNY": 8, "ORYN": 9, "MAJNYY": 10, "XOR3": 11, "MAJ": 12}


class Params(C.Structure):
    _fields_ = [("n", C.c_int32), ("N", C.c_int32), ("bg_bits", C.c_int32), ("l", C.c_int32),
                ("ks_base_bits", C.c_int32), ("ks_t", C.c_int32),
                ("lwe_sigma", C.c_double), ("glwe_sigma", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(Params), C.c_uint64]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_params_default.argtypes = [C.POINTER(Params)]
        L.orc_params_toy.argtypes = [C.POINTER(Params)]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        for f in ("orc_negacyclic_schoolbook", "orc_negacyclic_karatsuba"):
            getattr(L, f).argtypes = [u32p, u32p, u32p, C.c_int]
        L.orc_monomial_mul.argtypes = [u32p, u32p, C.c_int, C.c_int]
        L.orc_bk_words.restype = C.c_size_t
        L.orc_bk_words.argtypes = [C.c_void_p]
        L.orc_ksk_words.restype = C.c_size_t
        L.orc_ksk_words.argtypes = [C.c_void_p]
        for f in ("orc_lwe_key", "orc_glwe_key", "orc_bk", "orc_ksk"):
            getattr(L, f).restype = C.c_void_p
            getattr(L, f).argtypes = [C.c_void_p]
        L.orc_encrypt.argtypes = [C.c_void_p, u32p, C.c_size_t, C.c_uint64, C.c_uint64, u32p]
        L.orc_encrypt_bits.argtypes = [C.c_void_p, u8p, C.c_size_t, C.c_uint64, C.c_uint64, u32p]
        L.orc_phase.argtypes = [C.c_void_p, u32p, C.c_size_t, u32p]
        L.orc_phase_big.argtypes = [C.c_void_p, u32p, C.c_size_t, u32p]
        L.orc_decrypt_bits.argtypes = [C.c_void_p, u32p, C.c_size_t, u8p]
        L.orc_modswitch.restype = C.c_uint32
        L.orc_modswitch.argtypes = [C.c_uint32, C.c_int]
        L.orc_decompose.argtypes = [C.c_uint32, C.c_int, C.c_int, i32p]
        L.orc_external_product.argtypes = [C.c_void_p, C.c_int, u32p, u32p]
        L.orc_blind_rotate.argtypes = [C.c_void_p, u32p, u32p]
        L.orc_sample_extract.argtypes = [C.c_int, u32p, u32p]
        L.orc_keyswitch.argtypes = [C.c_void_p, u32p, u32p]
        L.orc_gate_lincomb.argtypes = [C.c_int, C.c_int, u32p, u32p, u32p]
        L.orc_gate.argtypes = [C.c_void_p, C.c_int, u32p, u32p, u32p]
        L.orc_gate3.argtypes = [C.c_void_p, C.c_int, u32p, u32p, u32p, u32p]
        L.orc_gate_lincomb3.argtypes = [C.c_int, C.c_int, u32p, u32p, u32p, u32p]
        L.orc_gate_plain3.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_netlist3.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_gate_batch.argtypes = [C.c_void_p, i32p, u32p, u32p, u32p, C.c_size_t]
        L.orc_not.argtypes = [C.c_int, u32p, u32p]
        L.orc_netlist.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_gate_plain.argtypes = [C.c_int, C.c_int, C.c_int]
        L.orc_netlist_eval_plain.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, u8p, u8p]
        L.orc_scan.argtypes = [C.c_void_p, C.c_int, C.c_int, u32p, u32p, C.c_int, C.c_int,
                               C.POINTER(C.c_void_p), u32p, C.POINTER(C.c_void_p), C.c_longlong]
        L.orc_netlist_plain.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p,
                                        C.POINTER(C.c_int32)]
        L.orc_netlist_plain_eval.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, u8p, u8p]
        L.orc_scan_plain.argtypes = [C.c_void_p, C.c_int, C.c_int, u32p, C.c_uint64, C.c_uint64, C.c_int, C.c_int,
                                     C.POINTER(C.c_void_p), u32p, C.POINTER(C.c_void_p), C.c_longlong]
        L.orc_sum_netlist.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.POINTER(C.c_int32)]
        L.orc_sum_eval_plain.argtypes = [C.c_int, C.c_int, C.c_int, u8p, u8p]
        L.orc_aggregate_sum.argtypes = [C.c_void_p, u32p, C.c_int, C.c_int, C.c_int, u32p]
        L.orc_extreme_netlist.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]
        L.orc_extreme_eval_plain.argtypes = [C.c_int, C.c_int, C.c_int, u8p, u8p]
        L.orc_aggregate_extreme.argtypes = [C.c_void_p, C.c_int, u32p, C.c_void_p, C.c_int, C.c_int, u32p]
        L.orc_encrypt_big_bits.argtypes = [C.c_void_p, u8p, C.c_size_t, C.c_uint64, C.c_uint64, u32p]
        L.orc_decrypt_big_bits.argtypes = [C.c_void_p, u32p, C.c_size_t, u8p]
        L.orc_gate3_ks_first.argtypes = [C.c_void_p, C.c_int, u32p, u32p, C.c_void_p, u32p]
        L.orc_scan_ks_first.argtypes = [C.c_void_p, C.c_int, C.c_int, u32p, u32p, C.c_int, C.c_int,
                                        C.POINTER(C.c_void_p), u32p, C.POINTER(C.c_void_p), C.c_longlong]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def default_params() -> Params:
    p = Params()
    lib().orc_params_default(C.byref(p))
    return p


def toy_params() -> Params:
    p = Params()
    lib().orc_params_toy(C.byref(p))
    return p


def splitmix64(start: int, k: int) -> int:
    return int(lib().orc_splitmix64(start, k))


def set_threads(k: int) -> None:
    lib().orc_set_threads(int(k))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def _u32(x):
    return np.ascontiguousarray(x, dtype=np.uint32)


def negacyclic_schoolbook(a, b):
    a, b = _u32(a), _u32(b)
    c = np.zeros_like(a)
    lib().orc_negacyclic_schoolbook(a, b, c, a.size)
    return c


def negacyclic_karatsuba(a, b):
    a, b = _u32(a), _u32(b)
    c = np.zeros_like(a)
    lib().orc_negacyclic_karatsuba(a, b, c, a.size)
    return c


def monomial_mul(a, e):
    a = _u32(a)
    out = np.zeros_like(a)
    lib().orc_monomial_mul(a, out, a.size, int(e))
    return out


def modswitch(x: int, N: int) -> int:
    return int(lib().orc_modswitch(int(x) & 0xFFFFFFFF, N))


def decompose(x: int, bg_bits: int = 7, l: int = 3):
    d = np.zeros(l, dtype=np.int32)
    lib().orc_decompose(int(x) & 0xFFFFFFFF, bg_bits, l, d)
    return d


def gate_plain(gate: int, x: int, y: int) -> int:
    return int(lib().orc_gate_plain(gate, x, y))


def netlist(pred: int, w: int, n_payload: int = 0, pw: int = 0):
    """Per-row netlist: (types, a, b, match_wire, n_inputs)."""
    m, ninp = C.c_int32(), C.c_int32()
    g = lib().orc_netlist(pred, w, n_payload, pw, None, None, None, C.byref(m), C.byref(ninp))
    if g < 0:
        raise ValueError("bad netlist request")
    t = np.zeros(g, np.int32)
    a = np.zeros(g, np.int32)
    b = np.zeros(g, np.int32)
    lib().orc_netlist(pred, w, n_payload, pw, t.ctypes.data, a.ctypes.data, b.ctypes.data,
                      C.byref(m), C.byref(ninp))
    return t, a, b, int(m.value), int(ninp.value)


def netlist3(pred: int, w: int, n_payload: int = 0, pw: int = 0):
    """Per-row netlist with third inputs: (types, a, b, c, match_wire, n_inputs); c = -1 for two-input gates."""
    m, ninp = C.c_int32(), C.c_int32()
    g = lib().orc_netlist3(pred, w, n_payload, pw, None, None, None, None, C.byref(m), C.byref(ninp))
    if g < 0:
        raise ValueError("bad netlist request")
    t, a, b, c = (np.zeros(g, np.int32) for _ in range(4))
    lib().orc_netlist3(pred, w, n_payload, pw, t.ctypes.data, a.ctypes.data, b.ctypes.data, c.ctypes.data,
                       C.byref(m), C.byref(ninp))
    return t, a, b, c, int(m.value), int(ninp.value)


def gate_plain3(gate: int, x: int, y: int, z: int) -> int:
    return int(lib().orc_gate_plain3(gate, x, y, z))


def netlist_eval_plain(pred: int, w: int, n_payload: int, pw: int, inputs):
    t, _, _, _, m, ninp = netlist3(pred, w, n_payload, pw)
    inp = np.ascontiguousarray(inputs, dtype=np.uint8)
    assert inp.size == ninp
    wires = np.zeros(ninp + t.size, np.uint8)
    lib().orc_netlist_eval_plain(pred, w, n_payload, pw, inp, wires)
    return wires, m


LIT_FALSE, LIT_TRUE = -1, -2


def _plain_consts(consts):
    k = [int(v) for v in consts] + [0, 0]
    return k[0], k[1]


def netlist_plain(pred: int, w: int, n_payload: int, pw: int, consts):
    """Netlist for plaintext query constants (k,) or (lo, hi): (types, a, b,
    match literal, output literals, n_inputs).  A literal is 2*wire + negated,
    or LIT_FALSE / LIT_TRUE; wires are column bits, payload bits, gate outputs."""
    k0, k1 = _plain_consts(consts)
    m, ninp = C.c_int32(), C.c_int32()
    g = lib().orc_netlist_plain(pred, w, n_payload, pw, k0, k1, None, None, None, C.byref(m), None, C.byref(ninp))
    if g < 0:
        raise ValueError("bad netlist request")
    t, a, b = (np.zeros(max(g, 1), np.int32) for _ in range(3))
    ol = np.zeros(max(1, n_payload * pw), np.int32)
    lib().orc_netlist_plain(pred, w, n_payload, pw, k0, k1, t.ctypes.data, a.ctypes.data, b.ctypes.data,
                            C.byref(m), ol.ctypes.data, C.byref(ninp))
    return t[:g], a[:g], b[:g], int(m.value), ol[:n_payload * pw], int(ninp.value)


def netlist_plain_eval(pred: int, w: int, n_payload: int, pw: int, consts, inputs):
    """(match bit, masked payload bits) of one row under plaintext constants."""
    k0, k1 = _plain_consts(consts)
    inp = np.ascontiguousarray(inputs, dtype=np.uint8)
    assert inp.size == w + n_payload * pw
    out = np.zeros(1 + n_payload * pw, np.uint8)
    if lib().orc_netlist_plain_eval(pred, w, n_payload, pw, k0, k1, inp, out) < 0:
        raise ValueError("bad netlist request")
    return int(out[0]), out[1:]


def gate_lincomb3(gate: int, n: int, a, b, c):
    """Linear combination of a three-input (or two-input) gate on [n+1] words."""
    a, b, c = _u32(a).ravel(), _u32(b).ravel(), _u32(c).ravel()
    out = np.zeros(n + 1, np.uint32)
    if lib().orc_gate_lincomb3(gate, n, a, b, c, out) != 0:
        raise ValueError("bad gate")
    return out


def sum_netlist(rows: int, pw: int, ow: int):
    """SUM-aggregation circuit: (types, a, b, c, output literals [ow], n_inputs)."""
    ninp = C.c_int32()
    g = lib().orc_sum_netlist(rows, pw, ow, None, None, None, None, None, C.byref(ninp))
    if g < 0:
        raise ValueError("bad aggregation shape")
    t, a, b, c = (np.zeros(max(g, 1), np.int32) for _ in range(4))
    ol = np.zeros(ow, np.int32)
    lib().orc_sum_netlist(rows, pw, ow, t.ctypes.data, a.ctypes.data, b.ctypes.data, c.ctypes.data, ol.ctypes.data,
                          C.byref(ninp))
    return t[:g], a[:g], b[:g], c[:g], ol, int(ninp.value)


def sum_eval_plain(rows: int, pw: int, ow: int, values) -> int:
    """The SUM circuit evaluated on plaintext bits of the given row values."""
    vals = [int(v) for v in values]
    assert len(vals) == rows
    bits = np.array([(v >> j) & 1 for v in vals for j in range(pw)], np.uint8)
    out = np.zeros(ow, np.uint8)
    if lib().orc_sum_eval_plain(rows, pw, ow, bits, out) < 0:
        raise ValueError("bad aggregation shape")
    return int(sum(int(out[j]) << j for j in range(ow)))


def extreme_netlist(is_min: bool, rows: int, w: int):
    """MAX (is_min False) or MIN circuit: (types, a, b, c, output literals [w], n_inputs)."""
    ninp = C.c_int32()
    g = lib().orc_extreme_netlist(int(is_min), rows, w, None, None, None, None, None, C.byref(ninp))
    if g < 0:
        raise ValueError("bad aggregation shape")
    t, a, b, c = (np.zeros(max(g, 1), np.int32) for _ in range(4))
    ol = np.zeros(w, np.int32)
    lib().orc_extreme_netlist(int(is_min), rows, w, t.ctypes.data, a.ctypes.data, b.ctypes.data, c.ctypes.data,
                              ol.ctypes.data, C.byref(ninp))
    return t[:g], a[:g], b[:g], c[:g], ol, int(ninp.value)


def extreme_eval_plain(is_min: bool, w: int, values, match=None) -> int:
    """The MAX / MIN circuit on plaintext row values (and match bits for MIN)."""
    vals = [int(v) for v in values]
    bits = [(v >> j) & 1 for v in vals for j in range(w)]
    if is_min:
        bits += [int(m) for m in match]
    out = np.zeros(w, np.uint8)
    if lib().orc_extreme_eval_plain(int(is_min), len(vals), w, np.array(bits, np.uint8), out) < 0:
        raise ValueError("bad aggregation shape")
    return int(sum(int(out[j]) << j for j in range(w)))


class Oracle:
    """Keys for one seed plus the TFHE operations, all on the CPU."""

    def __init__(self, seed: int, params: Params | None = None):
        self.params = params if params is not None else default_params()
        self.seed = int(seed)
        self._h = lib().orc_create(C.byref(self.params), self.seed)
        self.n = int(self.params.n)
        self.N = int(self.params.N)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # keys ---------------------------------------------------------------
    def lwe_key(self):
        return np.ctypeslib.as_array(C.cast(lib().orc_lwe_key(self._h), C.POINTER(C.c_uint8)), (self.n,)).copy()

    def glwe_key(self):
        return np.ctypeslib.as_array(C.cast(lib().orc_glwe_key(self._h), C.POINTER(C.c_uint8)), (self.N,)).copy()

    def bk(self):
        w = lib().orc_bk_words(self._h)
        a = np.ctypeslib.as_array(C.cast(lib().orc_bk(self._h), C.POINTER(C.c_uint32)), (w,)).copy()
        return a.reshape(self.n, 2 * self.params.l, 2, self.N)

    def ksk(self):
        w = lib().orc_ksk_words(self._h)
        a = np.ctypeslib.as_array(C.cast(lib().orc_ksk(self._h), C.POINTER(C.c_uint32)), (w,)).copy()
        nd = (1 << self.params.ks_base_bits) - 1
        return a.reshape(self.N, self.params.ks_t, nd, self.n + 1)

    # client side ----------------------------------------------------------
    def encrypt(self, mu, stream: int, first_index: int = 0):
        mu = _u32(mu).ravel()
        out = np.zeros((mu.size, self.n + 1), np.uint32)
        lib().orc_encrypt(self._h, mu, mu.size, stream, first_index, out)
        return out

    def encrypt_bits(self, bits, stream: int, first_index: int = 0):
        bits = np.ascontiguousarray(bits, dtype=np.uint8).ravel()
        out = np.zeros((bits.size, self.n + 1), np.uint32)
        lib().orc_encrypt_bits(self._h, bits, bits.size, stream, first_index, out)
        return out

    def phase(self, ct):
        ct = _u32(ct).reshape(-1, self.n + 1)
        out = np.zeros(ct.shape[0], np.uint32)
        lib().orc_phase(self._h, ct, ct.shape[0], out)
        return out

    def phase_big(self, ct):
        ct = _u32(ct).reshape(-1, self.N + 1)
        out = np.zeros(ct.shape[0], np.uint32)
        lib().orc_phase_big(self._h, ct, ct.shape[0], out)
        return out

    def decrypt_bits(self, ct):
        ct = _u32(ct).reshape(-1, self.n + 1)
        out = np.zeros(ct.shape[0], np.uint8)
        lib().orc_decrypt_bits(self._h, ct, ct.shape[0], out)
        return out

    # server side ----------------------------------------------------------
    def external_product(self, i: int, glwe):
        glwe = _u32(glwe).ravel()
        out = np.zeros(2 * self.N, np.uint32)
        lib().orc_external_product(self._h, i, glwe, out)
        return out

    def blind_rotate(self, lwe):
        lwe = _u32(lwe).ravel()
        acc = np.zeros(2 * self.N, np.uint32)
        lib().orc_blind_rotate(self._h, lwe, acc)
        return acc

    def sample_extract(self, acc):
        acc = _u32(acc).ravel()
        out = np.zeros(self.N + 1, np.uint32)
        lib().orc_sample_extract(self.N, acc, out)
        return out

    def keyswitch(self, big):
        big = _u32(big).ravel()
        out = np.zeros(self.n + 1, np.uint32)
        lib().orc_keyswitch(self._h, big, out)
        return out

    def lincomb(self, gate: int, a, b):
        a, b = _u32(a).ravel(), _u32(b).ravel()
        out = np.zeros(self.n + 1, np.uint32)
        if lib().orc_gate_lincomb(gate, self.n, a, b, out) != 0:
            raise ValueError("bad gate")
        return out

    def gate(self, gate: int, a, b):
        a, b = _u32(a).ravel(), _u32(b).ravel()
        out = np.zeros(self.n + 1, np.uint32)
        if lib().orc_gate(self._h, gate, a, b, out) != 0:
            raise ValueError("bad gate")
        return out

    def gate3(self, gate: int, a, b, c):
        a, b, c = _u32(a).ravel(), _u32(b).ravel(), _u32(c).ravel()
        out = np.zeros(self.n + 1, np.uint32)
        if lib().orc_gate3(self._h, gate, a, b, c, out) != 0:
            raise ValueError("bad gate")
        return out

    def gate_batch(self, gates, a, b):
        gates = np.ascontiguousarray(gates, dtype=np.int32).ravel()
        a = _u32(a).reshape(-1, self.n + 1)
        b = _u32(b).reshape(-1, self.n + 1)
        out = np.zeros_like(a)
        if lib().orc_gate_batch(self._h, gates, a, b, out, gates.size) != 0:
            raise ValueError("bad gate")
        return out

    def not_(self, a):
        a = _u32(a).ravel()
        out = np.zeros_like(a)
        lib().orc_not(self.n, a, out)
        return out

    def scan(self, pred: int, w: int, column, consts, payloads, pw: int):
        """Scan every row given: returns (match [rows, n+1], [payload outs [rows, pw, n+1]])."""
        W = self.n + 1
        column = _u32(column).reshape(-1, w, W)
        rows = column.shape[0]
        consts = _u32(consts).reshape(-1, W)
        pays = [_u32(p).reshape(rows, pw, W) for p in payloads]
        match = np.zeros((rows, W), np.uint32)
        outs = [np.zeros((rows, pw, W), np.uint32) for _ in pays]
        pin = (C.c_void_p * max(1, len(pays)))(*[p.ctypes.data for p in pays])
        pout = (C.c_void_p * max(1, len(outs)))(*[o.ctypes.data for o in outs])
        rc = lib().orc_scan(self._h, pred, w, column, consts, len(pays), pw, pin, match, pout, rows)
        if rc != 0:
            raise ValueError("scan failed")
        return match, outs

    def aggregate_sum(self, values, rows: int, pw: int, ow: int):
        """Encrypted SUM of rows values of pw bits ([rows, pw, n+1]) mod 2^ow -> [ow, n+1]."""
        W = self.n + 1
        vals = _u32(values).reshape(rows * pw * W)
        out = np.zeros((ow, W), np.uint32)
        if lib().orc_aggregate_sum(self._h, vals, rows, pw, ow, out) != 0:
            raise ValueError("aggregation failed")
        return out

    def aggregate_extreme(self, is_min: bool, values, rows: int, w: int, match=None):
        """Encrypted MAX / MIN of rows values [rows, w, n+1] (MIN: match bits [rows, n+1]) -> [w, n+1]."""
        W = self.n + 1
        vals = _u32(values).reshape(max(rows * w * W, 1)) if rows else np.zeros(1, np.uint32)
        m = _u32(match).reshape(rows * W) if (is_min and rows) else None
        out = np.zeros((w, W), np.uint32)
        rc = lib().orc_aggregate_extreme(self._h, int(is_min), vals, m.ctypes.data if m is not None else None,
                                         rows, w, out)
        if rc != 0:
            raise ValueError("aggregation failed")
        return out

    # ---- keyswitch-first order: ciphertexts of N + 1 words under the N-bit key
    def encrypt_big_bits(self, bits, stream: int, first_index: int = 0):
        bits = np.ascontiguousarray(bits, dtype=np.uint8).ravel()
        out = np.zeros((bits.size, self.N + 1), np.uint32)
        lib().orc_encrypt_big_bits(self._h, bits, bits.size, stream, first_index, out)
        return out

    def decrypt_big_bits(self, ct):
        ct = _u32(ct).reshape(-1, self.N + 1)
        out = np.zeros(ct.shape[0], np.uint8)
        lib().orc_decrypt_big_bits(self._h, ct.ravel(), ct.shape[0], out)
        return out

    def gate3_ks_first(self, gate: int, a, b, c=None):
        a, b = _u32(a).ravel(), _u32(b).ravel()
        cc = _u32(c).ravel() if c is not None else None
        out = np.zeros(self.N + 1, np.uint32)
        if lib().orc_gate3_ks_first(self._h, gate, a, b, cc.ctypes.data if cc is not None else None, out) != 0:
            raise ValueError("bad gate")
        return out

    def scan_ks_first(self, pred: int, w: int, column, consts, payloads, pw: int):
        """orc_scan in keyswitch-first order: every ciphertext [N+1] words."""
        W = self.N + 1
        column = _u32(column).reshape(-1, w, W)
        rows = column.shape[0]
        consts = _u32(consts).reshape(-1, W)
        pays = [_u32(p).reshape(rows, pw, W) for p in payloads]
        match = np.zeros((rows, W), np.uint32)
        outs = [np.zeros((rows, pw, W), np.uint32) for _ in pays]
        pin = (C.c_void_p * max(1, len(pays)))(*[p.ctypes.data for p in pays])
        pout = (C.c_void_p * max(1, len(outs)))(*[o.ctypes.data for o in outs])
        if lib().orc_scan_ks_first(self._h, pred, w, column, consts, len(pays), pw, pin, match, pout, rows) != 0:
            raise ValueError("scan failed")
        return match, outs

    def scan_plain(self, pred: int, w: int, column, consts, payloads, pw: int):
        """Scan with plaintext query constants (k,) or (lo, hi): returns
        (match [rows, n+1], [payload outs [rows, pw, n+1]])."""
        W = self.n + 1
        column = _u32(column).reshape(-1, w, W)
        rows = column.shape[0]
        k0, k1 = _plain_consts(consts)
        pays = [_u32(p).reshape(rows, pw, W) for p in payloads]
        match = np.zeros((rows, W), np.uint32)
        outs = [np.zeros((rows, pw, W), np.uint32) for _ in pays]
        pin = (C.c_void_p * max(1, len(pays)))(*[p.ctypes.data for p in pays])
        pout = (C.c_void_p * max(1, len(outs)))(*[o.ctypes.data for o in outs])
        rc = lib().orc_scan_plain(self._h, pred, w, column, k0, k1, len(pays), pw, pin, match, pout, rows)
        if rc != 0:
            raise ValueError("scan failed")
        return match, outs
