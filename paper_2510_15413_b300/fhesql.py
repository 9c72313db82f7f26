"""Python binding of libfhesql.so (include/fhesql.h): argument marshalling only.

Every homomorphic step runs in the library's CUDA kernels; this module only
turns numpy arrays / torch tensors into pointers and checks return codes.
If the in-tree library is missing, loading raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfhesql.so")

FSQL_OK, FSQL_ERR_ARG, FSQL_ERR_OOM, FSQL_ERR_CUDA, FSQL_ERR_TIMEOUT, FSQL_ERR_ADMISSION, FSQL_ERR_UNSUPPORTED = range(7)
GATES = {"NAND": 0, "AND": 1, "OR": 2, "XOR": 3, "XNOR": 4, "NOR": 5, "ANDNY": 6, "ANDYN": 7, "ORNY": 8, "ORYN": 9,
         "MAJNYY": 10, "XOR3": 11, "MAJ": 12}
FSQL_EQ, FSQL_LT, FSQL_RANGE, FSQL_LT_MAJ, FSQL_RANGE_MAJ = 0, 1, 2, 3, 4
FSQL_ENGINE_DEFAULT, FSQL_ENGINE_GOLDILOCKS, FSQL_ENGINE_DUAL_PRIME = -1, 0, 1
ENGINES = {"default": -1, "goldilocks": 0, "dual_prime": 1}

# every symbol include/fhesql.h declares
API = ["fsql_params_default", "fsql_params_toy", "fsql_ctx_create", "fsql_ctx_create_engine", "fsql_ctx_engine",
       "fsql_ctx_set_br_gates", "fsql_ctx_br_gates", "fsql_ctx_set_br_shape", "fsql_ctx_br_shape",
       "fsql_br_shape_info", "fsql_ctx_set_latency_mode", "fsql_autotune", "fsql_measure_alu_peaks",
       "fsql_ctx_set_walk", "fsql_walk_status", "fsql_debug_walk_skip_block",
       "fsql_ctx_destroy", "fsql_ctx_params",
       "fsql_ctx_device_bytes", "fsql_export_keys", "fsql_encrypt", "fsql_encrypt_bits", "fsql_encrypt_uint",
       "fsql_phase", "fsql_decrypt_bits", "fsql_decrypt_uint", "fsql_gate_batch", "fsql_blind_rotate_extract",
       "fsql_keyswitch", "fsql_debug_ntt_mul", "fsql_plan_info", "fsql_scan_select", "fsql_scan_select_host",
       "fsql_scan_select_plain", "fsql_plan_info_plain", "fsql_aggregate_sum", "fsql_sum_plan_info",
       "fsql_encrypt_big_bits", "fsql_decrypt_big_bits", "fsql_gate_batch_ks_first", "fsql_scan_select_ks_first",
       "fsql_aggregate_max", "fsql_aggregate_min", "fsql_extreme_plan_info",
       "fsql_profile_begin", "fsql_profile_end", "fsql_gate_batch_noalloc", "fsql_server_create",
       "fsql_server_submit", "fsql_server_status", "fsql_server_wait", "fsql_server_cancel",
       "fsql_server_get_stats", "fsql_server_destroy", "fsql_last_error"]
FSQL_MAX_PAYLOADS = 8
Q_WAITING, Q_RUNNING, Q_DONE, Q_FAILED, Q_CANCELLED = range(5)


class FsqlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fhesql error {code}: {msg}")
        self.code = code


class fsql_kernel_times(C.Structure):
    _fields_ = [("blind_rotate_ms", C.c_double), ("keyswitch_ms", C.c_double),
                ("blind_rotate_launches", C.c_uint64), ("keyswitch_launches", C.c_uint64), ("gates", C.c_uint64)]


class fsql_query(C.Structure):
    _fields_ = [("d_column", C.c_void_p), ("rows", C.c_size_t), ("width", C.c_uint32), ("pred", C.c_uint32),
                ("d_const", C.c_void_p), ("n_payloads", C.c_uint32), ("payload_width", C.c_uint32),
                ("d_payloads", C.c_void_p * 8), ("d_match", C.c_void_p), ("d_out_payloads", C.c_void_p * 8),
                ("plain", C.c_uint32), ("pad", C.c_uint32), ("consts", C.c_uint64 * 2)]


class fsql_server_stats(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("rounds", C.c_uint64), ("gates", C.c_uint64), ("busy_ms", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("waiting", C.c_uint64), ("running", C.c_uint64),
                ("scratch_used", C.c_size_t)]


class fsql_alu_peaks(C.Structure):
    _fields_ = [("imad_per_s", C.c_double), ("imad_hi_per_s", C.c_double), ("imad_wide_per_s", C.c_double),
                ("dual_prime_bfly_per_s", C.c_double), ("goldilocks_bfly_per_s", C.c_double),
                ("dual_prime_bfly_wide_per_s", C.c_double), ("dual_prime_bfly_madwide_per_s", C.c_double),
                ("sm_count", C.c_int), ("clock_mhz", C.c_double)]


class fsql_params(C.Structure):
    _fields_ = [("n", C.c_uint32), ("N", C.c_uint32), ("bg_bits", C.c_uint32), ("l", C.c_uint32),
                ("ks_base_bits", C.c_uint32), ("ks_t", C.c_uint32),
                ("lwe_sigma", C.c_double), ("glwe_sigma", C.c_double)]


_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2510_15413_b300/build.py "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, sz, u32, u64, i32 = C.c_void_p, C.c_size_t, C.c_uint32, C.c_uint64, C.c_int
    sig = {
        "fsql_params_default": (i32, [C.POINTER(fsql_params)]),
        "fsql_params_toy": (i32, [C.POINTER(fsql_params)]),
        "fsql_ctx_create": (i32, [C.POINTER(fsql_params), u64, i32, C.POINTER(vp)]),
        "fsql_ctx_create_engine": (i32, [C.POINTER(fsql_params), u64, i32, i32, C.POINTER(vp)]),
        "fsql_ctx_engine": (i32, [vp, C.POINTER(i32)]),
        "fsql_ctx_set_br_gates": (i32, [vp, i32]),
        "fsql_ctx_set_latency_mode": (i32, [vp, i32]),
        "fsql_ctx_br_gates": (i32, [vp, C.POINTER(i32)]),
        "fsql_ctx_set_br_shape": (i32, [vp, i32]),
        "fsql_ctx_set_walk": (i32, [vp, i32, C.c_double]),
        "fsql_walk_status": (i32, [vp, vp, C.POINTER(C.c_uint)]),
        "fsql_debug_walk_skip_block": (i32, [vp, i32]),
        "fsql_ctx_br_shape": (i32, [vp, C.POINTER(i32)]),
        "fsql_br_shape_info": (i32, [i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
        "fsql_autotune": (i32, [vp, sz, vp, C.POINTER(i32), C.POINTER(C.c_double)]),
        "fsql_ctx_destroy": (None, [vp]),
        "fsql_ctx_params": (i32, [vp, C.POINTER(fsql_params)]),
        "fsql_ctx_device_bytes": (i32, [vp, C.POINTER(sz), C.POINTER(sz)]),
        "fsql_export_keys": (i32, [vp, vp, vp, vp, vp]),
        "fsql_encrypt": (i32, [vp, vp, sz, u64, u64, vp]),
        "fsql_encrypt_bits": (i32, [vp, vp, sz, u64, u64, vp]),
        "fsql_encrypt_uint": (i32, [vp, vp, sz, u32, u64, u64, vp]),
        "fsql_phase": (i32, [vp, vp, sz, vp]),
        "fsql_decrypt_bits": (i32, [vp, vp, sz, vp]),
        "fsql_decrypt_uint": (i32, [vp, vp, sz, u32, vp]),
        "fsql_gate_batch": (i32, [vp, vp, vp, vp, vp, sz, vp]),
        "fsql_gate_batch_noalloc": (i32, [vp, vp, vp, vp, vp, sz, vp]),
        "fsql_blind_rotate_extract": (i32, [vp, vp, vp, vp, vp, sz, vp]),
        "fsql_keyswitch": (i32, [vp, vp, vp, sz, vp]),
        "fsql_debug_ntt_mul": (i32, [vp, vp, vp, vp, vp]),
        "fsql_plan_info": (i32, [u32, u32, u32, u32, C.POINTER(u32), C.POINTER(u32), vp, u32]),
        "fsql_scan_select": (i32, [vp, vp, sz, u32, u32, vp, u32, vp, u32, vp, vp, i32, vp]),
        "fsql_scan_select_host": (i32, [vp, vp, sz, u32, u32, vp, u32, vp, u32, vp, vp, vp]),
        "fsql_scan_select_plain": (i32, [vp, vp, sz, u32, u32, vp, u32, vp, u32, vp, vp, i32, vp]),
        "fsql_aggregate_sum": (i32, [vp, vp, sz, u32, u32, vp, vp]),
        "fsql_encrypt_big_bits": (i32, [vp, vp, sz, u64, u64, vp]),
        "fsql_decrypt_big_bits": (i32, [vp, vp, sz, vp]),
        "fsql_gate_batch_ks_first": (i32, [vp, vp, vp, vp, vp, sz, vp]),
        "fsql_scan_select_ks_first": (i32, [vp, vp, sz, u32, u32, vp, u32, vp, u32, vp, vp, i32, vp]),
        "fsql_aggregate_max": (i32, [vp, vp, sz, u32, vp, vp]),
        "fsql_aggregate_min": (i32, [vp, vp, vp, sz, u32, vp, vp]),
        "fsql_extreme_plan_info": (i32, [i32, sz, u32, C.POINTER(u32), C.POINTER(u32)]),
        "fsql_sum_plan_info": (i32, [sz, u32, u32, C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]),
        "fsql_plan_info_plain": (i32, [u32, u32, u32, u32, vp, C.POINTER(u32), C.POINTER(u32), vp, u32,
                                       C.POINTER(u32)]),
        "fsql_profile_begin": (i32, [vp]),
        "fsql_profile_end": (i32, [vp, C.POINTER(fsql_kernel_times)]),
        "fsql_server_create": (i32, [vp, sz, sz, C.POINTER(vp)]),
        "fsql_server_submit": (i32, [vp, C.POINTER(fsql_query), C.POINTER(u64)]),
        "fsql_server_status": (i32, [vp, u64, C.POINTER(i32), C.POINTER(C.c_double)]),
        "fsql_server_wait": (i32, [vp, u64, C.c_double]),
        "fsql_server_cancel": (i32, [vp, u64]),
        "fsql_server_get_stats": (i32, [vp, C.POINTER(fsql_server_stats)]),
        "fsql_server_destroy": (None, [vp]),
        "fsql_measure_alu_peaks": (i32, [i32, C.POINTER(fsql_alu_peaks)]),
        "fsql_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int) -> None:
    if rc != FSQL_OK:
        raise FsqlError(rc, load().fsql_last_error().decode())


def _ptr(x) -> int:
    """Device or host address of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    if x is None:
        return 0
    return int(x)


def _count(x) -> int:
    return int(x.numel()) if hasattr(x, "numel") else int(np.asarray(x).size)


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    return int(getattr(stream, "cuda_stream", stream))


BR_SHAPES = 9


def br_shape_info(shape: int) -> dict:
    """(kernel kind, gates per CTA, gadget rows per step, staging slots) of a launch shape."""
    k, g, r, st = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(load().fsql_br_shape_info(int(shape), C.byref(k), C.byref(g), C.byref(r), C.byref(st)))
    return {"kind": ["packed", "prime_split", "packed_own_slot"][k.value], "gates_per_cta": g.value,
            "rows_per_step": r.value,
            "stages": st.value}


def measure_alu_peaks(device: int = 0) -> dict:
    """Integer-ALU rates of the GPU (operations per second), from the
    library's in-register microkernels."""
    out = fsql_alu_peaks()
    _check(load().fsql_measure_alu_peaks(device, C.byref(out)))
    return {name: getattr(out, name) for name, _ in fsql_alu_peaks._fields_}


def params_default() -> fsql_params:
    p = fsql_params()
    _check(load().fsql_params_default(C.byref(p)))
    return p


def params_toy() -> fsql_params:
    p = fsql_params()
    _check(load().fsql_params_toy(C.byref(p)))
    return p


def plan_info(pred: int, width: int, n_payloads: int, payload_width: int, max_levels: int = 256):
    g, lv = C.c_uint32(), C.c_uint32()
    widths = np.zeros(max_levels, np.uint32)
    _check(load().fsql_plan_info(pred, width, n_payloads, payload_width, C.byref(g), C.byref(lv),
                                 widths.ctypes.data, max_levels))
    return int(g.value), [int(x) for x in widths[: lv.value]]


def sum_plan_info(rows: int, width: int, out_width: int):
    """(gates, levels, literal outputs) of the SUM-aggregation circuit."""
    g, lv, lit = C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(load().fsql_sum_plan_info(rows, width, out_width, C.byref(g), C.byref(lv), C.byref(lit)))
    return int(g.value), int(lv.value), int(lit.value)


def extreme_plan_info(is_min: bool, rows: int, width: int):
    """(gates, levels) of the MAX (is_min False) or MIN circuit."""
    g, lv = C.c_uint32(), C.c_uint32()
    _check(load().fsql_extreme_plan_info(int(bool(is_min)), rows, width, C.byref(g), C.byref(lv)))
    return int(g.value), int(lv.value)


def _consts_array(consts):
    k = [int(v) for v in consts] + [0, 0]
    return (C.c_uint64 * 2)(k[0], k[1])


def plan_info_plain(pred: int, width: int, n_payloads: int, payload_width: int, consts, max_levels: int = 256):
    """(gates per row, level widths, outputs per row no gate writes) of the
    plaintext-constant circuit for consts = (k,) or (lo, hi)."""
    g, lv, lit = C.c_uint32(), C.c_uint32(), C.c_uint32()
    widths = np.zeros(max_levels, np.uint32)
    _check(load().fsql_plan_info_plain(pred, width, n_payloads, payload_width, _consts_array(consts), C.byref(g),
                                       C.byref(lv), widths.ctypes.data, max_levels, C.byref(lit)))
    return int(g.value), [int(x) for x in widths[: lv.value]], int(lit.value)


class Context:
    """A seeded key set (client secrets on the host, server keys on the device)."""

    def __init__(self, seed: int, params: fsql_params | None = None, device: int = 0, engine="default"):
        self.params = params if params is not None else params_default()
        h = C.c_void_p()
        eng = ENGINES[engine] if isinstance(engine, str) else int(engine)
        _check(load().fsql_ctx_create_engine(C.byref(self.params), int(seed), int(device), eng, C.byref(h)))
        self._h = h
        e = C.c_int()
        _check(load().fsql_ctx_engine(h, C.byref(e)))
        self.engine = int(e.value)
        self.seed = int(seed)
        self.device = device
        self.n = int(self.params.n)
        self.N = int(self.params.N)
        self.words = self.n + 1

    def close(self) -> None:
        if self._h:
            load().fsql_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def br_gates(self) -> int:
        g = C.c_int()
        _check(load().fsql_ctx_br_gates(self._h, C.byref(g)))
        return int(g.value)

    @br_gates.setter
    def br_gates(self, g: int) -> None:
        _check(load().fsql_ctx_set_br_gates(self._h, int(g)))

    def set_latency_mode(self, mode) -> None:
        """Kernel for batches under two gates per SM: 0 (or False) one gate per
        128-thread CTA, 1 (or True) one gate per CTA of three groups, 2 (the
        default) one gate per cluster of six CTAs."""
        _check(load().fsql_ctx_set_latency_mode(self._h, int(mode)))

    @property
    def br_shape(self) -> int:
        """Launch shape index of the blind rotation for large batches (see br_shape_info)."""
        v = C.c_int()
        _check(load().fsql_ctx_br_shape(self._h, C.byref(v)))
        return int(v.value)

    @br_shape.setter
    def br_shape(self, shape: int) -> None:
        _check(load().fsql_ctx_set_br_shape(self._h, int(shape)))

    def set_walk(self, on: bool, timeout_ms: float = 2000.0) -> None:
        """Batched scans as one device-walked launch (bounded grid barriers)."""
        _check(load().fsql_ctx_set_walk(self._h, int(bool(on)), float(timeout_ms)))

    def walk_status(self, stream=None) -> None:
        """Raises FsqlError(FSQL_ERR_TIMEOUT) if a walker barrier wait ran out of time."""
        b = C.c_uint()
        _check(load().fsql_walk_status(self._h, _stream(stream), C.byref(b)))

    def debug_walk_skip_block(self, block: int) -> None:
        _check(load().fsql_debug_walk_skip_block(self._h, int(block)))

    def autotune(self, probe_gates: int = 0, stream=None):
        """Pick the fastest blind-rotation launch shape; returns (shape index, {shape: ms})."""
        best = C.c_int()
        ms = (C.c_double * BR_SHAPES)()
        _check(load().fsql_autotune(self._h, probe_gates, _stream(stream), C.byref(best), ms))
        return int(best.value), {i: float(ms[i]) for i in range(BR_SHAPES) if ms[i] >= 0}

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def device_bytes(self):
        k, s = C.c_size_t(), C.c_size_t()
        _check(load().fsql_ctx_device_bytes(self._h, C.byref(k), C.byref(s)))
        return int(k.value), int(s.value)

    # ---------------------------------------------------------------- keys
    def export_keys(self):
        p = self.params
        s = np.zeros(p.n, np.uint8)
        S = np.zeros(p.N, np.uint8)
        bk = np.zeros((p.n, 2 * p.l, 2, p.N), np.uint32)
        ksk = np.zeros((p.N, p.ks_t, (1 << p.ks_base_bits) - 1, p.n + 1), np.uint32)
        _check(load().fsql_export_keys(self._h, s.ctypes.data, S.ctypes.data, bk.ctypes.data, ksk.ctypes.data))
        return s, S, bk, ksk

    # ---------------------------------------------------------------- client side
    def encrypt(self, mu, stream: int, first_index: int = 0) -> np.ndarray:
        mu = np.ascontiguousarray(mu, dtype=np.uint32).ravel()
        out = np.zeros((mu.size, self.words), np.uint32)
        _check(load().fsql_encrypt(self._h, mu.ctypes.data, mu.size, stream, first_index, out.ctypes.data))
        return out

    def encrypt_bits(self, bits, stream: int, first_index: int = 0) -> np.ndarray:
        bits = np.ascontiguousarray(bits, dtype=np.uint8).ravel()
        out = np.zeros((bits.size, self.words), np.uint32)
        _check(load().fsql_encrypt_bits(self._h, bits.ctypes.data, bits.size, stream, first_index, out.ctypes.data))
        return out

    def encrypt_uint(self, values, width: int, stream: int, first_index: int = 0) -> np.ndarray:
        values = np.ascontiguousarray(values, dtype=np.uint64).ravel()
        out = np.zeros((values.size, width, self.words), np.uint32)
        _check(load().fsql_encrypt_uint(self._h, values.ctypes.data, values.size, width, stream, first_index,
                                        out.ctypes.data))
        return out

    def phase(self, ct) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32).reshape(-1, self.words)
        out = np.zeros(ct.shape[0], np.uint32)
        _check(load().fsql_phase(self._h, ct.ctypes.data, ct.shape[0], out.ctypes.data))
        return out

    def decrypt_bits(self, ct) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32).reshape(-1, self.words)
        out = np.zeros(ct.shape[0], np.uint8)
        _check(load().fsql_decrypt_bits(self._h, ct.ctypes.data, ct.shape[0], out.ctypes.data))
        return out

    def decrypt_uint(self, ct, width: int) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32).reshape(-1, width, self.words)
        out = np.zeros(ct.shape[0], np.uint64)
        _check(load().fsql_decrypt_uint(self._h, ct.ctypes.data, ct.shape[0], width, out.ctypes.data))
        return out

    # ---------------------------------------------------------------- server side (device tensors)
    def gate_batch(self, types, a, b, out, stream=None) -> None:
        count = _count(types)
        _check(load().fsql_gate_batch(self._h, _ptr(types), _ptr(a), _ptr(b), _ptr(out), count, _stream(stream)))

    def gate_batch_noalloc(self, types, a, b, out, stream=None) -> None:
        """fsql_gate_batch without any device allocation (at most 1024 gates)."""
        count = _count(types)
        _check(load().fsql_gate_batch_noalloc(self._h, _ptr(types), _ptr(a), _ptr(b), _ptr(out), count,
                                              _stream(stream)))

    def blind_rotate_extract(self, types, a, b, big, stream=None) -> None:
        count = _count(types)
        _check(load().fsql_blind_rotate_extract(self._h, _ptr(types), _ptr(a), _ptr(b), _ptr(big), count,
                                                _stream(stream)))

    def keyswitch(self, big, out, count: int, stream=None) -> None:
        _check(load().fsql_keyswitch(self._h, _ptr(big), _ptr(out), count, _stream(stream)))

    def debug_ntt_mul(self, digits, poly, out, stream=None) -> None:
        _check(load().fsql_debug_ntt_mul(self._h, _ptr(digits), _ptr(poly), _ptr(out), _stream(stream)))

    def scan_select(self, column, rows: int, width: int, pred: int, const, payloads, payload_width: int, match,
                    out_payloads, per_gate: bool = False, stream=None) -> None:
        k = len(payloads)
        pin = (C.c_void_p * max(1, k))(*[_ptr(p) for p in payloads])
        pout = (C.c_void_p * max(1, k))(*[_ptr(p) for p in out_payloads])
        _check(load().fsql_scan_select(self._h, _ptr(column), rows, width, pred, _ptr(const), k, pin,
                                       payload_width, _ptr(match), pout, int(bool(per_gate)), _stream(stream)))

    # ---- keyswitch-first order: ciphertexts of N + 1 words under the N-bit key
    @property
    def big_words(self) -> int:
        return int(self.params.N) + 1

    def encrypt_big_bits(self, bits, stream: int, first_index: int = 0) -> np.ndarray:
        bits = np.ascontiguousarray(bits, dtype=np.uint8).ravel()
        out = np.zeros((bits.size, self.big_words), np.uint32)
        _check(load().fsql_encrypt_big_bits(self._h, bits.ctypes.data, bits.size, stream, first_index,
                                            out.ctypes.data))
        return out

    def decrypt_big_bits(self, ct) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint32).reshape(-1, self.big_words)
        out = np.zeros(ct.shape[0], np.uint8)
        _check(load().fsql_decrypt_big_bits(self._h, ct.ctypes.data, ct.shape[0], out.ctypes.data))
        return out

    def gate_batch_ks_first(self, types, a, b, out, stream=None) -> None:
        _check(load().fsql_gate_batch_ks_first(self._h, _ptr(types), _ptr(a), _ptr(b), _ptr(out), _count(types),
                                               _stream(stream)))

    def scan_select_ks_first(self, column, rows: int, width: int, pred: int, const, payloads, payload_width: int,
                             match, out_payloads, per_gate: bool = False, stream=None) -> None:
        k = len(payloads)
        pin = (C.c_void_p * max(1, k))(*[_ptr(p) for p in payloads])
        pout = (C.c_void_p * max(1, k))(*[_ptr(p) for p in out_payloads])
        _check(load().fsql_scan_select_ks_first(self._h, _ptr(column), rows, width, pred, _ptr(const), k, pin,
                                                payload_width, _ptr(match), pout, int(bool(per_gate)),
                                                _stream(stream)))

    def aggregate_sum(self, values, rows: int, width: int, out_width: int, out, stream=None) -> None:
        """fsql_aggregate_sum: values [rows, width, n+1] -> out [out_width, n+1], sum mod 2^out_width."""
        _check(load().fsql_aggregate_sum(self._h, _ptr(values), rows, width, out_width, _ptr(out), _stream(stream)))

    def aggregate_max(self, values, rows: int, width: int, out, stream=None) -> None:
        """fsql_aggregate_max: values [rows, width, n+1] -> out [width, n+1]."""
        _check(load().fsql_aggregate_max(self._h, _ptr(values), rows, width, _ptr(out), _stream(stream)))

    def aggregate_min(self, values, match, rows: int, width: int, out, stream=None) -> None:
        """fsql_aggregate_min: values [rows, width, n+1], match [rows, n+1] -> out [width, n+1]."""
        _check(load().fsql_aggregate_min(self._h, _ptr(values), _ptr(match), rows, width, _ptr(out),
                                         _stream(stream)))

    def scan_select_plain(self, column, rows: int, width: int, pred: int, consts, payloads, payload_width: int,
                          match, out_payloads, per_gate: bool = False, stream=None) -> None:
        """fsql_scan_select_plain: consts = (k,) or (lo, hi) as plaintext integers."""
        k = len(payloads)
        pin = (C.c_void_p * max(1, k))(*[_ptr(p) for p in payloads])
        pout = (C.c_void_p * max(1, k))(*[_ptr(p) for p in out_payloads])
        _check(load().fsql_scan_select_plain(self._h, _ptr(column), rows, width, pred, _consts_array(consts), k,
                                             pin, payload_width, _ptr(match), pout, int(bool(per_gate)),
                                             _stream(stream)))

    def scan_select_host(self, column, rows: int, width: int, pred: int, const, payloads, payload_width: int,
                         match, out_payloads, stream=None) -> None:
        k = len(payloads)
        pin = (C.c_void_p * max(1, k))(*[_ptr(p) for p in payloads])
        pout = (C.c_void_p * max(1, k))(*[_ptr(p) for p in out_payloads])
        _check(load().fsql_scan_select_host(self._h, _ptr(column), rows, width, pred, _ptr(const), k, pin,
                                            payload_width, _ptr(match), pout, _stream(stream)))

    def profile_begin(self) -> None:
        _check(load().fsql_profile_begin(self._h))

    def profile_end(self) -> dict:
        t = fsql_kernel_times()
        _check(load().fsql_profile_end(self._h, C.byref(t)))
        return {"blind_rotate_ms": t.blind_rotate_ms, "keyswitch_ms": t.keyswitch_ms,
                "blind_rotate_launches": int(t.blind_rotate_launches),
                "keyswitch_launches": int(t.keyswitch_launches), "gates": int(t.gates)}


class Server:
    """Continuous-batching scan server on a context's device (fsql_server_*)."""

    def __init__(self, ctx: Context, scratch_budget_bytes: int, max_batch_gates: int = 0):
        h = C.c_void_p()
        _check(load().fsql_server_create(ctx.handle, int(scratch_budget_bytes), int(max_batch_gates), C.byref(h)))
        self._h = h
        self.ctx = ctx

    def submit(self, column, rows: int, width: int, pred: int, const, payloads, payload_width: int, match,
               out_payloads, plain_consts=None) -> int:
        """Queue a scan; const is the encrypted constant (device), or None with
        plain_consts = (k,) or (lo, hi) for plaintext constants."""
        q = fsql_query()
        q.d_column, q.rows, q.width, q.pred = _ptr(column), rows, width, pred
        q.d_const, q.n_payloads, q.payload_width = _ptr(const), len(payloads), payload_width
        if plain_consts is not None:
            k = [int(v) for v in plain_consts] + [0, 0]
            q.plain, q.consts[0], q.consts[1] = 1, k[0], k[1]
        for i, (a, b) in enumerate(zip(payloads, out_payloads)):
            q.d_payloads[i] = _ptr(a)
            q.d_out_payloads[i] = _ptr(b)
        q.d_match = _ptr(match)
        qid = C.c_uint64()
        _check(load().fsql_server_submit(self._h, C.byref(q), C.byref(qid)))
        return int(qid.value)

    def status(self, qid: int):
        st, lat = C.c_int(), C.c_double()
        _check(load().fsql_server_status(self._h, qid, C.byref(st), C.byref(lat)))
        return int(st.value), float(lat.value)

    def wait(self, qid: int, timeout_ms: float = 600000.0) -> None:
        _check(load().fsql_server_wait(self._h, qid, timeout_ms))

    def cancel(self, qid: int) -> None:
        _check(load().fsql_server_cancel(self._h, qid))

    def stats(self) -> dict:
        st = fsql_server_stats()
        _check(load().fsql_server_get_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in fsql_server_stats._fields_}

    def close(self) -> None:
        if self._h:
            load().fsql_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
