#!/usr/bin/env python
"""Benchmark of the oblivious scan-select hot path on B300.

One step = one full oblivious scan (all rows, every circuit level: XNOR
layer, AND tree, payload masks; each gate one TFHE gate bootstrap) of the
4096-row uint32 equality workload by default, with inputs resident in HBM.
Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead, on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank scans its own replica of the table on its own
GPU (rows are independent; no data-path collective); the barrier and the
max-over-ranks time use torch.distributed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic modular multiplications of one gate bootstrap: n CMux x (8
# transforms x N/2 log N butterflies + 2l x 2 x N multiply-accumulate
# products), one multiplication mod p per item with one transform prime; the
# two-prime engine does each of them once per prime.
MODMULS_PER_BOOTSTRAP = 630 * (8 * 5120 + 12 * 1024)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="eq32x4096",
                    choices=["eq32x4096", "eq4x16", "range16x65536", "range16x65536maj", "lt8x64", "lt8x64maj", "range4x16",
                             "range4x16maj", "eq32x4096plain", "range16x65536plain", "eq4x16plain", "eq32x4096sum",
                             "eq32x4096plainsum", "eq32x4096ksfirst", "gates",
                             "serving"])
    ap.add_argument("--queries", type=int, default=200, help="measured queries per serving phase")
    ap.add_argument("--warm-queries", type=int, default=20, help="warm-up queries per serving phase")
    ap.add_argument("--serve-log2", default="8,10",
                    help="serving tables: rows = round(2^U[lo, hi]) (the serving workload statement: 8,16)")
    ap.add_argument("--catalog", type=int, default=8, help="distinct encrypted tables the served queries scan")
    ap.add_argument("--serve-inflight", type=int, default=8, help="outstanding queries in the saturated phase")
    ap.add_argument("--serve-budget-gb", type=float, default=96.0, help="server scratch budget (GiB)")
    ap.add_argument("--verify-queries", type=int, default=2, help="served queries per phase checked by the oracle")
    ap.add_argument("--serve-loads", default="0.5,0.9",
                    help="Poisson phases, as fractions of the saturated query rate")
    ap.add_argument("--batch", type=int, default=65536, help="gates per step of the gate microbenchmark")
    ap.add_argument("--sweep", default="",
                    help="gate microbenchmark over these batch sizes (comma separated, e.g. 1,16,256,4096,65536,1048576)")
    ap.add_argument("--engine", default="default", choices=["default", "dual_prime", "goldilocks"])
    ap.add_argument("--rows", type=int, default=None, help="override the workload's row count")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-rows", type=int, default=1, help="rows of the workload the oracle times")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-gate", action="store_true", help="skip the per-gate-launch baseline")
    ap.add_argument("--verify-rows", type=int, default=2,
                    help="rows of the timed scan the CPU oracle recomputes word for word (first, matching, last...)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--exact-warmup", action="store_true",
                    help="run exactly --warmup warm-up steps even below 3 (single long measurements; the line says so)")
    ap.add_argument("--walk", action="store_true", help="batched scans as one device-walked launch")
    ap.add_argument("--br-shape", type=int, default=None,
                    help="blind-rotation launch shape index (implies --no-autotune)")
    ap.add_argument("--seed", type=int, default=1)
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        busy = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def bus_id_of(dev: int) -> str | None:
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return None


class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, use_cuda: bool):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl" if use_cuda else "gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            if self.pg.get_backend() == "nccl":
                import torch
                self.pg.barrier(device_ids=[self.local])
                torch.cuda.synchronize()
            else:
                self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def gates_per_row(table) -> int:
    """Gate bootstraps per row of the table's circuit (the library's scheduler)."""
    from paper_2510_15413_b300 import fhesql as F

    npay = len(table.payloads)
    if table.plain:
        return F.plan_info_plain(table.pred, table.width, npay, table.payload_width, table.consts)[0]
    return F.plan_info(table.pred, table.width, npay, table.payload_width)[0]


def oracle_gates_per_row(table) -> int:
    """Gate bootstraps per row from the oracle's own netlist (the reference
    arm loads nothing of the library)."""
    from oracle import oracle as O

    npay = len(table.payloads)
    if table.plain:
        return int(O.netlist_plain(table.pred, table.width, npay, table.payload_width, table.consts)[0].size)
    return int(O.netlist3(table.pred, table.width, npay, table.payload_width)[0].size)


def warmups(args) -> int:
    """Warm-up steps: at least 3 (the timing rule), unless --exact-warmup."""
    return args.warmup if args.exact_warmup else max(3, args.warmup)


def pick_shape(ctx, args):
    """The blind-rotation launch shape: given on the command line, else the
    library's autotuner (timed on synthetic gates before anything is timed
    here), else the context's default; and the device level walker if asked."""
    if args.walk:
        ctx.set_walk(True)
    if args.br_shape is not None:
        ctx.br_shape = args.br_shape
        return None
    return None if args.no_autotune else ctx.autotune()


def oracle_scan(o, table, col, cst, pays):
    if table.ks_first:
        return o.scan_ks_first(table.pred, table.width, col, cst, pays, table.payload_width)
    if table.plain:
        return o.scan_plain(table.pred, table.width, col, table.consts, pays, table.payload_width)
    return o.scan(table.pred, table.width, col, cst, pays, table.payload_width)


# ------------------------------------------------------------------ CPU oracle timing
def oracle_rate(table, seed: int, rows: int):
    """Time the oracle on `rows` rows of the table (own encryption, untimed);
    returns (gate bootstraps/s, threads, seconds, gates)."""
    from oracle import oracle as O
    from paper_2510_15413_b300 import workloads as WL

    threads = os.cpu_count() or 1
    O.set_threads(threads)
    o = O.Oracle(seed)
    idx = list(range(rows))
    w, pw = table.width, table.payload_width
    enc = o.encrypt_big_bits if table.ks_first else o.encrypt_bits
    col = np.concatenate([enc(table.column_bits().reshape(table.rows, w)[r], WL.STREAM_COLUMN, r * w)
                          for r in idx])
    cst = enc(table.const_bits(), WL.STREAM_CONST, 0)
    pays = [np.concatenate([enc(table.payload_bits(q).reshape(table.rows, pw)[r], WL.STREAM_PAYLOAD,
                                           q * table.rows * pw + r * pw) for r in idx])
            for q in range(len(table.payloads))]
    t0 = time.perf_counter()
    oracle_scan(o, table, col, cst, pays)
    dt = time.perf_counter() - t0
    gates = rows * oracle_gates_per_row(table)
    o.close()
    return gates / dt, O.max_threads(), dt, gates


def verify_rows_with_oracle(table, seed, k, match, outs):
    """Recompute k rows (first, a matching one, last, then evenly spaced) with
    the CPU oracle from its own encryptions and compare every output word."""
    from oracle import oracle as O
    from paper_2510_15413_b300 import workloads as WL

    O.set_threads(os.cpu_count() or 1)
    o = O.Oracle(seed)
    m_want, _ = table.expected()
    cand = [0, int(np.argmax(m_want)) if m_want.any() else 1, table.rows - 1]
    cand += [int(r) for r in np.linspace(0, table.rows - 1, max(k, 3)).astype(int)]
    rows = []
    for r in cand:
        if r not in rows:
            rows.append(r)
        if len(rows) == k:
            break
    rows = sorted(rows)
    w, pw = table.width, table.payload_width
    enc = o.encrypt_big_bits if table.ks_first else o.encrypt_bits
    col = np.concatenate([enc(table.column_bits().reshape(table.rows, w)[r], WL.STREAM_COLUMN, r * w)
                          for r in rows])
    cst = enc(table.const_bits(), WL.STREAM_CONST, 0)
    pays = [np.concatenate([enc(table.payload_bits(q).reshape(table.rows, pw)[r], WL.STREAM_PAYLOAD,
                                           q * table.rows * pw + r * pw) for r in rows])
            for q in range(len(table.payloads))]
    t0 = time.perf_counter()
    om, oouts = oracle_scan(o, table, col, cst, pays)
    dt = time.perf_counter() - t0
    o.close()
    gm = match.cpu().numpy().view(np.uint32)[rows]
    same = bool(np.array_equal(gm, om))
    for q, out in enumerate(outs):
        same &= bool(np.array_equal(out.cpu().numpy().view(np.uint32)[rows], oouts[q]))
    return {"rows": [int(r) for r in rows], "words_equal": same, "oracle_seconds": dt}


def run_reference(args, dist):
    from paper_2510_15413_b300 import workloads as WL

    if dist.rank != 0:
        return
    t = WL.table(args.workload, seed=args.seed, rows=args.rows)
    rates, secs = [], []
    for _ in range(args.warmup):
        oracle_rate(t, args.seed, args.cpu_rows)
    for _ in range(args.steps):
        r, threads, dt, gates = oracle_rate(t, args.seed, args.cpu_rows)
        rates.append(r)
        secs.append(dt)
    value = statistics.median(rates)
    dt = statistics.median(secs)
    gpr = oracle_gates_per_row(t)
    sample = f"{args.cpu_rows} row(s) of {args.workload} = {args.cpu_rows * gpr} gate bootstraps per step"
    line = {"impl": "reference", "metric": "gate bootstraps/s", "value": value, "unit": "gate bootstraps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (exact integer)",
            "data": "synthetic", "rows_per_s": value / gpr,
            "config": {"workload": args.workload, "rows": t.rows, "width": t.width,
                       "gates_per_row": gpr, "parallelism": "oracle threads over independent gates"},
            "cpu_baseline": {"value": value, "unit": "gate bootstraps/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "gate bootstraps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ gate microbenchmark
def run_gates(args, dist):
    """One step = one batch of independent random gate bootstraps."""
    import torch

    from oracle import oracle as O
    from paper_2510_15413_b300 import fhesql as F
    from paper_2510_15413_b300 import workloads as WL

    dev = dist.local
    torch.cuda.set_device(dev)
    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ctx = F.Context(args.seed, device=dev, engine=args.engine)
    alu = F.measure_alu_peaks(dev)
    tuned = pick_shape(ctx, args)
    B = args.batch
    types, xb, yb = WL.gates(B, seed=args.seed)
    x = ctx.encrypt_bits(xb, WL.STREAM_GATES, 0)
    y = ctx.encrypt_bits(yb, WL.STREAM_GATES, B)
    dt = torch.from_numpy(types).to(f"cuda:{dev}")
    da = torch.from_numpy(x.view(np.int32)).to(f"cuda:{dev}")
    db = torch.from_numpy(y.view(np.int32)).to(f"cuda:{dev}")
    out = torch.zeros((B, ctx.words), dtype=torch.int32, device=f"cuda:{dev}")
    st = torch.cuda.current_stream()
    for _ in range(warmups(args)):
        ctx.gate_batch(dt, da, db, out, stream=st)
    torch.cuda.synchronize()
    sampler = ClockSampler(bus_id_of(dev))
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.4)
    ctx.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.gate_batch(dt, da, db, out, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    dist.barrier()
    kt = ctx.profile_end()
    clocks = sampler.stop()
    ms = dist.max(e0.elapsed_time(e1))
    value = dist.world * B * args.steps / (ms / 1e3)
    truth = np.array([[1, 1, 1, 0], [0, 0, 0, 1], [0, 1, 1, 1], [0, 1, 1, 0], [1, 0, 0, 1]], np.uint8)[types, 2 * xb + yb]
    correct = bool(np.array_equal(ctx.decrypt_bits(out.cpu().numpy().view(np.uint32)), truth))
    roof = roofline_of(kt, ms, sms, peaks, f"gates{B}", alu, ctx.engine, args.steps,
                       shape=ctx.br_shape, sm_mhz=(clocks or {}).get("sm_mhz"))
    # end to end: pinned host inputs -> device -> gates -> host, copies timed
    hx, hy, ht = (torch.from_numpy(x.view(np.int32)).pin_memory(), torch.from_numpy(y.view(np.int32)).pin_memory(),
                  torch.from_numpy(types).pin_memory())
    hout = torch.zeros((B, ctx.words), dtype=torch.int32).pin_memory()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(st)
    for _ in range(args.e2e_steps):
        dt.copy_(ht, non_blocking=True)
        da.copy_(hx, non_blocking=True)
        db.copy_(hy, non_blocking=True)
        ctx.gate_batch(dt, da, db, out, stream=st)
        hout.copy_(out, non_blocking=True)
    f1.record(st)
    torch.cuda.synchronize()
    e2e_ms = dist.max(f0.elapsed_time(f1))
    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        O.set_threads(threads)
        o = O.Oracle(args.seed)
        m = min(B, 8 * threads)
        ox = o.encrypt_bits(xb[:m], WL.STREAM_GATES, 0)
        oy = o.encrypt_bits(yb[:m], WL.STREAM_GATES, B)
        t0 = time.perf_counter()
        o.gate_batch(types[:m].astype(np.int32), ox, oy)
        dt_cpu = time.perf_counter() - t0
        cpu = {"value": m / dt_cpu, "unit": "gate bootstraps/s", "cores": O.max_threads(), "kind": "oracle",
               "sample": f"{m} random gates of the batch in {dt_cpu:.1f} s"}
        o.close()
    line = {"metric": "gate bootstraps/s", "value": value, "unit": "gate bootstraps/s", "n_gpus": dist.world,
            "steps": args.steps, "warmup": warmups(args), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 (exact integer)",
            "data": "synthetic (seeded random gates, seeded keys)",
            "config": {"workload": f"gates x{B}", "engine": ["goldilocks", "dual_prime"][ctx.engine],
                       "launch_shape": dict(F.br_shape_info(ctx.br_shape), index=ctx.br_shape,
                                         autotune_ms=tuned[1] if tuned else None),
                       "gate_types": "NAND/AND/OR/XOR/XNOR uniform",
                       "l2": "inputs %s L2 (%.0f MB)" % ("larger than" if 2 * B * 2524 > 126e6 else "within",
                                                          2 * B * 2524 / 1e6)},
            "correct": correct, "roofline": roof, "cpu_baseline": cpu,
            "e2e": ({"value": dist.world * B * args.e2e_steps / (e2e_ms / 1e3), "unit": "gate bootstraps/s",
                     "h2d_bytes_per_step": (2 * B * ctx.words * 4 + B), "d2h_bytes_per_step": B * ctx.words * 4}
                    if args.e2e_steps > 0 and e2e_ms > 0 else None),
            "gpu_launches": int(kt["blind_rotate_launches"] + kt["keyswitch_launches"]) + args.steps,
            "clocks": clocks, "peaks": {"kind": peak_kind, "hbm_gbs": peaks.get("hbm_gbs"), "sms": sms}}
    ctx.close()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def run_gate_sweep(args, dist):
    """Gate microbenchmark over batch sizes: for each B, CUDA-event time of
    whole batches of B independent random gate bootstraps (inputs resident),
    every output decrypted against the gate's truth table.  B = 1 is the
    per-gate launch path; larger B use the batched persistent launches."""
    import torch

    from paper_2510_15413_b300 import fhesql as F
    from paper_2510_15413_b300 import workloads as WL

    dev = dist.local
    torch.cuda.set_device(dev)
    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ctx = F.Context(args.seed, device=dev, engine=args.engine)
    alu = F.measure_alu_peaks(dev)
    st = torch.cuda.current_stream()
    truth_tab = np.array([[1, 1, 1, 0], [0, 0, 0, 1], [0, 1, 1, 1], [0, 1, 1, 0], [1, 0, 0, 1]], np.uint8)
    sizes = [int(v) for v in args.sweep.split(",") if v]
    sampler = ClockSampler(bus_id_of(dev))
    sampler.start()
    points, launches, all_ok = [], 0, True
    for B in sizes:
        types, xb, yb = WL.gates(B, seed=args.seed)
        x = ctx.encrypt_bits(xb, WL.STREAM_GATES, 0)
        y = ctx.encrypt_bits(yb, WL.STREAM_GATES, B)
        dt = torch.from_numpy(types).to(f"cuda:{dev}")
        da = torch.from_numpy(x.view(np.int32)).to(f"cuda:{dev}")
        db = torch.from_numpy(y.view(np.int32)).to(f"cuda:{dev}")
        out = torch.zeros((B, ctx.words), dtype=torch.int32, device=f"cuda:{dev}")
        warm = 3 if B <= (1 << 16) else 1
        for _ in range(warm):
            ctx.gate_batch(dt, da, db, out, stream=st)
        torch.cuda.synchronize()
        # enough whole batches for about a second of device time (at least one)
        t_est = time.perf_counter()
        ctx.gate_batch(dt, da, db, out, stream=st)
        torch.cuda.synchronize()
        one = time.perf_counter() - t_est
        steps = max(1, min(200, int(1.0 / max(one, 1e-6))))
        dist.barrier()
        torch.cuda.synchronize()
        ctx.profile_begin()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            ctx.gate_batch(dt, da, db, out, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        kt = ctx.profile_end()
        ms = dist.max(e0.elapsed_time(e1))
        launches += int(kt["blind_rotate_launches"] + kt["keyswitch_launches"]) + steps
        ok = bool(np.array_equal(ctx.decrypt_bits(out.cpu().numpy().view(np.uint32)),
                                 truth_tab[types, 2 * xb + yb]))
        all_ok &= ok
        roof = roofline_of(kt, ms, sms, peaks, f"gates{B}", alu, ctx.engine, steps)
        points.append({"batch": B, "gate_bootstraps_per_s": dist.world * B * steps / (ms / 1e3),
                       "ms_per_batch": ms / steps, "steps": steps, "warmup": warm, "correct": ok,
                       "br_ms_per_launch": roof["avg_launch_ms"], "frac": roof["frac"]})
        del dt, da, db, out
        torch.cuda.empty_cache()
    clocks = sampler.stop()
    head = points[-1]
    line = {"metric": "gate bootstraps/s", "value": head["gate_bootstraps_per_s"], "unit": "gate bootstraps/s",
            "n_gpus": dist.world, "steps": head["steps"], "warmup": head["warmup"],
            "ms_per_step": head["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 (exact integer)",
            "data": "synthetic (seeded random gates, seeded keys)",
            "config": {"workload": "gates sweep " + ",".join(map(str, sizes)),
                       "engine": ["goldilocks", "dual_prime"][ctx.engine],
                       "gate_types": "NAND/AND/OR/XOR/XNOR uniform",
                       "l2": "inputs within L2 below B = 2^14, larger above"},
            "correct": all_ok, "sweep": points, "gpu_launches": launches, "clocks": clocks,
            "batched_vs_per_gate": (head["gate_bootstraps_per_s"] / points[0]["gate_bootstraps_per_s"]
                                    if points[0]["batch"] == 1 else None),
            "peaks": {"kind": peak_kind, "hbm_gbs": peaks.get("hbm_gbs"), "sms": sms}}
    ctx.close()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving
def run_serving(args, dist):
    """Continuous batching under load (the serving workload).  A catalog of
    seeded encrypted tables with rows = round(2^U[lo, hi]), widths {8, 16,
    32}, EQ or RANGE (50/50), 1-2 payload columns of the column's width
    stays resident; every query scans one catalog table with its own
    encrypted constants and its own output buffers.  Phases: saturated
    (closed loop, --serve-inflight queries outstanding), then Poisson
    arrivals at 0.5x and 0.9x of the saturated query rate; each phase runs
    --warm-queries warm-up queries, then --queries measured ones (latency =
    submit to done, as the server records it).  Sampled finished queries have
    one row recomputed by the CPU oracle, word for word."""
    import random

    import torch

    from paper_2510_15413_b300 import fhesql as F
    from paper_2510_15413_b300 import workloads as WL

    dev = dist.local
    torch.cuda.set_device(dev)
    ctx = F.Context(args.seed, device=dev, engine=args.engine)
    tuned = pick_shape(ctx, args)
    W = ctx.words
    lo2, hi2 = (float(v) for v in args.serve_log2.split(","))
    catalog = WL.serving_queries(args.catalog, seed=args.seed, min_log2=lo2, max_log2=hi2)
    d = lambda a: torch.from_numpy(a.view(np.int32)).to(f"cuda:{dev}")
    tabs = []
    for t in catalog:
        col, _, pays = WL.encrypt_table(ctx, t)
        tabs.append({"t": t, "column": d(col), "payloads": [d(p) for p in pays]})
    torch.cuda.synchronize()
    budget = int(args.serve_budget_gb * (1 << 30))
    rng = np.random.default_rng(args.seed + 17)
    qcount = [0]

    def make_query():
        """A query on a random catalog table: fresh constants, encrypted at
        their own positions of the constant stream, and fresh outputs."""
        i = int(rng.integers(0, len(tabs)))
        base = tabs[i]["t"]
        w = base.width
        if base.pred == WL.PRED_EQ:
            consts = (int(base.column[int(rng.integers(0, base.rows))]),)
        else:
            span = max(1, (1 << w) // 10)
            lo = int(rng.integers(0, (1 << w) - span))  # hi stays a w-bit value
            consts = (lo, lo + span)
        t = WL.Table(base.name, base.rows, w, base.pred, base.column, base.payloads, base.payload_width, consts)
        k = qcount[0]
        qcount[0] += 1
        cst_first = k * 2 * w
        cst = ctx.encrypt_bits(t.const_bits(), WL.STREAM_CONST, cst_first)
        return {"i": i, "t": t, "k": k, "cst_first": cst_first, "const": d(cst),
                "match": torch.zeros((t.rows, W), dtype=torch.int32, device=f"cuda:{dev}"),
                "outs": [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device=f"cuda:{dev}")
                         for _ in t.payloads]}

    def submit(srv, q):
        tb = tabs[q["i"]]
        # the server's stream does not wait for torch's: the new outputs'
        # zero-fill and the constant's copy must be complete first
        torch.cuda.current_stream().synchronize()
        q["id"] = srv.submit(tb["column"], q["t"].rows, q["t"].width, q["t"].pred, q["const"], tb["payloads"],
                             q["t"].payload_width, q["match"], q["outs"])

    def finish(srv, q, keep):
        state, lat = srv.status(q["id"])
        q["lat_ms"] = lat
        q["ok"] = state == F.Q_DONE
        m_want, p_want = q["t"].expected()
        got = ctx.decrypt_bits(q["match"].cpu().numpy().view(np.uint32))
        q["correct"] = bool(np.array_equal(got, m_want))
        if keep:  # keep the outputs of queries the oracle will check
            q["match_h"] = q["match"].cpu().numpy().view(np.uint32)
            q["outs_h"] = [o.cpu().numpy().view(np.uint32) for o in q["outs"]]
        del q["match"], q["outs"], q["const"]

    def phase(rate_qps):
        """rate 0: saturated closed loop; else Poisson arrivals at that rate."""
        srv = F.Server(ctx, scratch_budget_bytes=budget)
        total = args.warm_queries + args.queries
        rnd = random.Random(args.seed + int(rate_qps * 1000))
        pending, done = [], []
        t0 = time.perf_counter()
        next_t = 0.0
        submitted = 0
        while submitted < total or pending:
            now = time.perf_counter() - t0
            can_submit = submitted < total and (
                (rate_qps == 0 and len(pending) < args.serve_inflight) or (rate_qps > 0 and now >= next_t))
            if can_submit:
                q = make_query()
                q["measured"] = submitted >= args.warm_queries
                submit(srv, q)
                q["t_sub"] = time.perf_counter() - t0
                pending.append(q)
                submitted += 1
                if rate_qps > 0:
                    next_t += rnd.expovariate(rate_qps)
                continue
            still = []
            for q in pending:
                if srv.status(q["id"])[0] in (F.Q_DONE, F.Q_FAILED, F.Q_CANCELLED):
                    q["t_done"] = time.perf_counter() - t0
                    finish(srv, q, keep=q["measured"] and sum(1 for x in done if "match_h" in x) < args.verify_queries)
                    done.append(q)
                else:
                    still.append(q)
            pending = still
            time.sleep(0.002)
        st = srv.stats()
        srv.close()
        meas = [q for q in done if q["measured"]]
        wall = max(q["t_done"] for q in meas) - min(q["t_sub"] for q in meas)
        lat = [q["lat_ms"] for q in meas]
        rows = sum(q["t"].rows for q in meas)
        gates = sum(q["t"].rows * q["t"].gates_per_row for q in meas)
        return {"rate_qps": rate_qps, "warm_queries": args.warm_queries, "queries": len(meas), "wall_s": wall,
                "rows_per_s": rows / wall, "gate_bootstraps_per_s": gates / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(max(lat)), "rounds": st["rounds"], "server_busy_ms": st["busy_ms"],
                "correct": all(q["ok"] and q["correct"] for q in done)}, [q for q in done if "match_h" in q]

    sat, checked = phase(0.0)
    q_rate = sat["queries"] / sat["wall_s"]
    runs = [sat]
    for frac in (float(v) for v in args.serve_loads.split(",") if v):
        r, c = phase(frac * q_rate)
        r["load"] = frac
        runs.append(r)
        checked += c
    # oracle recomputation of one row of each kept query (the first matching row, else row 0)
    verified = None
    if args.verify_queries > 0 and checked and dist.rank == 0:
        from oracle import oracle as O
        O.set_threads(os.cpu_count() or 1)
        o = O.Oracle(args.seed)
        same, rows_checked = True, 0
        for q in checked:
            t = q["t"]
            m_want, _ = t.expected()
            r = int(np.argmax(m_want)) if m_want.any() else 0
            w, pw = t.width, t.payload_width
            ocol = o.encrypt_bits(t.column_bits().reshape(t.rows, w)[r], WL.STREAM_COLUMN, r * w)
            opays = [o.encrypt_bits(t.payload_bits(k).reshape(t.rows, pw)[r], WL.STREAM_PAYLOAD,
                                    k * t.rows * pw + r * pw) for k in range(len(t.payloads))]
            ocst = o.encrypt_bits(t.const_bits(), WL.STREAM_CONST, q["cst_first"])
            om, oouts = o.scan(t.pred, w, ocol, ocst, opays, pw)
            same &= bool(np.array_equal(q["match_h"][r], om[0]))
            for gout, oo in zip(q["outs_h"], oouts):
                same &= bool(np.array_equal(gout.reshape(t.rows, pw, W)[r], oo.reshape(pw, W)))
            rows_checked += 1
        o.close()
        verified = {"queries_checked": rows_checked, "words_equal": same}
    head = runs[-1]
    line = {"metric": "served encrypted rows/s", "value": head["rows_per_s"], "unit": "rows/s",
            "n_gpus": dist.world, "steps": len(runs), "warmup": args.warm_queries,
            "ms_per_step": head["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 (exact integer)", "data": "synthetic (seeded table catalog and query mix)",
            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
            "config": {"workload": "serving", "queries_per_phase": args.queries, "warm_queries": args.warm_queries,
                       "rows": f"round(2^U[{lo2:g},{hi2:g}])", "catalog_tables": len(catalog),
                       "widths": [8, 16, 32], "preds": "EQ/RANGE 50/50 (ripple comparator)",
                       "payload_columns": "1-2", "saturated_inflight": args.serve_inflight,
                       "scratch_budget_gb": args.serve_budget_gb, "engine": ["goldilocks", "dual_prime"][ctx.engine],
                       "launch_shape": dict(F.br_shape_info(ctx.br_shape), index=ctx.br_shape)},
            "phases": runs, "oracle_rows": verified,
            "correct": all(r["correct"] for r in runs)}
    ctx.close()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def code_only(text: bytes) -> bytes:
    """C++ source without // comments, trailing blanks and empty lines (what
    the kernel hash covers, so that comment edits keep it)."""
    lines = (re.sub(rb"//.*$", b"", ln).rstrip() for ln in text.split(b"\n"))
    return b"\n".join(ln for ln in lines if ln)


def kernel_source_hash(root: str = ROOT) -> str:
    """sha256 of the throughput blind-rotation kernel's code: ntt.cuh and
    kernels.cu up to the end of blind_rotate_kernel (twiddle tables, gate
    linear forms, the kernel body and its wrapper), comments and blank lines
    removed."""
    h = hashlib.sha256()
    with open(os.path.join(root, "paper_2510_15413_b300", "csrc", "ntt.cuh"), "rb") as fh:
        h.update(code_only(fh.read()))
    with open(os.path.join(root, "paper_2510_15413_b300", "csrc", "kernels.cu"), "rb") as fh:
        text = fh.read()
    marker = b"// ---------------------------------------------------------------- end of blind_rotate_kernel's device code"
    assert marker in text, "kernels.cu lost its end-of-blind_rotate_kernel marker"
    h.update(code_only(text.split(marker)[0]))
    return h.hexdigest()


def profile_fields(path: str) -> dict:
    """The `- key: value` lines of a committed profile summary."""
    fields = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip()
    return fields


def measured_traffic(workload: str, root: str = ROOT, code_hash: str | None = None):
    """Per-launch DRAM bytes of the blind rotation from the committed ncu
    summary of this workload, if it was taken on the current kernel code."""
    try:
        fields = profile_fields(os.path.join(root, "profiles", f"blind_rotate_{workload}_dram.md"))
        if fields.get("kernel_source_sha256") != (code_hash or kernel_source_hash(root)):
            return None
        return float(fields["dram_bytes_per_launch"])
    except Exception:
        return None


def measured_issue(shape, root: str = ROOT, code_hash: str | None = None):
    """Warp instructions of blind_rotate_kernel per gate per CMux from the
    committed ncu capture of launch shape `shape`, if it was taken on the
    current kernel code (else None)."""
    try:
        fields = profile_fields(os.path.join(root, "profiles", "blind_rotate_own_slot_gates888.md"))
        if fields.get("kernel_source_sha256") != (code_hash or kernel_source_hash(root)):
            return None
        if int(fields["launch_shape"]) != shape:
            return None
        return float(fields["warp_instructions"]) / (float(fields["gates"]) * float(fields["cmux_per_gate"]))
    except Exception:
        return None


def roofline_of(kt, ms, sms, peaks, workload=None, alu=None, engine=1, steps=1, shape=None, sm_mhz=None):
    """Roofline of the blind rotation (the dominant kernel): algorithmic
    modular multiplications per second over its CUDA-event time, against the
    measured rate of the engine's butterfly (one modular multiplication each)
    from the library's in-register microkernel.  Two-prime engine: every
    algorithmic multiplication is done once per prime, so it counts twice,
    against the 32-bit Shoup butterfly rate; the one-prime engine counts it
    once, against the 64-bit-prime butterfly rate (the definition of the
    per-bootstrap figure)."""
    br_ms = kt["blind_rotate_ms"]
    launches = max(1, kt["blind_rotate_launches"])
    per_bootstrap = MODMULS_PER_BOOTSTRAP * (2 if engine == 1 else 1)
    achieved = per_bootstrap * kt["gates"] / (br_ms / 1e3) / 1e12 if br_ms > 0 else 0.0
    out = {"bound": "alu", "kernel": "blind_rotate_kernel", "achieved": achieved, "unit": "Tmodmul/s",
           "modmuls_per_bootstrap": per_bootstrap,
           "traffic": measured_traffic(workload) if workload else None, "traffic_unit": "DRAM bytes per launch",
           "avg_launch_ms": br_ms / launches, "share_of_step": br_ms / ms if ms else None,
           "keyswitch_ms_total": kt["keyswitch_ms"], "keyswitch_ms_per_step": kt["keyswitch_ms"] / max(1, steps)}
    if alu:
        peak = (alu["dual_prime_bfly_per_s"] if engine == 1 else alu["goldilocks_bfly_per_s"]) / 1e12
        out.update({"peak": peak, "frac": achieved / peak if peak else None,
                    "peak_kind": "measured: in-register %s butterfly rate of this GPU (library microkernel)"
                                 % ("two-prime Shoup" if engine == 1 else "64-bit-prime"),
                    "alu_rates_per_s": {k: alu[k] for k in ("imad_per_s", "imad_hi_per_s", "imad_wide_per_s",
                                                            "dual_prime_bfly_per_s", "goldilocks_bfly_per_s")}})
        if engine == 1 and br_ms > 0:
            # the same kernel against the planned single-prime definition:
            # 33.55 M multiplications mod 2^64 - 2^32 + 1 per bootstrap
            g_ach = MODMULS_PER_BOOTSTRAP * kt["gates"] / (br_ms / 1e3) / 1e12
            g_peak = alu["goldilocks_bfly_per_s"] / 1e12
            out["goldilocks_equivalent"] = {"achieved": g_ach, "peak": g_peak, "frac": g_ach / g_peak}
    else:
        out.update({"peak": None, "frac": None, "peak_kind": "unavailable"})
    # the instruction-issue ceiling beside the ALU one: 4 warp instructions
    # per SM per clock at the SM clock measured during the timed region
    inst = measured_issue(shape) if shape is not None else None
    if inst and sm_mhz and br_ms > 0:
        full = sms * 4 * sm_mhz * 1e6 / (inst * 630)
        rate = kt["gates"] / (br_ms / 1e3)
        out["issue_ceiling"] = {"warp_instructions_per_gate_per_cmux": inst, "sm_mhz": sm_mhz,
                                "bootstraps_per_s_at_full_issue": full, "achieved_bootstraps_per_s": rate,
                                "frac": rate / full,
                                "source": "profiles/blind_rotate_own_slot_gates888.md (ncu, same kernel code)"}
    else:
        out["issue_ceiling"] = None
    return out


# ------------------------------------------------------------------ GPU run
def run_ours(args, dist):
    import torch

    from paper_2510_15413_b300 import fhesql as F
    from paper_2510_15413_b300 import workloads as WL

    dev = dist.local
    torch.cuda.set_device(dev)
    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    ctx = F.Context(args.seed, device=dev, engine=args.engine)
    alu = F.measure_alu_peaks(dev)
    tuned = pick_shape(ctx, args)
    t = WL.table(args.workload, seed=args.seed, rows=args.rows)
    col, cst, pays = WL.encrypt_table(ctx, t)
    W = ctx.big_words if t.ks_first else ctx.words
    dec_bits = ctx.decrypt_big_bits if t.ks_first else ctx.decrypt_bits

    def dec_uint(ct, width):
        bits = dec_bits(ct.reshape(-1, W)).reshape(-1, width).astype(np.uint64)
        return (bits << np.arange(width, dtype=np.uint64)).sum(axis=1)

    dcol = torch.from_numpy(col.view(np.int32)).to(f"cuda:{dev}")
    dcst = torch.from_numpy(cst.view(np.int32)).to(f"cuda:{dev}")
    dpay = [torch.from_numpy(p.view(np.int32)).to(f"cuda:{dev}") for p in pays]
    match = torch.zeros((t.rows, W), dtype=torch.int32, device=f"cuda:{dev}")
    outs = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32, device=f"cuda:{dev}") for _ in pays]
    st = torch.cuda.current_stream()

    sums = [torch.zeros((t.sum_width, W), dtype=torch.int32, device=f"cuda:{dev}") for _ in pays] \
        if t.aggregate else []

    def step():
        if t.plain:
            ctx.scan_select_plain(dcol, t.rows, t.width, t.pred, t.consts, dpay, t.payload_width, match, outs,
                                  stream=st)
        elif t.ks_first:
            ctx.scan_select_ks_first(dcol, t.rows, t.width, t.pred, dcst, dpay, t.payload_width, match, outs,
                                     stream=st)
        else:
            ctx.scan_select(dcol, t.rows, t.width, t.pred, dcst, dpay, t.payload_width, match, outs, stream=st)
        for o_, s_ in zip(outs, sums):
            ctx.aggregate_sum(o_, t.rows, t.payload_width, t.sum_width, s_, stream=st)

    for _ in range(warmups(args)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: exactly K steps, device-resident inputs
    sampler = ClockSampler(bus_id_of(dev))
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.4)
    ctx.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    dist.barrier()
    ktimes = ctx.profile_end()
    clocks = sampler.stop()
    ms = dist.max(e0.elapsed_time(e1))
    if args.walk:
        ctx.walk_status()  # raises if a grid-barrier wait of the walker ran out of time
    gpr = gates_per_row(t)
    sum_gates = len(sums) * F.sum_plan_info(t.rows, t.payload_width, t.sum_width)[0] if t.aggregate else 0
    gates_per_step = t.rows * gpr + sum_gates
    value = dist.world * gates_per_step * args.steps / (ms / 1e3)

    # ---- correctness of the timed outputs (plaintext answer)
    m_want, p_want = t.expected()
    got_m = dec_bits(match.cpu().numpy().view(np.uint32))
    correct = bool(np.array_equal(got_m, m_want))
    for q, o_ in enumerate(outs):
        correct &= bool(np.array_equal(dec_uint(o_.cpu().numpy().view(np.uint32), t.payload_width), p_want[q]))
    for q, s_ in enumerate(sums):
        bits = dec_bits(s_.cpu().numpy().view(np.uint32))
        got_sum = sum(int(b) << j for j, b in enumerate(bits))
        correct &= got_sum == int(p_want[q].astype(object).sum()) % (1 << t.sum_width)

    # ---- roofline of the dominant kernel (blind rotation)
    roofline = roofline_of(ktimes, ms, sms, peaks, args.workload, alu, ctx.engine, args.steps,
                           shape=ctx.br_shape, sm_mhz=(clocks or {}).get("sm_mhz"))
    if args.walk:
        roofline["kernel"] = "scan_walk_kernel (blind rotations and keyswitches of every level, one launch)"

    # ---- end to end through the public C-ABI with host buffers (copies inside the timed region)
    h2d = (col.size + (0 if t.plain else cst.size) + sum(p.size for p in pays)) * 4
    d2h = (t.rows * W + len(pays) * t.rows * t.payload_width * W + len(sums) * t.sum_width * W) * 4
    e2e = None
    if args.e2e_steps > 0:
        hcol = torch.from_numpy(col.view(np.int32)).pin_memory()
        hcst = torch.from_numpy(cst.view(np.int32)).pin_memory()
        hpay = [torch.from_numpy(p.view(np.int32)).pin_memory() for p in pays]
        hmatch = torch.zeros((t.rows, W), dtype=torch.int32).pin_memory()
        houts = [torch.zeros((t.rows, t.payload_width, W), dtype=torch.int32).pin_memory() for _ in pays]

        hsums = [torch.zeros((t.sum_width, W), dtype=torch.int32).pin_memory() for _ in sums]

        def e2e_step():
            if t.plain or t.aggregate or t.ks_first:  # pinned host -> device, the step, device -> host
                dcol.copy_(hcol, non_blocking=True)
                if not t.plain:
                    dcst.copy_(hcst, non_blocking=True)
                for d_, h_ in zip(dpay, hpay):
                    d_.copy_(h_, non_blocking=True)
                step()
                hmatch.copy_(match, non_blocking=True)
                for h_, d_ in zip(houts, outs):
                    h_.copy_(d_, non_blocking=True)
                for h_, d_ in zip(hsums, sums):
                    h_.copy_(d_, non_blocking=True)
            else:
                ctx.scan_select_host(hcol, t.rows, t.width, t.pred, hcst, hpay, t.payload_width, hmatch, houts,
                                     stream=st)

        e2e_step()
        dist.barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(st)
        for _ in range(args.e2e_steps):
            e2e_step()
        f1.record(st)
        torch.cuda.synchronize()
        dist.barrier()
        e2e_ms = dist.max(f0.elapsed_time(f1))
        e2e = {"value": dist.world * gates_per_step * args.e2e_steps / (e2e_ms / 1e3), "unit": "gate bootstraps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        correct &= bool(np.array_equal(dec_bits(hmatch.numpy().view(np.uint32)), m_want))

    # ---- oracle recomputation of sampled rows of the timed scan
    verified = None
    if args.verify_rows > 0 and dist.rank == 0:
        verified = verify_rows_with_oracle(t, args.seed, args.verify_rows, match, outs)

    # ---- per-gate launch baseline and batched rate on the 16-row table
    small = None
    if not args.no_per_gate:
        ts = WL.table("eq4x16", seed=args.seed)
        scol, scst, spay = WL.encrypt_table(ctx, ts)
        s_dcol = torch.from_numpy(scol.view(np.int32)).cuda()
        s_dcst = torch.from_numpy(scst.view(np.int32)).cuda()
        s_dpay = [torch.from_numpy(p.view(np.int32)).cuda() for p in spay]
        s_match = torch.zeros((ts.rows, ctx.words), dtype=torch.int32, device="cuda")
        s_outs = [torch.zeros((ts.rows, ts.payload_width, ctx.words), dtype=torch.int32, device="cuda") for _ in spay]
        res = {}
        for mode in ("batched", "per_gate"):
            run = lambda: ctx.scan_select(s_dcol, ts.rows, ts.width, ts.pred, s_dcst, s_dpay, ts.payload_width,
                                          s_match, s_outs, per_gate=(mode == "per_gate"), stream=st)
            run()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            run()
            b.record(st)
            torch.cuda.synchronize()
            res[mode] = ts.rows * gates_per_row(ts) / (a.elapsed_time(b) / 1e3)
        small = {"workload": "eq4x16 (16 rows, 176 gate bootstraps)", "batched_gate_bootstraps_per_s": res["batched"],
                 "per_gate_gate_bootstraps_per_s": res["per_gate"],
                 "batched_over_per_gate": res["batched"] / res["per_gate"],
                 "large_batched_over_per_gate": value / dist.world / res["per_gate"]}

    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        r, threads, dt, gates = oracle_rate(t, args.seed, args.cpu_rows)
        cpu = {"value": r, "unit": "gate bootstraps/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_rows} row(s) of {args.workload} = {gates} gate bootstraps in {dt:.1f} s"}

    line = {
        "metric": "gate bootstraps/s", "value": value, "unit": "gate bootstraps/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": warmups(args), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (exact integer)",
        "data": "synthetic (seeded tables, seeded keys)",
        "rows_per_s": dist.world * t.rows * args.steps / (ms / 1e3),
        "config": {"workload": args.workload, "rows": t.rows, "width": t.width, "pred": t.pred,
                   "constants": "plaintext" if t.plain else "encrypted",
                   "order": "keyswitch first (N+1-word ciphertexts)" if t.ks_first else "keyswitch after bootstrap",
                   "payload_columns": len(t.payloads), "payload_width": t.payload_width,
                   "gates_per_row": gpr, "gate_bootstraps_per_step": gates_per_step,
                   "sum_gate_bootstraps_per_step": sum_gates,
                   "params": "n=630 N=1024 Bg=2^7 l=3 ks 4^8 Torus32",
                   "engine": ["goldilocks", "dual_prime"][ctx.engine],
                   "launch_shape": dict(F.br_shape_info(ctx.br_shape), index=ctx.br_shape,
                                         autotune_ms=tuned[1] if tuned else None),
                   "level_walk": "device walker (one launch per scan)" if args.walk else "one launch pair per level",
                   "l2": "inputs larger than L2 (%.0f MB column+payload per step)" % (h2d / 1e6),
                   "parallelism": f"replica per GPU x{dist.world}"},
        "correct": correct,
        "oracle_rows": verified,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(ktimes["blind_rotate_launches"] + ktimes["keyswitch_launches"]),
        "clocks": clocks,
        "per_gate_baseline": small,
        "peaks": {"kind": peak_kind, "hbm_gbs": peaks.get("hbm_gbs"), "sms": sms},
    }
    ctx.close()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        dist.init(use_cuda=False)
        run_reference(args, dist)
    else:
        dist.init(use_cuda=True)
        if args.workload == "gates" and args.sweep:
            run_gate_sweep(args, dist)
        else:
            {"gates": run_gates, "serving": run_serving}.get(args.workload, run_ours)(args, dist)
    dist.close()


if __name__ == "__main__":
    main()
