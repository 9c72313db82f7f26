"""Host logic of bench.py's roofline fields (CPU): the kernel-code hash that
keys the committed ncu summaries, the parsing of those summaries, and the
issue-ceiling arithmetic.  No GPU and no product library."""
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_code_only_ignores_comments_and_blank_lines():
    a = b"int x = 1;  // one\n\n// a note\nint y = 2;\n"
    b = b"int x = 1;\nint y = 2;   \n\n\n"
    assert bench.code_only(a) == bench.code_only(b) == b"int x = 1;\nint y = 2;"
    assert bench.code_only(b"int x = 3;\nint y = 2;") != bench.code_only(b)


def _tree(tmp_path):
    """A copy of the hashed sources and the two profile summaries."""
    for rel in ("paper_2510_15413_b300/csrc/ntt.cuh", "paper_2510_15413_b300/csrc/kernels.cu",
                "profiles/blind_rotate_own_slot_gates888.md", "profiles/blind_rotate_eq32x4096_dram.md"):
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    return tmp_path


def test_kernel_hash_follows_code_not_comments(tmp_path):
    root = str(_tree(tmp_path))
    h0 = bench.kernel_source_hash(root)
    assert h0 == bench.kernel_source_hash(ROOT)
    k = tmp_path / "paper_2510_15413_b300/csrc/kernels.cu"
    text = k.read_bytes()
    k.write_bytes(b"// an added comment line\n\n" + text)
    assert bench.kernel_source_hash(root) == h0
    # code after the end-of-kernel marker is not hashed
    k.write_bytes(text + b"\nint unrelated_host_code = 1;\n")
    assert bench.kernel_source_hash(root) == h0
    # code before it is
    k.write_bytes(b"static int changed = 1;\n" + text)
    assert bench.kernel_source_hash(root) != h0


def test_profile_fields_keyed_on_the_hash(tmp_path):
    root = str(_tree(tmp_path))
    h = bench.kernel_source_hash(root)
    f = bench.profile_fields(os.path.join(root, "profiles", "blind_rotate_own_slot_gates888.md"))
    for key in ("kernel_source_sha256", "launch_shape", "gates", "cmux_per_gate", "warp_instructions"):
        assert key in f, key
    want = float(f["warp_instructions"]) / (float(f["gates"]) * float(f["cmux_per_gate"]))
    if f["kernel_source_sha256"] == h:  # the committed summary was taken on this code
        assert bench.measured_issue(int(f["launch_shape"]), root) == pytest.approx(want)
        assert bench.measured_issue(int(f["launch_shape"]) - 1, root) is None  # another launch shape
    assert bench.measured_issue(int(f["launch_shape"]), root, code_hash="0" * 64) is None
    assert bench.measured_traffic("eq32x4096", root, code_hash="0" * 64) is None
    assert bench.measured_traffic("no_such_workload", root) is None
    # a summary with the matching hash is read
    p = tmp_path / "profiles/blind_rotate_eq32x4096_dram.md"
    p.write_text(f"- kernel_source_sha256: {h}\n- dram_bytes_per_launch: 12345\n")
    assert bench.measured_traffic("eq32x4096", root) == 12345.0


def test_issue_ceiling_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "measured_issue", lambda shape, *a, **k: 20000.0 if shape == 8 else None)
    kt = {"blind_rotate_ms": 2000.0, "blind_rotate_launches": 4, "keyswitch_ms": 100.0, "gates": 100000}
    r = bench.roofline_of(kt, 2100.0, 148, None, None, None, 1, 1, shape=8, sm_mhz=2000.0)
    ic = r["issue_ceiling"]
    full = 148 * 4 * 2000e6 / (20000.0 * 630)
    assert ic["bootstraps_per_s_at_full_issue"] == pytest.approx(full)
    assert ic["achieved_bootstraps_per_s"] == pytest.approx(50000.0)
    assert ic["frac"] == pytest.approx(50000.0 / full)
    assert r["share_of_step"] == pytest.approx(2000.0 / 2100.0)
    assert r["keyswitch_ms_per_step"] == pytest.approx(100.0)
    # no capture for this shape, or no clock sample: no ceiling
    assert bench.roofline_of(kt, 2100.0, 148, None, None, None, 1, 1, shape=2, sm_mhz=2000.0)["issue_ceiling"] is None
    assert bench.roofline_of(kt, 2100.0, 148, None, None, None, 1, 1, shape=8, sm_mhz=None)["issue_ceiling"] is None
