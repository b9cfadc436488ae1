"""Host-side arithmetic of bench.py (CPU): the roofline counts, the traffic
ratios read from the profile summaries, and the step's partition choice."""
import hashlib
import os
import types

import numpy as np
import pytest

import bench
import synth


def _w(k=40):
    return types.SimpleNamespace(k=k, p=1, q=2, grid="equal", m=10, n=20)


def test_gram_flop_counts():
    shapes = [(3, 10), (5, 7)]
    # both triangles: 2 L s^2; distinct entries: L s (s + 1)
    assert bench.gram_flops(shapes) == 2 * 10 * 9 + 2 * 7 * 25
    assert bench.gram_flops_min(shapes) == 10 * 3 * 4 + 7 * 5 * 6
    # the distinct count is half the full one plus the diagonal
    s, L = 100, 300
    assert bench.gram_flops_min([(s, L)]) == bench.gram_flops([(s, L)]) / 2 + L * s


def test_panel_roofline_counts_every_product():
    w = _w(k=40)
    shapes = [(100, 500), (20, 30)]
    rep = {"products": [3, 2], "launches": 4}
    peaks = {"hbm_gbs": 1000.0, "bf16_tflops": 2000.0}
    r = bench.panel_roofline(w, shapes, rep, filter_ms=2.0, peaks=peaks,
                             peak_kind="measured")
    b1, b2 = 64, 20             # k + 20 -> 64 columns; a block of 20 rows
    want = 3 * (4 * 100 ** 2 + 8 * 100 * b1) + 2 * (4 * 20 ** 2 + 8 * 20 * b2)
    assert r["algorithmic_bytes"] == want
    assert r["products"] == 5 and r["launches"] == 4
    assert r["achieved"] == pytest.approx(want / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    # a schedule's oversample sets the width: k = 10 + 4 -> 16 columns
    r16 = bench.panel_roofline(_w(k=10), [(100, 500)], {"products": [1]},
                               1.0, peaks, "measured", oversample=4)
    assert r16["algorithmic_bytes"] == 4 * 100 ** 2 + 8 * 100 * 16


def test_step_roofline_takes_the_binding_term():
    w = _w(k=4)
    r = types.SimpleNamespace(u_train=np.zeros(1000), u_test=np.zeros(100))
    peaks = {"hbm_gbs": 1.0, "bf16_tflops": 1e-6}   # 1 GB/s, 1 MFLOP/s
    shapes = [(2, 3)]
    out = bench.step_roofline(w, r, shapes, 4, 4, step_s=10.0, peaks=peaks,
                              peak_kind="measured")
    assert out["roofline_ms"] == pytest.approx(max(out["tensor_ms"],
                                                   out["hbm_ms"]))
    assert out["frac"] == pytest.approx(out["roofline_ms"] / 1e4)
    # bytes as the step roofline counts them: 12 a training rating,
    # 4 + 2 + 4 a dense cell (written, read by the bf16 Gram, read by the
    # projection), 12 + 8 k a query
    assert out["algorithmic_bytes"] == 12 * 1000 + 6 * 10 + 100 * (12 + 32)


def test_traffic_ratio_only_for_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "csrc"
    prof = tmp_path / "profiles"
    src.mkdir()
    prof.mkdir()
    (src / "k.cu").write_text("kernel source\n")
    sha = hashlib.sha256(b"kernel source\n").hexdigest()
    (prof / "k_small.md").write_text(
        "text\n\ntraffic_ratio: k_a 1.25 %s\n\nmore\n" % sha)
    monkeypatch.setattr(bench, "CSRC", str(src))
    monkeypatch.setattr(bench, "PROFILES", str(prof))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", {"k_a": "k.cu"})
    assert bench.profiled_traffic_ratio("k_a") == 1.25
    assert bench.profiled_traffic_ratio("k_other") is None
    (src / "k.cu").write_text("kernel source, changed\n")
    assert bench.profiled_traffic_ratio("k_a") is None


def test_committed_ratios_match_their_sources():
    """Every traffic_ratio line under profiles/ names a kernel bench.py
    knows, and the panel products' ratio belongs to the current source (a
    stale line would make the bench report no traffic)."""
    found = {}
    for name in os.listdir(bench.PROFILES):
        with open(os.path.join(bench.PROFILES, name)) as f:
            for line in f:
                parts = line.strip().split()
                if parts and parts[0] == "traffic_ratio:":
                    assert parts[1] in bench.KERNEL_SOURCES, line
                    found[parts[1]] = float(parts[2])
    assert "k_gpanel_tc" in found and "k_gram_bf16" in found
    assert bench.profiled_traffic_ratio("k_gpanel_tc") == found["k_gpanel_tc"]
    assert bench.profiled_traffic_ratio("k_gram_bf16") == found["k_gram_bf16"]


def test_step_partition_picks_the_call():
    calls = []

    class Ctx:
        def partition_quantile(self, *a):
            calls.append(("quantile", a))

        def partition(self, *a):
            calls.append(("equal", a))

    bench.step_partition(Ctx(), synth.UNEVEN, "u", "i", "x")
    bench.step_partition(Ctx(), synth.MEDIUM, "u", "i", "x")
    assert [c[0] for c in calls] == ["quantile", "equal"]
    w = synth.UNEVEN
    assert calls[0][1] == (w.m, w.n, "u", "i", "x", w.p, w.q)


def test_clock_sampler_parses_nvidia_smi_lines(tmp_path, monkeypatch):
    """The sampler reads nvidia-smi's CSV: median SM clock, the largest
    maximum, and every throttle reason seen active; with no samples (no
    nvidia-smi, or a run shorter than its first line) it reports None."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!/bin/sh\n"
        "echo '0, 1900, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, Active'\n"
        "echo '0, 2070, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
        "echo '0, 2000, 2070, 905.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
        "echo 'garbage line'\n"
        "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    import time
    deadline = time.time() + 10
    while time.time() < deadline:
        if os.path.exists(c.path) and open(c.path).read().count("\n") >= 4:
            break
        time.sleep(0.05)
    got = c.stop()
    assert got == {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "samples": 3,
                   "reasons": ["sw_power_cap"]}
    monkeypatch.setenv("PATH", str(tmp_path / "none"))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() is None
