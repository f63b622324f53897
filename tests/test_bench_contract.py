"""bench.py's reference arm (the FP64 oracle on the host cores) runs without a GPU: its
JSON line must carry the contract's keys, with the oracle described as the baseline."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "3",
           "--n", "256", "--ref-target-s", "0.02"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_profile_traffic_only_for_the_current_kernel_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu summary only while that summary's
    source hash matches the kernel file; a stale or incomplete summary gives null."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1806_01430_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() {}\n")
    sha = hashlib.sha256((csrc / "k.cu").read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = tmp_path / "profiles" / "k.md"
    prof.write_text(f"# k\n\ntraffic_bytes_per_launch: 123456\nsource_sha256: {sha}\n")
    assert bench.profile_traffic("k.cu", "k.md") == 123456.0
    (csrc / "k.cu").write_text("__global__ void k() { }\n")  # the kernel changed since the capture
    assert bench.profile_traffic("k.cu", "k.md") is None
    prof.write_text("# k\n\ntraffic_bytes_per_launch: 123456\n")  # no hash line
    assert bench.profile_traffic("k.cu", "k.md") is None
    assert bench.profile_traffic("k.cu", "missing.md") is None


def test_committed_profiles_name_their_command_and_source():
    """Every committed ncu summary gives the command that made it; those the bench reads carry
    a traffic figure and the hash of the kernel source they were taken on."""
    import re
    pdir = os.path.join(ROOT, "profiles")
    names = sorted(os.listdir(pdir))
    assert names
    for nm in names:
        text = open(os.path.join(pdir, nm)).read()
        assert nm.endswith((".md", ".txt")), nm
        assert "ncu " in text and "--clock-control none" in text, nm
        if re.search(r"traffic_bytes_per_launch:", text):
            assert re.search(r"source_sha256:\s*[0-9a-f]{64}", text), nm


def test_clock_summary_of_samples_in_the_timed_window():
    """The clock record beside a bench number: median SM clock, max clock and the throttle
    reasons seen during [t0, t1] only, from nvidia-smi's CSV lines (malformed lines skipped)."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    row = "0, {sm}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {cap}"
    c.lines = [(0.5, row.format(sm=1200, hw="Active", cap="Not Active")),   # before the window
               (1.0, row.format(sm=1980, hw="Not Active", cap="Active")),
               (1.2, row.format(sm=2010, hw="Not Active", cap="Not Active")),
               (1.4, "0, [N/A], 2070"),                                      # malformed
               (1.6, row.format(sm=1950, hw="Not Active", cap="Active")),
               (3.0, row.format(sm=900, hw="Active", cap="Not Active"))]     # after it
    s = c.summary(1.0, 2.0)
    assert s == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s_all = c.summary()
    assert s_all["samples"] == 5 and s_all["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.Clocks(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_pass_bytes_match_the_per_element_figures():
    """Algorithmic bytes of a memory-bound pass: INIT 4 B per element of each output, scale-add
    12 B (two reads, one write), transpose 8 B, row sums 4 B per element plus the vector; a
    fused pass does not count an intermediate that nothing after it reads."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    n = 96
    six = W.six_loop(n, 1, outputs=("C", "r", "f"))
    e = n * n
    assert bench.group_bytes(six, [0]) == 3 * 4 * e            # A, B, C written
    assert bench.group_bytes(six, [2]) == 12 * e                # D = C + 2A
    assert bench.group_bytes(six, [3]) == 8 * e                 # E = D^T
    assert bench.group_bytes(six, [4]) == 4 * e + 4 * n         # r = E 1
    assert bench.group_bytes(six, [5]) == 4 * e + 8             # f = ||E|| (binary64 out)
    assert bench.group_bytes(six, [2, 3]) == 12 * e             # D stays inside the pass
    keep_d = W.six_loop(n, 1, outputs=("D", "r", "f"))
    assert bench.group_bytes(keep_d, [2, 3]) == 16 * e          # unless D is an output
    m, k = 64, 32
    tw = W.twelve_loop(m, k, 2)
    ew = [i for i, lp in enumerate(tw.loops) if lp.kind in (W.RELU, W.AXPY, W.SQUARE)][1:]  # L6..L9
    # F = max(E,0), G = E - 0.5F, H = G.G, P = H + 0.25D as one pass: reads E and D, writes P
    assert bench.group_bytes(tw, ew) == 3 * 4 * m * m
