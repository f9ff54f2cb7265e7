"""Host logic of bench.py that needs no GPU: the clock sampler keeps only the
samples taken inside the timed region (NVML's when present, else
nvidia-smi's), and the oracle timer of the reference arm and of
cpu_baseline reports a positive rate on a bounded sample."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _smi_line(t, clk, cap="Not Active", hw="Not Active"):
    return "%s, %d, 2070, 900.0, %s, Not Active, Not Active, %s" % (
        t.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3], clk, hw, cap)


def test_clock_sampler_keeps_the_timed_window_from_nvidia_smi():
    c = bench.ClockSampler(0)
    now = datetime.datetime.now()
    sec = lambda x: now + datetime.timedelta(seconds=x)
    c.lines = [_smi_line(sec(-1.0), 900), _smi_line(sec(0.1), 2070, cap="Active"), _smi_line(sec(0.2), 2050),
               _smi_line(sec(0.3), 2060), _smi_line(sec(3.0), 600, hw="Active"), "garbage line"]
    c.t0, c.t1 = now, sec(1.0)
    s = c.summary()
    assert s["source"] == "nvidia-smi" and s["samples"] == 3
    assert s["sm_mhz"] == 2060.0 and s["sm_min_mhz"] == 2050.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]          # the hw_slowdown sample lies outside the window


def test_clock_sampler_prefers_nvml_inside_the_window():
    c = bench.ClockSampler(0)
    c.p0, c.p1 = 10.0, 11.0
    c.nvml_max = 2070.0
    c.nvml_samples = [(9.0, 500.0, ["hw_slowdown"]), (10.2, 2070.0, []), (10.4, 2070.0, []),
                      (10.6, 2040.0, ["sw_power_cap"]), (10.8, None, []), (12.0, 700.0, [])]
    s = c.summary()
    assert s["source"] == "nvml" and s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_min_mhz"] == 2040.0 and s["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_samples_says_so():
    c = bench.ClockSampler(0)
    c.p0, c.p1 = 1.0, 2.0
    s = c.summary()
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"]


def test_oracle_timer_reports_a_bounded_sample():
    from oracle import oracle as O
    O.build()
    rate, sample = bench.time_oracle("cube8k", 2.0, max_steps=2)
    assert rate > 0 and "cube8k" in sample and sample.startswith(("1 ", "2 "))


def test_counter_record_hash_ignores_comments_only():
    a = "int f(int x) {  // one\n    return x + 1; /* two */\n}\n"
    b = "// header\nint f(int x) {\n\n    return   x + 1;\n}\n"
    c = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
    assert len(bench.kernel_source_sha()) == 16


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    """bench.py --impl reference launched as the scaling run launches it (two
    ranks through torch.distributed.run on 127.0.0.1): rank 0 times the
    oracle and prints one JSON line, the other rank exits 0 without output."""
    import json
    import socket
    import subprocess
    from oracle import oracle as O
    O.build()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "cube8k", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
