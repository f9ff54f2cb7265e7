"""Benchmark of the GB300 MLS-MPM step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--workload block1m|slab30k|slab30k_sdf|block8m|cube8k] [--substeps S]
                [--pipeline fused|split]

A benchmark step is one call of mpm_step with S sub-steps (default 25, one
frame of the paper's simulation loop: 25 sub-steps per rendered frame) with
the scripted tool pose set before it.  The metric is particle-steps/s:
particles x sub-steps / time, summed over ranks.  `value` times the frames
with the state resident on the GPU (CUDA events on the simulation stream,
L2 flushed by a 256 MB write between frames); `e2e` times the same frames
through the C ABI with host buffers: the tool pose goes in from the host and
every frame's particle positions come back to pinned host memory, streamed
with mpm_read_particles_async so that each copy overlaps the next frame's
sub-steps (`e2e.value_with_synchronous_readback` waits for every copy).

--gpus N > 1 (under torchrun) runs N independent replicas of the scene, one
per GPU (the single-scene step does not shard; see the design notes), and
reports the aggregate over ranks from the slowest rank's time.

--impl reference times the FP64 CPU oracle (oracle/) on the host cores on a
bounded sample of the same workload; there is no other implementation of
this method to compare with.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_01181_gb300 import scenes  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="block1m", choices=sorted(scenes.SCENES))
    ap.add_argument("--substeps", type=int, default=25)
    ap.add_argument("--pipeline", default="fused", choices=["fused", "split"])
    ap.add_argument("--no-secondary", action="store_true", help="skip the 30K slab line")
    ap.add_argument("--no-differentiable", action="store_true", help="skip the differentiable-rollout line")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default fused-kernel configuration")
    ap.add_argument("--no-surface", action="store_true", help="skip the surface-extraction line")
    ap.add_argument("--kernel-config", type=int, default=None,
                    help="fused-kernel configuration to use instead of autotuning (MPM_KERNEL_*)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-environment measurement")
    ap.add_argument("--batch-envs", type=int, default=256)
    ap.add_argument("--no-sweep", action="store_true", help="skip the 8M block and the split-pipeline sub-lines")
    return ap.parse_args()


# --------------------------------------------------------------- helpers

def _code_only(text):
    """C/CUDA source without comments and blank lines, whitespace runs folded."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(" ".join(ln.split()) for ln in text.splitlines() if ln.strip())


def kernel_source_sha():
    """Hash of the fused kernel's code (comments excluded), which the ncu
    counters in profiles/traffic.json are tied to."""
    h = hashlib.sha256()
    for f in ("kernel_fused.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2402_01181_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(PEAKS_FILE) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class _Nvml:
    """Read-only NVML queries (SM clock, its maximum, clock-event reasons)
    through libnvidia-ml, the library nvidia-smi itself reads."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        import ctypes as ct
        self.ct = ct
        self.lib = ct.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ct.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ct.c_uint(index), ct.byref(self.h)) != 0:
            raise RuntimeError("no NVML device %d" % index)
        self.get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def _clock(self, fn):
        v = self.ct.c_uint(0)
        return float(v.value) if fn(self.h, 1, self.ct.byref(v)) == 0 else None     # 1: the SM clock domain

    def sm_clock(self):
        return self._clock(self.lib.nvmlDeviceGetClockInfo)

    def sm_max_clock(self):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def reasons(self):
        r = self.ct.c_ulonglong(0)
        if self.get_reasons(self.h, self.ct.byref(r)) != 0:
            return []
        return [nm for bit, nm in self.REASONS.items() if r.value & bit]


class ClockSampler:
    """SM clock and clock-event reasons during the timed region.  NVML is
    polled every 5 ms on a background thread, and nvidia-smi samples every
    50 ms alongside it; both run from before the warm-up to after the timed
    region, and summary() keeps the samples taken between mark_start() and
    mark_end() (NVML's if it loaded, else nvidia-smi's)."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50
    NVML_INTERVAL_S = 0.005

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.nvml = None
        self.nvml_samples = []
        self.stop = threading.Event()
        self.t0 = self.t1 = None
        self.p0 = self.p1 = None

    def mark_start(self):
        self.t0 = datetime.datetime.now()
        self.p0 = time.perf_counter()

    def mark_end(self):
        self.t1 = datetime.datetime.now()
        self.p1 = time.perf_counter()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        try:
            self.nvml = _Nvml(self.dev)
            self.nvml_max = self.nvml.sm_max_clock()
            self.tn = threading.Thread(target=self._poll, daemon=True)
            self.tn.start()
        except Exception:
            self.nvml = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def _poll(self):
        while not self.stop.is_set():
            self.nvml_samples.append((time.perf_counter(), self.nvml.sm_clock(), self.nvml.reasons()))
            time.sleep(self.NVML_INTERVAL_S)

    def __exit__(self, *a):
        self.stop.set()
        if self.nvml is not None:
            self.tn.join(timeout=2)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def _smi_samples(self):
        out = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            ts = None
            for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
                try:
                    ts = datetime.datetime.strptime(parts[0], fmt)
                    break
                except ValueError:
                    pass
            try:
                clk, cmax = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if ts is None or (self.t0 is not None and not (self.t0 <= ts <= (self.t1 or ts))):
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            out.append((clk, cmax, [nm for nm, val in zip(names, parts[4:8]) if val.lower() == "active"]))
        return out

    def summary(self):
        smi = self._smi_samples()
        nv = [(c, self.nvml_max, r) for t, c, r in self.nvml_samples
              if c is not None and (self.p0 is None or self.p0 <= t <= (self.p1 or t))]
        src, use = ("nvml", nv) if nv else ("nvidia-smi", smi)
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = sorted({nm for _, _, r in use for nm in r})
        return {"sm_mhz": float(np.median([c for c, _, _ in use])), "sm_min_mhz": float(min(c for c, _, _ in use)),
                "sm_max_mhz": use[-1][1], "reasons": reasons, "samples": len(use), "source": src,
                "window": "timed region", "nvidia_smi_samples": len(smi)}


# ------------------------------------------------------------ GPU workload

def run_gpu_workload(name, args, rank, device, barrier, max_over_ranks, with_e2e=True, with_roofline=True,
                     steps=None):
    import torch
    from paper_2402_01181_gb300 import mpm
    steps = steps or args.steps
    S = args.substeps
    from paper_2402_01181_gb300 import dist as D
    sc = scenes.SCENES[name](seed=D.replica_seed(rank))
    pipe = mpm.MPM_PIPELINE_FUSED if args.pipeline == "fused" else mpm.MPM_PIPELINE_SPLIT
    stream = torch.cuda.current_stream(device)
    sim = mpm.sim_from_scene(sc, pipeline=pipe)
    tool_frames = [(t, tool) for t, tool in enumerate(sc.tools)]
    s_next = [0]
    tuning = None
    if pipe == mpm.MPM_PIPELINE_FUSED and args.kernel_config is not None:
        sim.set_kernel_config(args.kernel_config)
        tuning = {"config": args.kernel_config, "name": mpm.KERNEL_CONFIG_NAMES[args.kernel_config],
                  "ms_per_step_by_config": None}
    elif pipe == mpm.MPM_PIPELINE_FUSED and not args.no_autotune:
        best, times = sim.autotune(S)          # restores the state it starts from
        tuning = {"config": best, "name": mpm.KERNEL_CONFIG_NAMES[best], "ms_per_step_by_config": times}

    def frame():
        s = s_next[0]
        for t, tool in tool_frames:
            sim.set_tool(t, tool.pose(s + S - 1), tool.shape, tool.field)
        sim.step(S)
        s_next[0] = s + S

    grid = sim.read_grid()
    active_nodes = int((grid[..., 0] > 0).sum())
    del grid
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(device) as clk:
        for _ in range(args.warmup):
            frame()
        sim.synchronize()
        barrier()
        torch.cuda.synchronize(device)
        clk.mark_start()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            frame()
            ev[i][1].record(stream)
        torch.cuda.synchronize(device)
        clk.mark_end()
    barrier()
    st = sim.status()
    if st != mpm.MPM_OK:
        raise RuntimeError("device error after timed region: %s" % mpm.mpm_last_error())
    frame_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = max_over_ranks(sum(frame_ms))
    res = {"n": sc.n, "n_grid": sc.n_grid, "frame_ms": frame_ms, "t_ms": t_ms, "clocks": clk.summary(),
           "active_nodes": active_nodes, "steps": steps, "tuning": tuning}

    if with_e2e:
        # end to end through the C ABI with host buffers
        import ctypes as ct
        host_x = [torch.empty((sc.n, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        xp = [ct.c_void_p(h.data_ptr()) for h in host_x]
        # every frame's positions read back with the synchronous call ...
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            frame()
            mpm.check(mpm.mpm_read_particles(sim.h, xp[0], None, None, None, 0))
        res["t_e2e_sync_ms"] = max_over_ranks((time.perf_counter() - t0) * 1e3)
        # ... and streamed: each frame's copy overlaps the next frame's sub-steps
        barrier()
        t0 = time.perf_counter()
        for i in range(steps):
            frame()
            mpm.check(mpm.mpm_read_particles_async(sim.h, xp[i & 1], None, None, None))
        mpm.check(mpm.mpm_wait_read(sim.h))
        mpm.check(mpm.mpm_synchronize(sim.h))
        t_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3)
        res["t_e2e_ms"] = t_e2e
        ntools = len(sc.tools)
        res["h2d"] = 112 * mpm.MPM_MAX_TOOLS * S if ntools else 0     # tool frames of the call
        res["d2h"] = sc.n * 12 + 4                                     # positions + status word
    sim.close()
    return res


def run_batched(args, rank, device, barrier, max_over_ranks, steps=6, loop_steps=2):
    """Batched environments: n_envs independent slab scenes
    of 5K-40K particles on their own 64^3 grids, stepped by one handle (one
    fused launch per sub-step over all environments), against the per-env
    loop of n_envs single-environment handles on the same GPU.  Metric:
    env-steps/s = environments x sub-steps / time."""
    import torch
    from paper_2402_01181_gb300 import dist as D
    from paper_2402_01181_gb300 import mpm
    S = args.substeps
    envs = scenes.batch_envs(args.batch_envs, seed=D.replica_seed(rank))
    ne = len(envs)
    total = sum(e.n for e in envs)
    stream = torch.cuda.current_stream(device)
    cfg = mpm.make_config(64, envs[0].dt, 1e4, 0.3, 1e3, friction=0.3, n_envs=ne, max_particles=total)
    sim = mpm.Sim(cfg)
    for i, sc in enumerate(envs):
        sim.set_env_material(i, sc.E, sc.nu, sc.rho)
    sim.load_batch([sc.x for sc in envs], [sc.particle_volume for sc in envs])
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(-1), sc.tools[0].shape)
    tuning = None
    if not args.no_autotune:
        best, times = sim.autotune(S)
        tuning = {"config": best, "name": mpm.KERNEL_CONFIG_NAMES[best], "ms_per_step_by_config": times}
    s_next = [0]

    def set_tools():
        s = s_next[0]
        for i, sc in enumerate(envs):
            sim.set_env_tool(i, 0, sc.tools[0].pose(s + S - 1), sc.tools[0].shape)
        s_next[0] = s + S

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    for _ in range(args.warmup):
        set_tools()
        sim.step(S)
    sim.synchronize()
    barrier()
    ms = 0.0
    for _ in range(steps):
        set_tools()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(S)
        b.record(stream)
        torch.cuda.synchronize(device)
        ms += a.elapsed_time(b)
    if sim.status() != mpm.MPM_OK:
        raise RuntimeError("device error in the batched run: %s" % mpm.mpm_last_error())
    sim.close()
    t_batched = max_over_ranks(ms)
    # the per-env loop: one handle per environment, stepped one after another
    sims = []
    for sc in envs:
        c1 = mpm.make_config(64, sc.dt, sc.E, sc.nu, sc.rho, friction=0.3, max_particles=sc.n)
        si = mpm.Sim(c1)
        si.load(sc.x, sc.particle_volume)
        si.set_tool(0, sc.tools[0].pose(-1), sc.tools[0].shape)
        sims.append(si)
    s_loop = [0]

    def loop_frame():
        s = s_loop[0]
        for si, sc in zip(sims, envs):
            si.set_tool(0, sc.tools[0].pose(s + S - 1), sc.tools[0].shape)
            si.step(S)
        s_loop[0] = s + S

    loop_frame()
    torch.cuda.synchronize(device)
    barrier()
    ms_loop = 0.0
    for _ in range(loop_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        loop_frame()
        b.record(stream)
        torch.cuda.synchronize(device)
        ms_loop += a.elapsed_time(b)
    for si in sims:
        si.close()
    t_loop = max_over_ranks(ms_loop)
    world = D.env()[0]
    env_steps = ne * S * steps * world / (t_batched / 1e3)
    loop_env_steps = ne * S * loop_steps * world / (t_loop / 1e3)
    return {"workload": "batch%d" % ne, "n_envs": ne, "particles": total, "n_grid": 64,
            "env_steps_per_s": env_steps, "particle_steps_per_s": total * S * steps * world / (t_batched / 1e3),
            "ms_per_step": t_batched / steps, "loop_env_steps_per_s": loop_env_steps,
            "loop_ms_per_step": t_loop / loop_steps, "speedup_vs_loop": env_steps / loop_env_steps,
            "gpu_launches_per_step": S, "tuning": tuning}


def run_differentiable(args, rank, device, barrier, max_over_ranks, reps=2):
    """The differentiable rollout: the 30K slab over 500
    sub-steps with checkpoints every 50, loss = mean |x(T) - target|^2 with
    a target rolled out on the GPU with E = 1.2e4, nu = 0.33 and shifted
    poses.  On the fused pipeline (the product path) and, for comparison, on
    the unsorted split pipeline: the recorded forward pass (mpm_tape_record)
    and the reverse pass (mpm_tape_backward, which recomputes every segment),
    against the plain fused forward of the same 500 sub-steps (20 calls of
    25 sub-steps, as the benchmark steps the slab)."""
    import torch
    from paper_2402_01181_gb300 import dist as D
    from paper_2402_01181_gb300 import mpm
    case = scenes.slab30k_diff(seed=D.replica_seed(rank))
    sc = case.scene
    K = case.poses.shape[0]
    stream = torch.cuda.current_stream(device)

    def fresh(E, nu, pipe):
        si = mpm.sim_from_scene(sc, pipeline=pipe, load=False)
        si.set_env_material(0, E, nu, sc.rho)
        si.load(sc.x, sc.particle_volume)
        si.set_tool(0, case.pose_init[0], sc.tools[0].shape)
        return si

    tgt = fresh(case.target_E, case.target_nu, mpm.MPM_PIPELINE_FUSED)
    tgt.tape_record(case.target_poses, case.checkpoint)
    target = torch.tensor(tgt.read()["x"], device=device)
    tgt.close()

    def timed(pipe):
        fwd, bwd, res = [], [], {}
        for r in range(reps + 1):
            si = fresh(sc.E, sc.nu, pipe)
            a, b, c0, c = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            barrier()
            a.record(stream)
            si.tape_record(case.poses, case.checkpoint)
            b.record(stream)
            x = torch.empty((sc.n, 3), dtype=torch.float32, device=device)
            si.read_device(x=x)
            loss = float(((x - target) ** 2).sum(dim=1).mean())
            gx = 2.0 * (x - target) / sc.n
            torch.cuda.synchronize(device)
            c0.record(stream)
            g = si.tape_backward(gx)
            c.record(stream)
            torch.cuda.synchronize(device)
            si.close()
            if r == 0:
                continue                      # warm-up
            fwd.append(a.elapsed_time(b))
            bwd.append(c0.elapsed_time(c))
            res = {"loss": loss, "dL_dE": g["E"], "dL_dnu": g["nu"], "max_abs_dL_dpose": float(abs(g["poses"]).max())}
        return max_over_ranks(min(fwd)), max_over_ranks(min(bwd)), res

    f, bk, res = timed(mpm.MPM_PIPELINE_FUSED)
    fs, bks, _ = timed(mpm.MPM_PIPELINE_SPLIT)
    # the plain fused forward of the same sub-steps: 20 calls of 25
    plain = []
    S = 25
    for r in range(reps + 1):
        sp = fresh(sc.E, sc.nu, mpm.MPM_PIPELINE_FUSED)
        d, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        d.record(stream)
        for k0 in range(0, K, S):
            sp.set_tool(0, case.poses[k0 + S - 1, 0], sc.tools[0].shape)
            sp.step(S)
        e.record(stream)
        torch.cuda.synchronize(device)
        sp.close()
        if r > 0:
            plain.append(d.elapsed_time(e))
    pl = max_over_ranks(min(plain))
    res.update({"workload": "slab30k_diff", "particles": sc.n, "substeps": K, "checkpoint_every": case.checkpoint,
                "pipeline": "fused", "forward_record_ms": f, "backward_ms": bk, "fused_forward_ms": pl,
                "backward_over_fused_forward": bk / pl, "backward_over_recorded_forward": bk / f,
                "split": {"forward_record_ms": fs, "backward_ms": bks, "backward_over_fused_forward": bks / pl},
                "note": "min over %d repetitions; the backward includes the segment recomputation" % reps})
    return res


def run_surface(args, rank, device, barrier, max_over_ranks, reps=10):
    """Surface extraction (the renderer's Marching Cubes step) of the 1M
    block after one 25-sub-step frame: the triangles of density 1/2 written
    to device memory, timed with CUDA events (counts, scan, total readback,
    triangles)."""
    import ctypes as ct
    import torch
    from paper_2402_01181_gb300 import dist as D
    from paper_2402_01181_gb300 import mpm
    sc = scenes.block1m(seed=D.replica_seed(rank))
    sim = mpm.sim_from_scene(sc)
    tool = sc.tools[0]
    sim.set_tool(0, tool.pose(24), tool.shape)
    sim.step(25)
    n_tri = ct.c_int64()
    mpm.check(mpm.mpm_extract_surface(sim.h, 0, 0.5, None, 0, ct.byref(n_tri), 0))
    T = n_tri.value
    out = torch.empty((max(T, 1), 9), dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    times = []
    for r in range(reps + 2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mpm.check(mpm.mpm_extract_surface(sim.h, 0, 0.5, ct.c_void_p(out.data_ptr()), T, ct.byref(n_tri), 1))
        b.record(stream)
        torch.cuda.synchronize(device)
        if r >= 2:
            times.append(a.elapsed_time(b))
    sim.close()
    ms = max_over_ranks(sorted(times)[len(times) // 2])
    n = sc.n_grid
    cells = (n - 1) ** 3
    # algorithmic bytes: the node masses read by both passes (4 B per node
    # each), the per-cell counts written, scanned and read (about 16 B per
    # cell), and the triangles written (36 B each)
    algo = 2 * 4 * n ** 3 + 16 * cells + 36 * T
    return {"workload": "block1m surface", "n_grid": n, "triangles": T, "ms": ms,
            "triangles_per_s": T / (ms / 1e3), "algorithmic_bytes": algo,
            "achieved_gbs": algo / (ms / 1e3) / 1e9, "note": "median of %d; includes one 4-byte readback" % reps}


def survey_bytes_per_particle_step(n, active_nodes):
    """Algorithmic DRAM traffic per particle-step of the method as the
    benchmark plan states it: the persistent FP32 state x, v, A, F (24 floats,
    96 B) read once and written once (192 B), plus 72 B per active grid node
    (clear 16, P2G result 16, grid read 16, velocity write 12, G2P read 12)."""
    return 192.0 + 72.0 * active_nodes / n


def cpu_description():
    """CPU model and the number of online cores of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    import platform
    return {"cpu_model": model or platform.machine(), "nproc": os.cpu_count(), "arch": platform.machine()}


def algorithmic_bytes_per_particle_step(n, active_nodes, S):
    """Minimum DRAM traffic of one fused sub-step, per particle: the particle
    state is read and written once (x, id: 16 B; F: 36 B; twice = 104 B); each
    active grid node is read once (16 B), accumulated into once (16 B) and
    cleared once (16 B); v and C (48 B) are written once per call."""
    return 104.0 + 48.0 * active_nodes / n + 48.0 / S


# --------------------------------------------------------------- oracle arm

def time_oracle(name, budget_s, rank_seed=0, max_steps=50):
    """Time the FP64 oracle on the workload; returns (particle-steps/s, sample)."""
    from oracle import oracle as O
    sc = scenes.SCENES[name](seed=rank_seed)
    prm = O.OracleParams.from_scene(sc)
    st = O.State(sc.x, sc.v, sc.C, sc.F)
    done, t0 = 0, time.perf_counter()
    while done < max_steps:
        frames, nt = O.frames_for_steps(sc.tools, done, 1, sc.dt, 1)
        O.run(prm, st, 1, frames, nt)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return sc.n * done / el, "%d sub-steps of the full %s workload (%d particles, %d^3 grid)" % (
        done, name, sc.n, sc.n_grid)


def time_oracle_adjoint(substeps=20, checkpoint=10):
    """Time the FP64 oracle's forward rollout and its reverse mode on the first
    sub-steps of the differentiable workload (the 30K slab, loss on the final
    positions); returns particle-steps/s of each and the sample."""
    from oracle import oracle as O
    case = scenes.slab30k_diff(steps=substeps, checkpoint=checkpoint)
    sc = case.scene
    prm = O.OracleParams.from_scene(sc)
    st0 = O.State(sc.x)
    t0 = time.perf_counter()
    st = st0.copy()
    fr, nt = O.rollout_frames(sc.tools, case.pose_init, case.poses, prm.dt)
    O.run(prm, st, substeps, fr, nt)
    t_fwd = time.perf_counter() - t0
    target = st.x + 1e-5
    t0 = time.perf_counter()
    O.rollout_loss_and_gradients(prm, st0, sc.tools, case.pose_init, case.poses, target, checkpoint=checkpoint)
    t_all = time.perf_counter() - t0
    units = sc.n * substeps
    return {"forward_particle_steps_per_s": units / t_fwd,
            "backward_particle_steps_per_s": units / max(t_all - t_fwd, 1e-9),
            "backward_over_forward": (t_all - t_fwd) / t_fwd, "cores": 1,
            "sample": "%d sub-steps of the differentiable workload (%d particles), checkpoints every %d; the "
                      "backward includes the recomputation of the segments" % (substeps, sc.n, checkpoint)}


def time_oracle_configs():
    """The FP64 oracle (one core) on bounded samples of the other benchmark
    workloads: particle-steps/s per workload, and env-steps/s of one batched
    environment of the mean size."""
    out = {}
    for name, budget, steps in (("cube8k", 3.0, 50), ("slab30k", 3.0, 50), ("block8m", 4.0, 1)):
        v, sample = time_oracle(name, budget, max_steps=steps)
        out[name] = {"particle_steps_per_s": v, "sample": sample}
    from oracle import oracle as O
    envs = scenes.batch_envs(256, seed=0)
    mean = float(np.mean([e.n for e in envs]))
    env = min(envs, key=lambda e: abs(e.n - mean))
    prm = O.OracleParams.from_scene(env)
    st = O.State(env.x)
    t0, done = time.perf_counter(), 0
    while done < 20 and time.perf_counter() - t0 < 3.0:
        frames, nt = O.frames_for_steps(env.tools, done, 1, env.dt, 1)
        O.run(prm, st, 1, frames, nt)
        done += 1
    el = time.perf_counter() - t0
    out["batch256"] = {"env_steps_per_s": done / el, "particle_steps_per_s": env.n * done / el,
                       "sample": "%d sub-steps of one batched environment of %d particles (the mean is %.0f)"
                                 % (done, env.n, mean)}
    return out


def reference_main(args):
    from paper_2402_01181_gb300 import dist as D
    world, rank, local = D.env()
    if rank != 0:          # under torchrun only rank 0 times the oracle; the others exit at once
        return
    budget = 8.0
    vals = []
    for _ in range(args.warmup):
        time_oracle(args.workload, budget / 4, max_steps=1)
    t0 = time.perf_counter()
    sample = ""
    for _ in range(args.steps):      # one full-size sub-step per step (about 0.5 s for block1m)
        v, sample = time_oracle(args.workload, budget, max_steps=1)
        vals.append(v)
    el = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "impl": "FP64 single-threaded C oracle"},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample, **cpu_description()},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ main

def main():
    args = parse()
    if args.impl == "reference":
        return reference_main(args)
    import torch
    from paper_2402_01181_gb300 import dist as D
    world, rank, local = D.env()
    device = local if torch.cuda.device_count() > local else 0
    torch.cuda.set_device(device)
    ranks = D.Ranks(device=device)
    barrier, max_over_ranks = ranks.barrier, ranks.max

    import __graft_entry__ as ge
    ge.build()
    S = args.substeps
    main_res = run_gpu_workload(args.workload, args, rank, device, barrier, max_over_ranks)
    n_units = main_res["n"] * S * args.steps * world
    value = n_units / (main_res["t_ms"] / 1e3)
    ms_per_step = main_res["t_ms"] / args.steps
    second = None
    if not args.no_secondary and args.workload != "slab30k":
        r2 = run_gpu_workload("slab30k", args, rank, device, barrier, max_over_ranks, with_e2e=True,
                              steps=max(args.steps, 20))
        second = {"workload": "slab30k", "n_particles": r2["n"], "n_grid": r2["n_grid"], "tuning": r2["tuning"],
                  "value": r2["n"] * S * r2["steps"] * world / (r2["t_ms"] / 1e3),
                  "ms_per_step": r2["t_ms"] / r2["steps"],
                  "e2e": r2["n"] * S * r2["steps"] * world / (r2["t_e2e_ms"] / 1e3)}
        # the same slab with the tool as a sampled 256^3 distance field
        r3 = run_gpu_workload("slab30k_sdf", args, rank, device, barrier, max_over_ranks, with_e2e=False,
                              steps=max(args.steps, 20))
        second["sampled_field"] = {"workload": "slab30k_sdf", "field_res": 256,
                                   "value": r3["n"] * S * r3["steps"] * world / (r3["t_ms"] / 1e3),
                                   "ms_per_step": r3["t_ms"] / r3["steps"]}

    # the roofline sweep of the benchmark plan: the 8M block (256^3 grid), and
    # sorted (fused) against unsorted (split) P2G on both blocks
    sweep = None
    if not args.no_sweep and args.workload == "block1m" and args.pipeline == "fused":
        sweep = {}
        split_args = argparse.Namespace(**{**vars(args), "pipeline": "split"})
        for wl, a, key in (("cube8k", args, "cube8k_fused"), ("block8m", args, "block8m_fused"),
                           ("block1m", split_args, "block1m_split"), ("block8m", split_args, "block8m_split")):
            steps = 10 if wl == "block8m" else args.steps
            r = run_gpu_workload(wl, a, rank, device, barrier, max_over_ranks, with_e2e=False, steps=steps)
            n_units_w = r["n"] * S * r["steps"] * world
            bpp_w = survey_bytes_per_particle_step(r["n"], r["active_nodes"])
            launch_w = r["t_ms"] / (r["steps"] * S)
            sweep[key] = {"workload": wl, "pipeline": a.pipeline, "n_particles": r["n"], "n_grid": r["n_grid"],
                          "value": n_units_w / (r["t_ms"] / 1e3), "unit": "particle-steps/s",
                          "us_per_substep": launch_w * 1e3, "tuning": r["tuning"], "clocks": r["clocks"],
                          "roofline_frac": bpp_w * r["n"] / (launch_w / 1e3) / 1e9 / measured_peak()[0]}
        for wl in ("block1m", "block8m"):
            fused_v = value if wl == "block1m" else sweep["block8m_fused"]["value"]
            sweep["%s_sorted_over_unsorted" % wl] = fused_v / sweep["%s_split" % wl]["value"]

    batched = None
    if not args.no_batched:
        batched = run_batched(args, rank, device, barrier, max_over_ranks)
    differentiable = None
    if not args.no_differentiable:
        differentiable = run_differentiable(args, rank, device, barrier, max_over_ranks)
    surface = None
    if not args.no_surface:
        surface = run_surface(args, rank, device, barrier, max_over_ranks)

    if rank != 0:
        ranks.close()
        return

    peak, peak_kind = measured_peak()
    bpp_design = algorithmic_bytes_per_particle_step(main_res["n"], main_res["active_nodes"], S)
    bpp = survey_bytes_per_particle_step(main_res["n"], main_res["active_nodes"])
    launch_ms = main_res["t_ms"] / (args.steps * S)      # per fused launch (frame time / sub-steps)
    achieved = bpp * main_res["n"] / (launch_ms / 1e3) / 1e9
    achieved_design = bpp_design * main_res["n"] / (launch_ms / 1e3) / 1e9
    traffic = None
    counts = None
    try:
        with open(TRAFFIC_FILE) as fh:
            tr = json.load(fh)
        rec = tr.get("configs", {}).get(str((main_res["tuning"] or {}).get("config", 0)))
        if tr.get("kernel_sha") == kernel_source_sha() and tr.get("workload") == args.workload and rec:
            traffic = rec.get("bytes_per_launch")
            counts = rec
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": "k_fused_step" if args.pipeline == "fused"
                else "p2g+grid+g2p", "algorithmic_bytes_per_particle_step": bpp,
                "basis": "benchmark plan: x, v, A, F read and written once (192 B) + 72 B per active grid node",
                "launch_us": launch_ms * 1e3,
                "fused_design_basis": {"algorithmic_bytes_per_particle_step": bpp_design,
                                       "achieved": achieved_design, "frac": achieved_design / peak,
                                       "basis": "state the fused kernel keeps: x, id, F read and written once "
                                                "(104 B) + 48 B per active node + v, C once per call"}}
    # the CUDA-core side: FP32 FLOPs and thread instructions per particle-step
    # from the ncu capture of this kernel, against the rates of this GPU at the
    # sampled maximum SM clock (128 FP32 lanes and 4 x 32 issue lanes per SM)
    alu = None
    if counts is not None:
        import torch
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        mhz = main_res["clocks"].get("sm_max_mhz") or 2070.0
        per_s = main_res["n"] / (launch_ms / 1e3)
        flops = counts["fp32_flop_per_particle_step"] * per_s
        insts = counts["thread_inst_per_particle_step"] * per_s
        fpeak = sms * 128 * 2 * mhz * 1e6
        ipeak = sms * 4 * 32 * mhz * 1e6
        alu = {"bound": "alu", "achieved": flops / 1e12, "peak": fpeak / 1e12, "unit": "TFLOP/s",
               "frac": flops / fpeak, "issue": {"achieved": insts / 1e12, "peak": ipeak / 1e12,
                                                "unit": "T thread-instructions/s", "frac": insts / ipeak},
               "per_particle_step": {"fp32_flop": counts["fp32_flop_per_particle_step"],
                                     "thread_inst": counts["thread_inst_per_particle_step"]},
               "peak_kind": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (sms, mhz)}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, sample = time_oracle(args.workload, 15.0)
        cpu = {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle", "sample": sample,
               **cpu_description()}
        if differentiable is not None:
            differentiable["oracle"] = time_oracle_adjoint()
        cpu["other_workloads"] = time_oracle_configs()
    e2e_val = main_res["n"] * S * args.steps * world / (main_res["t_e2e_ms"] / 1e3)
    launches_per_frame = S if args.pipeline == "fused" else 3 * S
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_particles": main_res["n"], "n_grid": main_res["n_grid"],
                   "substeps_per_step": S, "pipeline": args.pipeline, "parallelism": "replicas%d" % world,
                   "l2": "flushed between timed steps (256 MB write)", "kernel_tuning": main_res["tuning"]},
        "roofline": roofline,
        "alu_roofline": alu,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "particle-steps/s", "h2d_bytes_per_step": main_res["h2d"],
                "d2h_bytes_per_step": main_res["d2h"],
                "readback": "mpm_read_particles_async every frame into pinned memory (overlapping the next "
                            "frame), all copies waited for inside the timed region",
                "value_with_synchronous_readback": main_res["n"] * S * args.steps * world /
                                                   (main_res["t_e2e_sync_ms"] / 1e3)},
        "gpu_launches": launches_per_frame * args.steps,
        "clocks": main_res["clocks"],
        "secondary": second,
        "sweep": sweep,
        "batched": batched,
        "differentiable": differentiable,
        "surface": surface,
    }
    print(json.dumps(line))
    ranks.close()


if __name__ == "__main__":
    main()
