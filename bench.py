"""Benchmark of the batched UUV step on B300.

Default workload (N=1): 1,048,576 envs over five vehicle classes (4/6/8
thrusters, 10-200 kg), fused hover observation + reward every step, random
initial pose within 2 m and 30 degrees, K substeps (default 4) per control
step, dt = 0.01 s, FP32 state. A "step" is one mg_step call: every env
advances one control step (K substeps) and writes its observation and reward.

`value` is whole-job env-steps/s with actions already on the device; `e2e`
is the same through mg_step_host with pinned host buffers (actions in,
observations and rewards out, every step). Under torchrun each rank runs its
own 1,048,576 envs on its own GPU (weak scaling, no data-path collective).

`--impl reference` times the FP64 CPU oracle on this host on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "env-steps/s at 1M envs vs roofline; serving p50/p99 step latency; err vs FP64"
UNIT = "env-steps/s"
SEED = 0x4D47


def kernel_sha() -> str:
    """Hash of the sources that define the step kernel (the profile summaries
    record the one they measured; runtime and serving code are not part of it):
    its headers and instantiations, and mg_jit.cpp, which compiles its
    class-specialised form and chooses that form's launch bounds."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2503_09203_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted([os.path.join(csrc, n) for n in ("mg_step.cuh", "mg_device.cuh", "mg_internal.h", "mg_jit.cpp")] +
                    glob.glob(os.path.join(csrc, "mg_step_pm*.cu")) + glob.glob(os.path.join(ROOT, "include", "*.h"))):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "step_kernel_dram_hover_K4.json")


def profiled_traffic(E, K):
    """DRAM bytes (read + write) per step of the workload, from the committed
    machine-readable ncu record of these kernel sources: bytes per env-step
    measured on smaller batches of the same launches (each larger than L2, the
    bytes per env-step equal at the sizes measured), times E; None if the
    record measured other sources, another K, or batches whose bytes per
    env-step disagree. Returns (bytes per step, record)."""
    if not os.path.exists(TRAFFIC_RECORD):
        return None, None
    rec = json.load(open(TRAFFIC_RECORD))
    if rec.get("source_sha") != kernel_sha() or rec.get("K") != K or not rec.get("proportional"):
        return None, rec
    if E < max(rec["envs_measured"]):
        return None, rec
    return float(rec["dram_bytes_per_env_step"]) * E, rec


def num_sms() -> int:
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def fp32_peak(pk) -> float:
    """FP32 FLOP/s of this device: 2 (FMA) x 128 FP32 lanes per SM x SMs x the
    maximum SM clock."""
    return 2 * 128 * num_sms() * pk["sm_max_mhz"] * 1e6


def spin(seconds: float):
    """Keep this thread busy for `seconds` (no sleep): a host thread that
    sleeps comes back with its launch path several times slower for tens of
    milliseconds, which a short timed region would measure."""
    t0 = time.perf_counter()
    x = 0
    while time.perf_counter() - t0 < seconds:
        x += 1
    return x


def dist_max(x: float, device="cuda") -> float:
    """Max of a per-rank float over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(envs_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Env-steps per second of all ranks together (weak scaling: every rank runs
    its own envs_per_rank envs)."""
    return envs_per_rank * world * steps / seconds


def rank_seed(rank: int) -> int:
    """Each rank simulates an independent batch of envs."""
    return SEED + rank


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], sm_max_mhz=d.get("sm_max_mhz", 2032.0), src="measured")
    return dict(hbm_gbs=6400.0, sm_max_mhz=2032.0, src="fallback")


# ---------------------------------------------------------------------------
# Clock sampling (nvidia-smi) around the timed region.
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.lines = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = []
        for t, line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((t, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 <= r[0] <= t1 + 0.05]
        window = "timed"
        if len(inside) < 3:
            inside = rows
            window = "whole run"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside), "window": window}


# ---------------------------------------------------------------------------
# Workload helpers.
# ---------------------------------------------------------------------------
def workload(n_envs, K):
    from paper_2503_09203_b300 import vehicles, workloads
    classes = vehicles.five_classes()
    counts = workloads.class_counts(n_envs, len(classes))
    return classes, counts, dict(vehicles.HOVER)


def bench_config(E, K, world):
    """The workload description shared by both arms of the benchmark."""
    classes, counts, _ = workload(E, K)
    state_io = sum(n * (2 * 4 * (13 + c["n_thr"]) + 4 * c["n_thr"] + 12 + 52 + 4) for c, n in zip(classes, counts))
    return {"workload": f"hover step, {E} envs per GPU, 5 classes (4/6/8 thr), K={K}, dt=0.01",
            "envs_per_gpu": E, "K": K, "classes": [c["name"] for c in classes], "counts": counts,
            "l2": f"inputs larger than L2 ({state_io / 1e6:.0f} MB touched per step)",
            "parallelism": f"replicas x{world} (independent envs per GPU)"}


def algorithmic(classes, counts, K):
    """Bytes and FP32 ops per env-step of the hover step (class parameters, no
    current): state in + out 2*4*(13+n), actions 4n, target 12, observation 52,
    reward 4."""
    from paper_2503_09203_b300 import binding as B
    tot_b = tot_f = 0.0
    for c, n in zip(classes, counts):
        nt = c["n_thr"]
        sub, obs = B.mg_count_flops(nt, with_current=False)
        tot_b += n * (2 * 4 * (13 + nt) + 4 * nt + 12 + 52 + 4)
        tot_f += n * (K * sub + obs)
    E = sum(counts)
    return tot_b / E, tot_f / E


def link_bound(h2d_bytes, d2h_bytes, steps=50):
    """Seconds per step of the end-to-end path's copies alone: the same bytes
    host->device and device->host between pinned buffers, one copy each way
    per step on two streams (overlapped), no step kernel."""
    import torch
    h_in = torch.empty(h2d_bytes // 4, dtype=torch.float32).pin_memory()
    d_in = torch.empty_like(h_in, device="cuda")
    d_out = torch.zeros(d2h_bytes // 4, dtype=torch.float32, device="cuda")
    h_out = torch.empty(d2h_bytes // 4, dtype=torch.float32).pin_memory()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    for it in range(steps + 3):
        if it == 3:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        with torch.cuda.stream(s_in):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s_out):
            h_out.copy_(d_out, non_blocking=True)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / steps


def time_steps(sim, acts, steps, warmup, stream, repeats=1):
    """Device time of `steps` mg_step calls (events on the launching stream);
    with repeats > 1 the fastest of that many consecutive timed regions.
    The first warm-up steps compile the class-specialised kernels of this K;
    the host thread then spins and warms up again: a thread that has waited
    (setup, compiles) launches several times slower for a while, and a short
    step would measure the host (a 1M-env step at K=1: about 75 us per call
    against 46 us on the device)."""
    import torch
    from paper_2503_09203_b300 import binding as B
    n_act = acts.shape[0]
    for i in range(warmup):
        B.mg_step(sim.handle, acts[i % n_act], 1, sim.obs, sim.reward, stream)
    torch.cuda.synchronize()
    spin(0.3)
    for i in range(max(warmup, 100)):   # the slow launches last about 100 calls
        B.mg_step(sim.handle, acts[i % n_act], 1, sim.obs, sim.reward, stream)
    best = None
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            B.mg_step(sim.handle, acts[i % n_act], 1, sim.obs, sim.reward, stream)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        best = t if best is None else min(best, t)
    return best


def action_pool(sim, n_pool, seed):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    a = torch.rand(n_pool, sim.action_floats, device="cuda", generator=g) * 2 - 1
    return a


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload.
# ---------------------------------------------------------------------------
def cpu_baseline(n_envs, K, budget_s=12.0, sample_envs=4096, threads=None):
    import oracle
    from paper_2503_09203_b300 import workloads
    classes, counts, cfg = workload(n_envs, K)
    rng = np.random.default_rng(1)
    ids = np.sort(rng.choice(n_envs, min(sample_envs, n_envs), replace=False))
    ec = workloads.env_classes(counts)[ids]
    envs, s = oracle.reset(classes, ec, cfg, SEED, env_ids=ids)
    threads = threads or os.cpu_count() or 1
    a = workloads.actions(3, 1, len(ids))
    oracle.rollout(classes, envs, s.copy(), a, 0.01, K, threads=threads)  # warm-up
    t0 = time.perf_counter()
    steps = 0
    while True:
        s, _, _ = oracle.rollout(classes, envs, s, a, 0.01, K, threads=threads)
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    v = len(ids) * steps / dt
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(ids)} envs sampled from the {n_envs}-env workload x {steps} steps "
                      f"(K={K}, hover obs+reward), {dt:.1f} s"}


# ---------------------------------------------------------------------------
# Extras: sweep, adjoint, serving, parity (N=1 only).
# ---------------------------------------------------------------------------
def sweep(pk, stream, sizes=(65536, 131072, 262144, 524288, 1048576), Ks=(1, 4, 8), steps=200):
    from paper_2503_09203_b300 import binding as B
    out = []
    for E in sizes:
        for K in Ks:
            classes, counts, cfg = workload(E, K)
            sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=False, reset=cfg)
            sim.reset(seed=SEED)
            acts = action_pool(sim, 4, 7)
            t = time_steps(sim, acts, steps, 10, stream, repeats=3)
            bpe, fpe = algorithmic(classes, counts, K)
            v = E * steps / t
            alu_peak = fp32_peak(pk)
            out.append({"envs": E, "K": K, "env_steps_per_s": v, "us_per_step": t / steps * 1e6,
                        "hbm_frac": v * bpe / (pk["hbm_gbs"] * 1e9), "alu_frac": v * fpe / alu_peak,
                        "l2_resident": E * bpe < 126e6})
            sim.close()
    return out


def plain_bench(stream, E=1024, K=1, steps=1000):
    """The plain workload: 1024 envs of class 0, no DR, K=1, 1000 steps
    (launch-latency bound: reported as us per step), one launch per step and
    the same steps as one 1000-step launch."""
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import vehicles
    import torch
    sim = B.Sim([vehicles.heavy8()], [E], dt=0.01, K=K, per_env_params=False, reset=dict(vehicles.NO_DR))
    sim.reset(seed=SEED)
    acts = action_pool(sim, 4, 5)
    t = time_steps(sim, acts, steps, 50, stream)
    a_all = torch.rand(steps, sim.action_floats, device="cuda") * 2 - 1
    B.mg_step(sim.handle, a_all, steps, sim.obs, sim.reward, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.mg_step(sim.handle, a_all, steps, sim.obs, sim.reward, stream)
    e1.record(stream)
    e1.synchronize()
    t_fused = e0.elapsed_time(e1) * 1e-3
    sim.status()
    sim.close()
    return {"envs": E, "K": K, "steps": steps, "us_per_step": t / steps * 1e6,
            "us_per_step_one_launch": t_fused / steps * 1e6}


def tracking_bench(pk, stream, E=1 << 20, K=4, steps=200):
    """Trajectory-tracking variant of the headline step (helix references)."""
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import vehicles, workloads
    classes = vehicles.five_classes()
    counts = workloads.class_counts(E, 5)
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=False, reset=dict(vehicles.TRACK_HELIX),
                task=B.TASK_TRACK)
    sim.reset(seed=SEED)
    acts = action_pool(sim, 4, 9)
    t = time_steps(sim, acts, steps, 10, stream)
    bpe, fpe = algorithmic(classes, counts, K)
    bpe += 48 + 4   # trajectory planes read at the observation, counter written back
    v = E * steps / t
    sim.close()
    return {"envs": E, "K": K, "reference": "helix", "env_steps_per_s": v, "us_per_step": t / steps * 1e6,
            "hbm_frac": v * bpe / (pk["hbm_gbs"] * 1e9)}


def payload_bench(pk, stream, E=1 << 20, K=4, steps=200):
    """Payload disturbance (point mass per env, full 6x6 inverse) with per-env
    DR and current, against the same batch without the payload."""
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import vehicles, workloads
    classes = vehicles.five_classes()
    counts = workloads.class_counts(E, 5)
    bpe, _ = algorithmic(classes, counts, K)
    out = {"envs": E, "K": K}
    for name, cfg, pay, planes in (("per_env_dr", vehicles.HOVER_DR, False, 9),
                                   ("payload_dr", vehicles.PAYLOAD_DR, True, 15)):
        sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(cfg), payload=pay)
        sim.reset(seed=SEED)
        acts = action_pool(sim, 4, 9)
        t = time_steps(sim, acts, steps, 10, stream)
        sim.status()
        sim.close()
        v = E * steps / t
        b = bpe + 16 * planes + 4   # parameter planes read per step; full target float4
        out[name] = {"env_steps_per_s": v, "us_per_step": t / steps * 1e6, "bytes_per_env_step": b,
                     "hbm_frac": v * b / (pk["hbm_gbs"] * 1e9)}
    return out


def actuated_bench(pk, stream, E=1 << 20, K=4, steps=100):
    """The three propulsion types (multirotor, rudder-propeller with fins,
    tiltrotor with servos) with per-env DR and current, Euler and RK4."""
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import vehicles, workloads
    classes = vehicles.actuated_classes()
    counts = workloads.class_counts(E, 3)
    out = {"envs": E, "K": K, "classes": [c["name"] for c in classes]}
    bpe, _ = algorithmic(classes, counts, K)
    b = bpe + 16 * 9 + 4   # parameter planes read per step; full target float4
    for name, integ in (("euler", B.MG_INTEG_EULER), ("rk4", B.MG_INTEG_RK4)):
        sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR),
                    integrator=integ)
        sim.reset(seed=SEED)
        acts = action_pool(sim, 4, 9)
        t = time_steps(sim, acts, steps, 10, stream)
        sim.status()
        sim.close()
        v = E * steps / t
        out[name] = {"env_steps_per_s": v, "us_per_step": t / steps * 1e6, "bytes_per_env_step": b,
                     "hbm_frac": v * b / (pk["hbm_gbs"] * 1e9)}
    return out


def hetero_graph_bench(stream, E=16384, K=4, T=100, reps=20, lanes=0):
    """Heterogeneous batch: 5 classes, per-env DR + current, K substeps; a
    T-step rollout (observation and reward every step) captured once as a CUDA
    graph after the autotuner chose the launch shape (lanes per env, envs per
    block, resident blocks per SM), then replayed. The same graph with one
    lane per env is timed beside it."""
    import torch
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import vehicles, workloads
    classes = vehicles.five_classes()
    counts = workloads.class_counts(E, 5)
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR))
    sim.reset(seed=SEED)
    acts = (torch.rand(T, sim.action_floats, device="cuda") * 2 - 1)
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    st = torch.cuda.Stream()
    out = {"envs": E, "K": K, "steps_per_graph": T}

    def time_graph():
        with torch.cuda.stream(st):
            g = B.mg_graph_capture(sim.handle, acts, T, obs, rew, st)
            for _ in range(3):
                B.mg_graph_launch(g, st)
            st.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                B.mg_graph_launch(g, st)
            e1.record(st)
            e1.synchronize()
            B.mg_graph_destroy(g)
        return e0.elapsed_time(e1) * 1e-3 / reps

    if lanes:   # a fixed shape (profiling: timings under a profiler would mislead the autotuner)
        B.mg_set_launch_shape(sim.handle, lanes, 0)
        shape = B.mg_get_launch_shape(sim.handle)
    else:
        with torch.cuda.stream(st):
            shape = B.mg_autotune(sim.handle, T, st)
    t = time_graph()
    out.update({"launch_shape": shape, "graph_s": t, "env_steps_per_s": E * T / t})
    if shape["lanes_per_env"] != 1 and not lanes:
        B.mg_set_launch_shape(sim.handle, 1, 0)
        t1 = time_graph()
        out["one_lane"] = {"graph_s": t1, "env_steps_per_s": E * T / t1}
    B.mg_status(sim.handle, st)
    sim.close()
    return out


def adjoint_bench(stream, E=8192, T=200, K=4, ckpt=20, pk=None):
    import torch
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import vehicles, workloads
    classes = vehicles.five_classes()
    counts = workloads.class_counts(E, 5)
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR),
                record_steps=T, ckpt_every=ckpt)
    sim.reset(seed=SEED)
    shape = B.mg_autotune(sim.handle, T, stream)   # launch shape of the recording rollout
    s0 = sim.get_state()
    acts = (torch.rand(T, sim.action_floats, device="cuda") * 2 - 1) * 0.99
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    g_rew = -torch.ones(T, sim.n_slots, device="cuda")
    g_act = torch.zeros(T, sim.action_floats, device="cuda")
    gA = torch.zeros(sim.n_slots, 6, device="cuda")
    gD = torch.zeros(sim.n_slots, 12, device="cuda")
    # One untimed repetition compiles the class-specialised adjoint kernels;
    # before each timed one the host thread spins (a thread that has waited
    # launches slowly for a while, and the backward's launches would start
    # late). The median of the timed repetitions is reported.
    times = []
    for rep in range(9):
        sim.set_state(s0)
        torch.cuda.synchronize()
        spin(0.05)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        B.mg_rollout(sim.handle, acts, T, None, rew, True, stream)
        e1.record(stream)
        B.mg_step_backward(sim.handle, acts, None, g_rew, None, g_act, gA, gD, None, stream)
        e2.record(stream)
        e2.synchronize()
        if rep > 0:
            times.append((e0.elapsed_time(e1) * 1e-3, e1.elapsed_time(e2) * 1e-3))
    tf, tb = np.median([t[0] for t in times]), np.median([t[1] for t in times])
    sim.close()
    # FP32 work: the recording rollout (K substeps + observation per step) and
    # the reverse pass (per substep: recompute + vector-Jacobian product).
    f_fwd = f_bwd = 0.0
    for c, n in zip(classes, counts):
        sub, obs, adj = B.mg_count_flops(c["n_thr"], adjoint=True, with_current=True)
        f_fwd += n * T * (K * sub + obs)
        f_bwd += n * T * K * adj
    out = {"envs": E, "horizon": T, "K": K, "ckpt_every": ckpt, "launch_shape": shape, "forward_s": tf, "backward_s": tb,
           "env_steps_per_s": E * T / (tf + tb), "backward_env_steps_per_s": E * T / tb,
           "fp32_tflops": (f_fwd + f_bwd) / (tf + tb) / 1e12}
    if pk:
        out["alu_frac"] = out["fp32_tflops"] * 1e12 / fp32_peak(pk)
        out["roofline_note"] = "latency bound: the reverse warps' dependent chain (130 four-warp blocks at 8192 envs); FMA = 2"
    return out


def serving_bench(plain_rate, n_req=10000, load=0.7, seed=11, horizon_max=1000, pk=None):
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import vehicles
    rng = np.random.default_rng(seed)
    classes = vehicles.five_classes()
    reqs = []
    for i in range(n_req):
        n = int(np.exp(rng.uniform(0, np.log(16384))))
        reqs.append((int(rng.integers(0, 5)), max(1, n), int(rng.integers(1, horizon_max + 1)),
                     int(rng.integers(1, 9)), int(rng.integers(1 << 62))))
    mean_work = np.mean([r[1] * r[2] * r[3] for r in reqs])  # env-substeps per request
    # Offered load: `load` x the plain path's substep throughput.
    lam = load * plain_rate / mean_work
    srv = B.mg_server_create(classes, 0.01, budget_bytes=8 << 30, max_requests=4096, reset=dict(vehicles.HOVER))
    t0 = time.perf_counter()
    ids = []
    t_next = t0
    for r in reqs:
        t_next += rng.exponential(1.0 / lam)
        while time.perf_counter() < t_next:
            time.sleep(min(0.001, max(0.0, t_next - time.perf_counter())))
        ids.append(B.mg_server_submit(srv, *r))
    B.mg_server_wait_idle(srv, 600.0)
    wall = time.perf_counter() - t0
    st = B.mg_server_stats_get(srv)
    for i in ids:
        B.mg_server_release(srv, i)
    B.mg_server_destroy(srv)
    # Work per env-step of the mix (weights: envs x horizon): FP32 ops of K
    # substeps + observation, and bytes of a device step (state in + out,
    # 10 per-env parameter planes, return read + write; actions drawn on the device).
    w = np.array([r[1] * r[2] for r in reqs], dtype=np.float64)
    per_nt = {c["n_thr"]: B.mg_count_flops(c["n_thr"]) for c in classes}
    flops = np.array([r[3] * per_nt[classes[r[0]]["n_thr"]][0] + per_nt[classes[r[0]]["n_thr"]][1] for r in reqs])
    nbytes = np.array([2 * 4 * (13 + classes[r[0]]["n_thr"]) + 160 + 8 for r in reqs], dtype=np.float64)
    busy = st["env_steps"] / max(st["busy_seconds"], 1e-9)
    roof = {"flops_per_env_step": float(np.sum(w * flops) / np.sum(w)),
            "bytes_per_env_step": float(np.sum(w * nbytes) / np.sum(w))}
    if pk:
        roof["busy_alu_frac"] = busy * roof["flops_per_env_step"] / fp32_peak(pk)
        roof["busy_hbm_frac"] = busy * roof["bytes_per_env_step"] / (pk["hbm_gbs"] * 1e9)
    return {"requests": n_req, "offered_load": load, "arrival_rate_per_s": lam, "wall_s": wall,
            "env_steps_per_s": st["env_steps"] / wall, "busy_env_steps_per_s": st["env_steps"] / max(st["busy_seconds"], 1e-9),
            "step_latency_p50_ms": st["step_latency_p50"] * 1e3, "step_latency_p99_ms": st["step_latency_p99"] * 1e3,
            "queue_delay_p50_ms": st["queue_delay_p50"] * 1e3, "queue_delay_p99_ms": st["queue_delay_p99"] * 1e3,
            "tick_p50_ms": st["tick_p50"] * 1e3, "tick_p99_ms": st["tick_p99"] * 1e3, "ticks": st["ticks"],
            "request_mix": "class U{0..4}, envs log-uniform [1,16384], horizon U{1..%d}, K U{1..8}" % horizon_max,
            "roofline_while_busy": roof}


def parity_sample(sim_classes, counts, K, n=512):
    """Sampled one-step error of the benchmark workload vs the oracle."""
    import torch
    import oracle
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import workloads
    E = sum(counts)
    cfg = workload(E, K)[2]
    sim = B.Sim(sim_classes, counts, dt=0.01, K=K, per_env_params=False, reset=cfg)
    sim.reset(seed=SEED)
    rng = np.random.default_rng(2)
    ids = np.sort(rng.choice(E, n, replace=False))
    a_s = workloads.actions(5, 1, n)
    a_env = np.zeros((1, E, 8), np.float32)
    a_env[:, ids] = a_s
    sim.step(sim.pack_actions(a_env))
    torch.cuda.synchronize()
    gpu = sim.get_state()[ids].astype(np.float64)
    envs, s0 = oracle.reset(sim_classes, workloads.env_classes(counts)[ids], cfg, SEED, env_ids=ids)
    ref, _, _ = oracle.rollout(sim_classes, envs, s0, a_s, 0.01, K)
    sgn = np.sign(np.sum(gpu[:, 3:7] * ref[:, 3:7], 1, keepdims=True))
    gpu[:, 3:7] *= np.where(sgn == 0, 1, sgn)
    err = np.linalg.norm(gpu - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1)
    sim.close()
    return {"one_step_max_rel_err": float(err.max()), "p99": float(np.quantile(err, 0.99)), "sampled_envs": n,
            "tol": 1e-5}


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=1 << 20)
    ap.add_argument("--substeps", type=int, default=4)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint workload (8k envs, T=200, K=4) and print its line (profiling)")
    ap.add_argument("--profile-range", action="store_true",
                    help="after the warm-up, run --steps steps of the headline workload between "
                         "cudaProfilerStart/Stop and exit (for an ncu range replay of DRAM traffic)")
    ap.add_argument("--hetero-lanes", type=int, default=0,
                    help="with --hetero-only: fix the launch shape to this many lanes per env instead of autotuning")
    ap.add_argument("--hetero-only", action="store_true",
                    help="run only the heterogeneous CUDA-graph workload (16k envs, 5 classes, K=4, 100 steps) "
                         "and print its line (profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.hetero_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"hetero_graph": hetero_graph_bench(torch.cuda.current_stream(), lanes=args.hetero_lanes)}))
        return
    if args.adjoint_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"adjoint": adjoint_bench(torch.cuda.current_stream())}))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    E, K = args.envs, args.substeps

    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(E, K, budget_s=max(5.0, 2.0 * args.steps / 1000.0 + 8.0))
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": bench_config(E, K, world),
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2503_09203_b300 import binding as B
    from paper_2503_09203_b300 import build as mgbuild

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mgbuild.build()
    pk = peaks()
    classes, counts, cfg = workload(E, K)
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=False, reset=cfg)
    sim.reset(seed=rank_seed(rank))
    stream = torch.cuda.current_stream()
    acts = action_pool(sim, 8, 100 + rank)
    bpe, fpe = algorithmic(classes, counts, K)
    n_launches = sim.launches_per_step()

    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    spin(0.5)   # the sampler starts; the host thread stays busy (see spin)
    # Warm-up, then exactly `steps` timed steps between barriers.
    for i in range(args.warmup):
        B.mg_step(sim.handle, acts[i % 8], 1, sim.obs, sim.reward, stream)
    torch.cuda.synchronize()
    if args.profile_range:
        clocks.stop()
        torch.cuda.profiler.start()
        for i in range(args.steps):
            B.mg_step(sim.handle, acts[i % 8], 1, sim.obs, sim.reward, stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        B.mg_status(sim.handle, stream)
        print(json.dumps({"profile_range": {"envs": E, "K": K, "steps": args.steps,
                                            "launches": args.steps * n_launches, "source_sha": kernel_sha()}}))
        sim.close()
        return
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    e0.record(stream)
    for i in range(args.steps):
        B.mg_step(sim.handle, acts[i % 8], 1, sim.obs, sim.reward, stream)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    tw1 = time.time()
    t = dist_max(e0.elapsed_time(e1) * 1e-3)
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        clocks.stop()
    B.mg_status(sim.handle, stream)
    value = whole_job_rate(E, world, args.steps, t)
    # Per-step device times of the same steps run again with an event after
    # each one (kept out of the timed region: an event between two steps ends
    # the programmatic overlap of their launches, about 3 us a step).
    n_ev = min(args.steps, 100)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev + 1)]
    ev[0].record(stream)
    for i in range(n_ev):
        B.mg_step(sim.handle, acts[i % 8], 1, sim.obs, sim.reward, stream)
        ev[i + 1].record(stream)
    ev[-1].synchronize()
    step_us = [round(ev[i].elapsed_time(ev[i + 1]) * 1e3, 2) for i in range(n_ev)]

    # End to end through the host-buffer entry point (pinned buffers).
    a_host = acts[0].cpu().pin_memory()
    o_host = torch.zeros(sim.n_slots, 13).pin_memory()
    r_host = torch.zeros(sim.n_slots).pin_memory()
    for _ in range(3):
        B.mg_step_host(sim.handle, a_host, 1, o_host, r_host, stream)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        B.mg_step_host(sim.handle, a_host, 1, o_host, r_host, stream)
    te = dist_max(time.perf_counter() - t0)
    e2e = {"value": whole_job_rate(E, world, args.e2e_steps, te), "unit": UNIT,
           "h2d_bytes_per_step": int(sim.action_floats * 4), "d2h_bytes_per_step": int(sim.n_slots * 14 * 4),
           "steps": args.e2e_steps, "api": "mg_step_host"}
    t_link = link_bound(e2e["h2d_bytes_per_step"], e2e["d2h_bytes_per_step"])
    e2e["link_bound"] = {"env_steps_per_s": E / t_link, "frac": e2e["value"] / world / (E / t_link),
                         "note": "the same bytes as plain pinned copies, one each way per step on two streams"}

    if rank != 0:
        sim.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    per_step = t / args.steps
    achieved_gbs = E * bpe / per_step / 1e9
    alu_peak = fp32_peak(pk)
    achieved_flops = E * fpe / per_step
    t_mem, t_alu = E * bpe / (pk["hbm_gbs"] * 1e9), E * fpe / alu_peak
    if t_mem >= t_alu:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved_gbs / pk["hbm_gbs"], "traffic": None,
                "peak_src": f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = {"bound": "alu", "achieved": achieved_flops / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved_flops / alu_peak, "traffic": None,
                "peak_src": f"2 x 128 FP32 lanes x {num_sms()} SMs x max SM clock"}
    traffic, trec = profiled_traffic(E, K)
    roof["traffic"] = traffic
    roof["traffic_note"] = (f"DRAM read+write bytes per step: bytes per env-step from ncu range replays of 2 and "
                            f"6 consecutive steps (differenced; write-backs included) at "
                            f"{' and '.join(str(e) for e in trec['envs_measured'])} envs, the same launches "
                            f"({trec['launches_per_step']} a step), times {E} envs: "
                            f"{os.path.relpath(TRAFFIC_RECORD, ROOT)}"
                            if traffic else "null: no ncu record of these kernel sources at this workload")
    shape = B.mg_get_launch_shape(sim.handle)
    kname = ("mg_step_kernel<NT, 0, 0, 1, 0, 0, JitLit> (class constants as literals: one kernel per class compiled "
             "at run time with NVRTC)" if shape["specialised_launches"] == n_launches else
             "mg_step_kernel<NT, 0, 0, 1, 0, 0> (class tables as the kernel parameter)")
    roof.update({"kernel": f"{kname}; propellers, Euler; {n_launches} launches per step", "launch_shape": shape,
                 "bytes_per_env_step": bpe, "flops_per_env_step": fpe,
                 "hbm_frac": achieved_gbs / pk["hbm_gbs"], "alu_frac": achieved_flops / alu_peak})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(E, K, world),
            "e2e": e2e, "gpu_launches": args.steps * n_launches, "roofline": roof,
            "step_us": {"per_step": step_us, "median": float(np.median(step_us)),
                        "note": "a second pass of the timed steps with an event after each step"},
            "clocks": clocks.summary(tw0, tw1)}
    if world == 1 and not args.no_extras:
        line["cpu_baseline"] = cpu_baseline(E, K)
        line["cpu_baseline_1core"] = cpu_baseline(E, K, budget_s=4.0, sample_envs=1024, threads=1)
        line["plain"] = plain_bench(stream)
        sim.close()
        line["parity"] = parity_sample(classes, counts, K)
        line["sweep"] = sweep(pk, stream)
        line["sweep_timing"] = ("per configuration: warm-up, the host thread kept busy, 100 more steps, then the "
                                "fastest of 3 consecutive timed regions of 200 mg_step calls (CUDA events)")
        line["tracking"] = tracking_bench(pk, stream)
        line["payload"] = payload_bench(pk, stream)
        line["actuated"] = actuated_bench(pk, stream)
        line["hetero_graph"] = hetero_graph_bench(stream)
        line["adjoint"] = adjoint_bench(stream, pk=pk)
        plain_substeps = max(r["env_steps_per_s"] * r["K"] for r in line["sweep"] if r["envs"] == 65536)
        line["serving"] = [serving_bench(plain_substeps, load=0.7, pk=pk), serving_bench(plain_substeps, load=0.9, pk=pk)]
    else:
        sim.close()
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
