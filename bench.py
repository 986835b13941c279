#!/usr/bin/env python
"""Benchmark of the fused binary-fluid LB step on GB300.

Headline workload: the 8192 x 8192 spinodal lattice (D2Q9 two-population
MRT, walls at y = 0 and y = 8191, phi uniform in [-0.1, 0.1) from SplitMix64
seed 12345, a = kappa = 0.04, Gamma = 0.1, tau_alpha 1.5, tau_beta 0.6), FP32
deviation storage.  One bench step = one full time step of every node
(pull-stream, moments, phi stencils with wetting ghosts, Step 2, equilibria,
MRT collision, store).  The state (9.7 GB) is far larger than L2, so no flush
is needed between steps.

Printed: one JSON line with MLUPS (whole job), the roofline of the step
kernel (algorithmic 144 B per node update over its event-timed duration,
against the measured HBM copy bandwidth), the end-to-end number through the
C ABI with host buffers, the FP64 oracle on the host cores, and extras: the
FP64 build (ALU-bound on GB300) and the batched 256-domain workload against
a per-domain launch loop.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own replica of the headline lattice (weak
scaling, no collective on the data path) and a node-balanced share of the
batched workload's domains; rank 0 prints.
"""
from __future__ import annotations

import argparse
import math
import ctypes
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbinputs  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
BYTES_PER_NODE = {"fp32": 144, "fp64": 288, "fp32c": 104}  # fp32c: compact g storage


# Device-code sources of the step kernels: an ncu figure recorded under
# profiles/ stays valid while these are unchanged.
KERNEL_SOURCES = ("lb_async.cuh", "lb_internal.h", "lb_node.cuh", "lb_node_x2.cuh", "lb_step.cuh",
                  "lb_step_compact.cuh", "lb_step_kernels.cuh", "lb_step_f32.cu",
                  "lb_step_f64.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_0812_1282_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


def profile_value(name: str, key: str):
    """A number recorded from an ncu capture (profiles/<name>.txt, lines
    'source_hash: ...' and '<key>: ...'); None when the kernel sources
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", name + ".txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    m_val = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
    if not m_hash or not m_val or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_val.group(1))


def profile_traffic(name: str):
    """DRAM bytes per launch of an ncu capture (None when stale)."""
    return profile_value(name, "dram_bytes_per_launch")


def sm_max_mhz() -> float:
    """Maximum SM clock of GPU 0 (nvidia-smi), 2070 MHz if unreadable."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", "0"], capture_output=True, text=True, timeout=30).stdout
        return float(out.split()[0])
    except Exception:
        return 2070.0


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path:
                try:
                    os.unlink(self.path)
                except OSError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, value: float) -> float:
    """Largest value over all ranks (the job's elapsed time is the slowest
    rank's); a timing collective only, nothing on the data path."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(nodes_per_rank: int, steps: int, ws: int, max_elapsed: float) -> float:
    """Whole-job MLUPS: every rank advances its own replica by `steps`
    steps; the job takes as long as the slowest rank."""
    return nodes_per_rank * steps * ws / max_elapsed / 1e6


# ------------------------------------------------------------ our arm
def time_steps(sim, steps, torch):
    stream = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_headline(lbf, torch, ws, steps, warmup, precision="fp32", size=None, tile=None,
                 compact=False):
    c = lbinputs.SPINODAL_8192
    nx = ny = size or c["nx"]
    n = nx * ny
    p = lbf.params(precision=precision, compact_g=compact, **c["params"])
    sim = lbf.Lattice(p, nx, ny)
    sim.init_random(c["amp"], c["seed"])
    if tile:
        sim.set_tile(*tile)
        tile = sim.tile()
    else:
        tile = sim.autotune(reps=3)
        sim.init_random(c["amp"], c["seed"])
    sim.step(warmup)
    torch.cuda.synchronize()
    launches0 = sim.launch_count
    barrier(ws)
    dt = time_steps(sim, steps, torch)
    barrier(ws)
    launches = sim.launch_count - launches0
    st = sim.stats()
    return sim, dict(seconds=dt, nodes=n, tile=list(tile[:2]), launches=launches,
                     mass=st["mass"], max_u=st["max_u"], nonfinite=st["nonfinite"])


def run_e2e(lbf, torch, steps, compact=False, tile=None):
    """The same job through the public API with host buffers: upload phi0
    from pinned host memory, run `steps` steps reading the diagnostics back
    every 100 steps, and download the final phi field."""
    import numpy as np

    c = lbinputs.SPINODAL_8192
    nx, ny = c["nx"], c["ny"]
    phi0 = torch.from_numpy(lbinputs.random_field(nx, ny, c["amp"], c["seed"])).pin_memory()
    out_phi = torch.empty((ny, nx), dtype=torch.float64).pin_memory()
    p = lbf.params(precision="fp32", compact_g=compact, **c["params"])
    sim = lbf.Lattice(p, nx, ny)
    if tile:  # the launch shape the device-timed run settled on
        sim.set_tile(*tile)
    else:
        sim.autotune(reps=3)
    stats = lbf.Stats()

    def job():
        # every call below returns once its results are on the host (the
        # steps run asynchronously until the next statistics read), so host
        # clock readings between calls split the job without extra waits
        d2h, marks = 0, [time.perf_counter()]
        lbf.lib().lb_init_phi(sim.h, 0, ctypes.c_void_p(phi0.data_ptr()), 0)
        marks.append(time.perf_counter())
        done = 0
        while done < steps:
            k = min(100, steps - done)
            sim.step(k)
            done += k
            lbf.lib().lb_moments(sim.h, 0, 0, None, None, None, None, ctypes.byref(stats))
            d2h += 48
        marks.append(time.perf_counter())
        lbf.lib().lb_moments(sim.h, 0, 0, None, ctypes.c_void_p(out_phi.data_ptr()), None,
                             None, None)
        marks.append(time.perf_counter())
        return d2h, marks

    job()  # warm-up: the step graphs are built on first use
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h, marks = job()
    dt = time.perf_counter() - t0
    d2h += out_phi.numel() * 8
    h2d = phi0.numel() * 8
    ok = bool(np.isfinite(out_phi.numpy()).all())
    sim.close()
    split = [round((b - a) * 1e3, 2) for a, b in zip(marks, marks[1:])]
    return dict(seconds=dt, h2d=h2d, d2h=d2h, finite=ok,
                breakdown_ms={"upload_and_init": split[0], "steps_and_stats": split[1],
                              "phi_readback": split[2]})


def fp64_pipe_peak(lbf):
    """Measured FP64 operations per second of this GPU, per operation kind
    (lb_fp64_peak: independent DFMA, DADD or DMUL chains over the whole
    GPU), best of three runs each."""
    out = {}
    for kind, name in ((0, "dfma"), (1, "dadd"), (2, "dmul")):
        out[name] = max(lbf.lb_fp64_peak(kind) for _ in range(3))
    return out


def run_fp64(lbf, torch, steps, size=None, tile=None):
    """The headline workload in FP64 storage and arithmetic.  On this GPU
    the step is bound by the FP64 pipe, so besides its bytes it reports the
    pipe's operations per second against the pipe's measured peak
    (lb_fp64_peak), with the operations per node counted by ncu
    (profiles/lb_step_mrt_fp64_2048.txt)."""
    c = lbinputs.SPINODAL_8192
    side = size or c["nx"]
    n = side * side
    p = lbf.params(precision="fp64", **c["params"])
    sim = lbf.Lattice(p, side, side)
    sim.init_random(c["amp"], c["seed"])
    if tile:
        sim.set_tile(*tile)
    else:
        tile = sim.autotune(reps=1)
    sim.step(2)
    with ClockSampler(torch.cuda.current_device()) as clk:
        dt = time_steps(sim, steps, torch)
    sim.close()
    with ClockSampler(torch.cuda.current_device()) as clk_peak:
        peak = fp64_pipe_peak(lbf)
    res = dict(mlups=n * steps / dt / 1e6, seconds_per_step=dt / steps, tile=list(tile[:2]),
               gbs=n * BYTES_PER_NODE["fp64"] * steps / dt / 1e9, bound="alu",
               clocks=clk.summary())
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clk_peak.summary().get("sm_mhz") or sm_max_mhz()
    res["pipe_peak_measured"] = {
        k + "_gops": round(v / 1e9, 1) for k, v in peak.items()}
    res["pipe_peak_measured"].update(
        {k + "_per_clk_per_sm": round(v / (sms * mhz * 1e6), 3) for k, v in peak.items()},
        sm_mhz=mhz, source="lb_fp64_peak: independent dependency chains of one FP64 operation "
                           "over the whole GPU, CUDA events, best of 3")
    # the FP64 pipe takes one DADD, DMUL or DFMA per slot: its roofline counts
    # those operations (a DFMA is two flops, the others one); the peak of the
    # step's own mix of the three kinds is the harmonic mean weighted by the
    # per-node counts ncu measured
    prof = "lb_step_mrt_fp64_2048"
    cnt = {k: profile_value(prof, k + "_per_node") for k in ("dfma", "dadd", "dmul")}
    opn = profile_value(prof, "fp64_ops_per_node")
    fpn = profile_value(prof, "fp64_flops_per_node")
    res["fp64_ops_per_node"] = opn
    res["fp64_flops_per_node"] = fpn
    if opn is not None and all(v is not None for v in cnt.values()):
        mix_peak = opn / sum(cnt[k] / peak[k] for k in cnt)   # operations per second
        rate = n * steps / dt
        res.update(achieved_gops=round(rate * opn / 1e9, 1),
                   peak_gops=round(mix_peak / 1e9, 1),
                   frac=round(rate * opn / mix_peak, 4),
                   achieved_tflops=round(rate * fpn / 1e12, 4),
                   peak_source="measured: lb_fp64_peak per kind, weighted by the step's "
                               "operation mix (ncu counts per node)")
    return res


def run_capillary(lbf, torch, steps=None):
    """Capillary filling (Sec. VI) on the 1000 x 120 set-up in FP32: the
    whole job (obstacle step, the meniscus fitted every 500 steps) timed on
    the host clock, and the Washburn force-balance fit of the filled length
    over the second half.  The autotuner picks between a launch per step and
    one persistent launch per graph of steps; both are timed."""
    import numpy as np

    c = lbinputs.CAPILLARY_1000x120
    steps = steps or c["steps"]
    p = lbf.params(precision="fp32", **c["params"])
    sim = lbf.Lattice(p, c["nx"], c["ny"])
    sim.init_channel(c["res_len"], c["ch_w"], lbf.lb_wetting_h(c["theta"]), c["h_block"])
    fluid = int((sim.geometry() == 0).sum())
    y0 = (c["ny"] - c["ch_w"]) // 2
    ts, ls, ths = [], [], []
    sim.autotune(reps=2)
    chosen = sim.schedule()
    sim.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 2
    while done < steps:
        k = min(c["every"] - done % c["every"], steps - done)
        sim.step(k)
        done += k
        xf, th, _ = sim.meniscus(c["res_len"], c["nx"], y0, y0 + c["ch_w"])
        ts.append(done)
        ls.append(xf - (c["res_len"] - 0.5))
        ths.append(th)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = sim.stats()

    # launch forms: 0 a launch per step, 1 one persistent launch per graph,
    # 2 two steps per launch
    def per_mode(s, mode):
        s.set_schedule(lbf.schedule(128, 16, ctas_per_sm=0, persist=int(mode == 1),
                                    steps_per_launch=2 if mode == 2 else 1))
        s.step(128)
        return time_steps(s, 2000, torch)

    mode_of = 1 if chosen["persist"] else (2 if chosen["steps_per_launch"] == 2 else 0)
    dt_mode = {m: per_mode(sim, m) for m in (0, 1, 2)}
    dt_steps = dt_mode[mode_of]
    sim.close()
    # latency floor of the same kernels: one CTA's tile (32 x 8 nodes with a
    # small block), stepped the same way; the capillary step cannot be faster
    tiny = lbf.Lattice(p, 32, 8)
    cls = np.zeros((8, 32), np.uint8)
    cls[2:5, 10:14] = 1
    tiny.set_geometry(cls, [0.0, 0.0])
    tiny.init_phi(np.zeros((8, 32)))
    dt_floor_mode = {m: per_mode(tiny, m) for m in (0, 1, 2)}
    dt_floor = dt_floor_mode[mode_of]
    tiny.close()
    t = np.array(ts, float)
    l = np.array(ls)
    nua = (c["params"]["tau_alpha"] - 0.5) / 3
    nub = (c["params"]["tau_beta"] - 0.5) / 3
    L = c["nx"] - c["res_len"]
    Y = (nua - nub) * l * l / 2 + nub * L * l
    late = t >= t[-1] / 2
    slope = float(np.polyfit(t[late], Y[late], 1)[0])
    theta_a = float(np.mean(np.array(ths)[late]))
    gamma = math.sqrt(8 * c["params"]["a"] * c["params"]["kappa"] / 9)
    k_theory = gamma * c["ch_w"] * math.cos(math.radians(theta_a)) / 6.0
    return dict(steps=steps, fluid_nodes=fluid, job_seconds=wall,
                step_us=dt_steps / 2000 * 1e6, mlups_fluid=fluid * 2000 / dt_steps / 1e6,
                bound="latency", latency_floor_us=dt_floor / 2000 * 1e6,
                floor_over_step=dt_floor / dt_steps,
                l_final=float(l[-1]), theta_a_late=theta_a,
                washburn_slope=slope, washburn_slope_theory=k_theory,
                nonfinite=int(st["nonfinite"]),
                launch=("per step", "persistent", "two steps per launch")[mode_of],
                per_step_launch_us=dt_mode[0] / 2000 * 1e6,
                persistent_launch_us=dt_mode[1] / 2000 * 1e6,
                two_step_launch_us=dt_mode[2] / 2000 * 1e6,
                latency_floor_per_step_launch_us=dt_floor_mode[0] / 2000 * 1e6,
                latency_floor_persistent_us=dt_floor_mode[1] / 2000 * 1e6,
                latency_floor_two_step_us=dt_floor_mode[2] / 2000 * 1e6,
                note="obstacle path (the state stays in L2, so launch, L2 and neighbour-wait "
                     "latency bound it): the fused obstacle step as a launch per step, as one "
                     "cooperative launch per 64-step graph with each 32 x 8 tile waiting only "
                     "for the tiles under its halo, or two steps per launch (each tile stepping "
                     "a four-node halo first); the autotuner picks (launch); step_us is the "
                     "pick, latency_floor_us the same launch form on a single 32 x 8 tile; "
                     "front by lb_meniscus every 500 steps; Washburn fit (nu_a - nu_b) l^2/2 + "
                     "nu_b L l vs t over the second half, theory gamma w cos(theta_a) / 6")


BATCH_JOB_STEPS = 10000
BATCH_GOLDEN = os.path.join(ROOT, "tests", "golden", "batch_angles.json")


def batch_params(lbf, specs, compact):
    # the momentum-relaxing reading of Step 2: with the literal rates 19 of
    # the 256 drops (high angle, viscosity ratio 10) go non-finite within the
    # 10000-step job; the throughput is the same either way
    return [lbf.params(collision="mrt", precision="fp32", tau_alpha=s["tau_alpha"],
                       tau_beta=s["tau_beta"], h_bottom=lbf.lb_wetting_h(s["theta"]),
                       step2_relax_momentum=True, compact_g=compact) for s in specs]


# The eight-class ladder the autotuner picks for the 256 drops (strips of 120,
# 184, 244, 308, 368, 432, 492 and 556 columns, 96 rows, the rows of the three
# narrowest classes sealed): a fixed schedule for profiling runs.
LADDER_BX = (64, 96, 128, 160, 192, 224, 256, 288)
LADDER_SEALED_UP_TO = 128


# fixed batched schedules (--schedule): (rows per item, persistent launches)
FIXED_SCHEDULES = {"ladder": (96, 0), "ladder-persist": (32, 1)}


def ladder_schedule(lbf, rows=64, persist=0):
    strip = lambda bx: (62 * (bx // 32) - 2) // 4 * 4
    return lbf.schedule(list(LADDER_BX), rows, ctas_per_sm=0,
                        max_nx=[strip(bx) for bx in LADDER_BX[:-1]], order=1, persist=persist,
                        fill_pct=85 if persist else 0,
                        seal_edges=[int(bx <= LADDER_SEALED_UP_TO) for bx in LADDER_BX])


# steps of the persistent-launch comparison on the batched workload
PERSIST_CMP_STEPS = 640


def run_batched(lbf, torch, loop_steps=20, compact=False, ws=1, rank=0, job_steps=None,
                fixed_schedule=False):
    """The 256 sessile drops (sides 64..512) of the batched workload: the
    whole 10000-step job in one batched handle per GPU (the autotuner picks
    the schedule), timed from the first step to the last; then, on a single
    GPU, the same domains stepped one launch per domain per step (each
    domain with its own tuned launch shape), timed over `loop_steps` steps
    and scaled to the job.  Under torchrun every rank takes a node-balanced
    share of the domains (no data-path collective) and the per-domain
    results are gathered at the end."""
    from paper_0812_1282_gb300 import shard

    job = job_steps or BATCH_JOB_STEPS
    specs = lbinputs.batch_specs()
    plist = batch_params(lbf, specs, compact)
    nodes_d = [s["nx"] * s["ny"] for s in specs]
    parts = shard.partition(nodes_d, ws)
    mine = parts[rank]
    bp = [plist[d] for d in mine]
    batch = lbf.Batch(bp, [specs[d]["nx"] for d in mine], [specs[d]["ny"] for d in mine])

    def init():
        for k, d in enumerate(mine):
            batch.init_drop(specs[d]["R"], specs[d]["cx"], specs[d]["cy"], dom=k)

    init()
    if fixed_schedule:
        batch.set_schedule(ladder_schedule(lbf, *fixed_schedule))
        tile = batch.tile()
    else:
        tile = batch.autotune(reps=2)
    sched = batch.schedule()
    batch.step(128)  # builds the step graphs
    init()
    torch.cuda.synchronize()
    launches0 = batch.launch_count
    barrier(ws)
    dt_b = max_over_ranks(ws, time_steps(batch, job, torch))
    launches = batch.launch_count - launches0
    # per-domain results of the timed job: angle, max |u|, non-finite count
    rows = {}
    for k, d in enumerate(mine):
        st = batch.stats(dom=k)
        try:
            th = batch.contact_angle(dom=k)[0] if st["nonfinite"] == 0 else float("nan")
        except lbf.LBError:
            th = float("nan")
        rows[d] = [th, st["max_u"], float(st["nonfinite"])]
    persist_cmp = None
    if compact and ws == 1 and not fixed_schedule:
        # the same ladder as persistent multi-step launches (each class's
        # steps of a 64-step graph in one launch), for comparison
        batch.set_schedule(ladder_schedule(lbf, 32, persist=1))
        batch.step(128)
        torch.cuda.synchronize()
        dt_p = time_steps(batch, PERSIST_CMP_STEPS, torch)
        n_all = sum(nodes_d)
        persist_cmp = dict(steps_timed=PERSIST_CMP_STEPS,
                           mlups=round(n_all * PERSIST_CMP_STEPS / dt_p / 1e6, 1),
                           achieved_gbs=round(n_all * PERSIST_CMP_STEPS * 104 / dt_p / 1e9, 1),
                           schedule=batch.schedule())
    batch.close()
    table = shard.gather_rows(len(specs), 3, rows, device="cuda" if ws > 1 else "cpu")
    nodes = sum(nodes_d)
    bpn = BYTES_PER_NODE["fp32c" if compact else "fp32"]
    res = dict(domains=len(specs), nodes=nodes, steps_timed=job, job_seconds=round(dt_b, 4),
               batched_mlups=nodes * job / dt_b / 1e6,
               batched_sims_per_s=len(specs) / dt_b,
               achieved_gbs=round(nodes * job * bpn / dt_b / 1e9, 1),
               algorithmic_bytes_per_node=bpn,
               gpu_launches=launches,
               schedule=sched, tile=list(tile[:2]),
               storage="compact g" if compact else "full",
               nonfinite_domains=sum(1 for r in table if r[2] > 0))
    if persist_cmp is not None:
        res["persistent_launches"] = persist_cmp
    if ws > 1:
        res.update(parallelism="%d ranks, node-balanced split of the domains (greedy, "
                               "largest first), no data-path collective" % ws,
                   nodes_per_rank=shard.rank_loads(nodes_d, parts))
    # angle error of the timed run against the FP64 oracle's stored angles
    if os.path.exists(BATCH_GOLDEN):
        with open(BATCH_GOLDEN) as fh:
            gold = json.load(fh)
        if gold["steps"] == job:
            errs = [abs(table[r["dom"]][0] - r["relax"]["theta"]) for r in gold["domains"]
                    if not r["relax"]["diverged"]]
            res["angle_err_max_deg"] = max(errs) if errs else None
            res["angle_err_domains"] = len(errs)
    if ws > 1 or rank != 0:
        return res
    # the per-domain launch loop, each domain with its own tuned launch shape
    sims = []
    for d, s in enumerate(specs):
        sim = lbf.Lattice(plist[d], s["nx"], s["ny"])
        sim.init_drop(s["R"], s["cx"], s["cy"])
        sim.autotune(reps=2)
        sim.init_drop(s["R"], s["cx"], s["cy"])
        sim.step(2)
        sims.append(sim)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(loop_steps):
        for sim in sims:
            sim.step(1)
    e1.record()
    torch.cuda.synchronize()
    dt_l = e0.elapsed_time(e1) / 1e3
    # stronger loop: each domain runs all its steps back to back from its own
    # captured CUDA graphs, one domain after another
    for sim in sims:
        sim.step(64)  # builds each domain's graphs
    torch.cuda.synchronize()
    e0.record()
    for sim in sims:
        sim.step(loop_steps)
    e1.record()
    torch.cuda.synchronize()
    dt_g = e0.elapsed_time(e1) / 1e3
    for sim in sims:
        sim.close()
    scale = job / loop_steps
    res.update(loop_mlups=nodes * loop_steps / dt_l / 1e6,
               loop_graph_mlups=nodes * loop_steps / dt_g / 1e6,
               loop_sims_per_s=len(specs) / (dt_l * scale),
               loop_graph_sims_per_s=len(specs) / (dt_g * scale),
               speedup_vs_loop=dt_l * scale / dt_b, speedup_vs_loop_graph=dt_g * scale / dt_b,
               note="batched: the whole %d-step job timed (CUDA events, one batched handle, "
                    "schedule from lb_autotune); loop = one launch per domain per step, each "
                    "domain with its own autotuned launch shape; loop_graph = each domain's "
                    "steps replayed from its own CUDA graphs, domains in sequence; both loops "
                    "timed over %d steps and scaled to the job; MRT with the momentum-"
                    "relaxing Step-2 reading; angle_err_max_deg = the timed run's angles "
                    "against the FP64 oracle's (tests/golden/batch_angles.json, 16 smallest "
                    "domains, compact and full storage both tested in "
                    "tests/test_gpu_batch_angles.py); persistent_launches = the eight-class "
                    "ladder (32 rows) as persistent multi-step launches, one per class per "
                    "64-step graph, timed over %d steps" % (job, loop_steps, PERSIST_CMP_STEPS))
    return res


def cpu_baseline(seconds=12.0):
    """The FP64 oracle, as written, on the host cores: the 512 x 512 cut of
    the same spinodal workload, stepped until about `seconds` elapse."""
    import oracle

    c = lbinputs.SPINODAL_8192
    n = c["sub"]
    p = oracle.params(**c["params"])
    lat = oracle.OracleLattice(p, n, n)
    lat.init_random(c["amp"], c["seed"])
    lat.step(1)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        lat.step(5)
        done += 5
    dt = time.perf_counter() - t0
    res = {"value": n * n * done / dt / 1e6, "unit": "MLUPS", "cores": oracle.get_threads(),
           "kind": "oracle",
           "sample": "%dx%d cut of the 8192^2 spinodal MRT workload, %d FP64 steps (%.1f s)"
                     % (n, n, done, dt)}
    # the same cut on one core, and the 100 x 50 BGK drop on all cores
    # (about 3 s each)
    threads = oracle.get_threads()

    def rate(lattice, nodes, budget):
        k, t1 = 0, time.perf_counter()
        while time.perf_counter() - t1 < budget:
            lattice.step(5)
            k += 5
        return nodes * k / (time.perf_counter() - t1) / 1e6

    try:
        oracle.set_threads(1)
        res["single_core_mlups"] = round(rate(lat, n * n, 3.0), 3)
    finally:
        oracle.set_threads(threads)
    d = lbinputs.DROP_100x50
    small = oracle.OracleLattice(oracle.params(**d["params"]), d["nx"], d["ny"])
    small.init_drop(d["R"], d["cx"], d["cy"])
    res["drop_100x50_mlups"] = round(rate(small, d["nx"] * d["ny"], 3.0), 3)
    return res


def ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__

    if rank == 0 or ws == 1:
        __graft_entry__.build()
    barrier(ws)
    import paper_0812_1282_gb300 as lbf

    lbf.lib()
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))

    if args.only:
        # one extra workload alone (profiling aid): its JSON object only
        if args.only == "batched":
            res = run_batched(lbf, torch, max(4, args.steps), compact=args.storage == "compact",
                              ws=ws, rank=rank, job_steps=args.job_steps,
                              fixed_schedule=FIXED_SCHEDULES.get(args.schedule))
            if rank != 0:
                return
        elif args.only == "fp64":
            tile = tuple(int(v) for v in args.tile.split("x")) if args.tile else None
            res = run_fp64(lbf, torch, max(3, args.steps), size=args.size, tile=tile)
        else:
            res = run_capillary(lbf, torch, max(1000, args.steps))
        print(json.dumps({"workload": args.only, **res}), flush=True)
        return
    tile = tuple(int(v) for v in args.tile.split("x")) if args.tile else None
    with ClockSampler(torch.cuda.current_device()) as clk:
        sim, head = run_headline(lbf, torch, ws, args.steps, args.warmup, size=args.size, tile=tile,
                                 compact=args.storage == "compact")
    clocks = clk.summary()
    sim.close()
    torch.cuda.empty_cache()
    side = args.size or 8192
    compact = args.storage == "compact"
    bpn = BYTES_PER_NODE["fp32c" if compact else "fp32"]
    dt = max_over_ranks(ws, head["seconds"])
    value = job_value(head["nodes"], args.steps, ws, dt)
    per_launch = dt / args.steps
    achieved = head["nodes"] * bpn / per_launch / 1e9
    prof = "lb_step_compact_mrt_fp32_8192" if compact else "lb_step_mrt_fp32_8192"
    traffic = profile_traffic(prof) if side == 8192 else None
    line = {
        "metric": "MLUPS (MRT, FP32, 8192^2) and HBM-roofline fraction",
        "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "spinodal %dx%d D2Q9 two-population MRT (FP32 deviation "
                               "storage), walls y=0/%d, seed 12345" % (side, side, side - 1),
                   "nx": side, "ny": side, "collision": "mrt", "tile": head["tile"],
                   "storage": ("compact g: phi word, Gamma mu, u_eq per node (tau_phi = 1); "
                               "9 f + 4 values = 104 B per node update") if compact else
                              "full: 9 f + 9 g = 144 B per node update",
                   "l2": "state %.1f GB >> 129 MB L2, no flush needed"
                         % (side * side * bpn / 1e9),
                   "parallelism": "replica per GPU" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": traffic,
                     "peak_source": "%s MEASURED_PEAKS.json hbm_gbs" % peak_kind,
                     "algorithmic_bytes_per_node": bpn},
        "gpu_launches": head["launches"],
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.quick:
        e2e = run_e2e(lbf, torch, args.steps, compact=compact, tile=head["tile"])
        line["e2e"] = {"value": round(head["nodes"] * args.steps / e2e["seconds"] / 1e6, 1),
                       "unit": "MLUPS", "h2d_bytes_per_step": e2e["h2d"] // args.steps,
                       "d2h_bytes_per_step": e2e["d2h"] // args.steps,
                       "job": "phi0 H2D from pinned memory, %d steps, stats D2H every 100 "
                              "steps, final phi D2H (after one untimed warm-up job that "
                              "builds the step graphs)" % args.steps,
                       "breakdown_ms": e2e["breakdown_ms"]}
        torch.cuda.empty_cache()
        extras = {}
        if compact:
            # the same workload with full g storage (144 B per node update)
            try:
                simf, headf = run_headline(lbf, torch, 1, max(20, args.steps // 2), args.warmup,
                                           size=args.size, compact=False)
                simf.close()
                nf = headf["nodes"] * max(20, args.steps // 2)
                gbs = nf * BYTES_PER_NODE["fp32"] / headf["seconds"] / 1e9
                extras["full_storage"] = {
                    "mlups": round(nf / headf["seconds"] / 1e6, 1), "tile": headf["tile"],
                    "achieved_gbs": round(gbs, 1), "frac": round(gbs / hbm, 4),
                    "algorithmic_bytes_per_node": BYTES_PER_NODE["fp32"]}
            except Exception as exc:
                extras["full_storage"] = {"error": str(exc)}
            torch.cuda.empty_cache()
        try:
            extras["fp64"] = run_fp64(lbf, torch, max(4, args.steps // 20))
        except Exception as exc:  # report, do not hide
            extras["fp64"] = {"error": str(exc)}
        torch.cuda.empty_cache()
        try:
            extras["batched"] = run_batched(lbf, torch, max(20, args.steps // 2), compact=compact)
        except Exception as exc:
            extras["batched"] = {"error": str(exc)}
        torch.cuda.empty_cache()
        try:
            extras["capillary"] = run_capillary(lbf, torch)
        except Exception as exc:
            extras["capillary"] = {"error": str(exc)}
        line["extras"] = extras
        line["cpu_baseline"] = cpu_baseline()
    elif ws > 1 and not args.quick:
        # the batched workload split over the ranks (node-balanced domains)
        res = run_batched(lbf, torch, compact=compact, ws=ws, rank=rank,
                          job_steps=args.job_steps)
        if rank == 0:
            line["extras"] = {"batched": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ------------------------------------------------------- reference arm
def reference(args):
    """The FP64 oracle on the host cores, on the same workload and metric;
    each step is one oracle step of the 512x512 cut."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    c = lbinputs.SPINODAL_8192
    n = c["sub"]
    lat = oracle.OracleLattice(oracle.params(**c["params"]), n, n)
    lat.init_random(c["amp"], c["seed"])
    lat.step(args.warmup)
    t0 = time.perf_counter()
    lat.step(args.steps)
    dt = time.perf_counter() - t0
    value = n * n * args.steps / dt / 1e6
    sample = "%dx%d cut of the 8192^2 spinodal MRT workload, %d FP64 steps" % (n, n, args.steps)
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS (MRT, FP32, 8192^2) and HBM-roofline fraction",
        "value": round(value, 3), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "spinodal 8192x8192 D2Q9 two-population MRT, walls y=0/8191, "
                               "seed 12345 (oracle runs the 512x512 cut)", "nx": 8192, "ny": 8192},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": oracle.get_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def experiment_ramp():
    """The paper's quasi-static ramp (Sec. IV): 300 x 100, drop R = 35 at
    90 degrees, a = kappa = 0.04, Gamma = 0.5, tau_alpha 3 / tau_beta 0.7;
    3e4 steps at h = 0, then h changed linearly over 1e6 steps towards
    h(160 deg) (up) or h(20 deg) (down), every 1000 steps, the angle read
    every 20000 steps; BGK, MRT and MRT with the relaxed Step-2 momentum.
    FP32 on the GPU; prints one JSON object per branch."""
    import paper_0812_1282_gb300 as lbf

    def theta_theory(h):
        # Eq. (theory) inverted by bisection on the library's monotone h(theta)
        lo, hi = 0.0, 180.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if lbf.lb_wetting_h(mid) < h:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    for coll, relax in (("mrt", False), ("mrt", True), ("bgk", False)):
        for direction, theta_end in (("up", 160.0), ("down", 20.0)):
            p = lbf.params(a=0.04, kappa=0.04, gamma_mob=0.5, tau_alpha=3.0, tau_beta=0.7,
                           collision=coll, precision="fp32", step2_relax_momentum=relax)
            sim = lbf.Lattice(p, 300, 100)
            sim.init_drop(35.0, 150.0, -0.5)
            sim.step(30000)
            h_end = lbf.lb_wetting_h(theta_end)
            rows, t, n = [], 0, 1000000
            while t < n:
                sim.step(1000)
                t += 1000
                h = h_end * t / n
                sim.set_wetting(h, 0.0)
                if t % 20000 == 0:
                    if sim.stats()["nonfinite"]:
                        rows.append([t, h, None])
                        break
                    rows.append([t, h, round(sim.contact_angle()[0], 3)])
            sim.close()
            print(json.dumps({"collision": coll, "step2_relax_momentum": relax,
                              "branch": direction,
                              "rows": [[r[0], round(r[1], 5), round(theta_theory(r[1]), 3),
                                        r[2]] for r in rows],
                              "columns": ["step", "h", "theta_theory", "theta_measured"]}),
                  flush=True)


def experiment_stripe():
    """The spurious-current stripe of Sec. IV.A: 28 x 15, a stripe of alpha
    across the channel between neutral walls, 20000 steps; BGK and MRT at
    tau 10 / 10 (the paper's case) and at the viscosity ratios 12.5 and 10,
    with mid-link walls and with node bounce-back walls (Fig. 4b: the same
    15 fluid rows between rows of wall nodes).
    Reports max |u| and the bulge of the stripe's edge (its x at mid-height
    less its x on the wall row; negative: barrel shaped), FP64 and FP32 on
    the GPU; prints one JSON object."""
    import numpy as np

    import paper_0812_1282_gb300 as lbf

    c = lbinputs.STRIPE_28x15
    cp = c["params"]
    ell = math.sqrt(2 * cp["kappa"] / cp["a"])
    x = np.arange(c["nx"], dtype=float)
    half = c["nx"] // 2
    prof = np.where(x < half, np.tanh((x - c["xa"]) / ell), -np.tanh((x - c["xb"]) / ell))
    phi0 = np.tile(prof, (c["ny"], 1))

    def left_edge(row):
        for i in range(1, row.size // 2):
            if row[i - 1] < 0.0 <= row[i]:
                return i - 1 + (-row[i - 1]) / (row[i] - row[i - 1])
        return float("nan")

    rows = []
    for walls in ("mid-link", "node"):
        for coll in ("bgk", "mrt"):
            for ta, tb in c["taus"]:
                for prec in ("fp64", "fp32"):
                    p = lbf.params(collision=coll, tau_alpha=ta, tau_beta=tb, precision=prec,
                                   **cp)
                    if walls == "node":
                        # the same 15 fluid rows between rows of wall nodes (Fig. 4b)
                        ny = c["ny"] + 2
                        sim = lbf.Lattice(p, c["nx"], ny)
                        cls = np.zeros((ny, c["nx"]), np.uint8)
                        cls[0] = cls[-1] = 8
                        sim.set_geometry(cls, [0.0])
                        sim.init_phi(np.tile(prof, (ny, 1)))
                        first = 1
                    else:
                        ny = c["ny"]
                        sim = lbf.Lattice(p, c["nx"], ny)
                        sim.init_phi(phi0)
                        first = 0
                    sim.step(c["steps"])
                    _, phi, ux, uy, st = sim.moments()
                    sim.close()
                    bulge = left_edge(phi[ny // 2]) - left_edge(phi[first])
                    rows.append([walls, coll, ta, tb, prec,
                                 float("%.4e" % np.hypot(ux, uy).max()), round(bulge, 4),
                                 int(st["nonfinite"])])
    print(json.dumps({"experiment": "stripe", "steps": c["steps"],
                      "columns": ["walls", "collision", "tau_alpha", "tau_beta", "precision",
                                  "max_u", "bulge", "nonfinite"], "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--quick", action="store_true", help="headline line only")
    ap.add_argument("--size", type=int, default=None,
                    help="side of a smaller square lattice (profiling aid; default 8192)")
    ap.add_argument("--tile", default=None,
                    help="fixed launch shape BXxROWS instead of autotuning (profiling aid)")
    ap.add_argument("--storage", choices=("full", "compact"), default="compact",
                    help="g storage of the headline lattice (compact: phi, Gamma mu, u_eq)")
    ap.add_argument("--only", choices=("batched", "capillary", "fp64"), default=None,
                    help="run one extra workload alone for --steps steps (profiling aid)")
    ap.add_argument("--job-steps", type=int, default=None,
                    help="steps of the batched job (profiling aid; default 10000)")
    ap.add_argument("--schedule", choices=("auto", "ladder", "ladder-persist"), default="auto",
                    help="batched job: autotuned schedule, or the fixed eight-class ladder "
                         "(one launch per class per step, or per class per graph of "
                         "persistent launches; profiling aid: no autotuning launches)")
    ap.add_argument("--experiment", choices=("ramp", "stripe"), default=None,
                    help="run a physics experiment instead of the benchmark and print its "
                         "JSON table (ramp: the quasi-static wetting ramp of Sec. IV; stripe: "
                         "the spurious-current stripe of Sec. IV.A)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.experiment == "ramp":
        experiment_ramp()
    elif args.experiment == "stripe":
        experiment_stripe()
    elif args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
