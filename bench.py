#!/usr/bin/env python3
"""Benchmark of the ES-DG Euler + buoyancy hot path on GB300.

Workload: rising thermal bubble on 32 x 32 x 32 hexahedra at N = 4 (4,096,000
LGL nodes) on the smoothly warped 1000 m cube (periodic x, y; walls z), 0.5 K
cosine bubble, dt from CFL 0.5.  A step is one LSRK(5,4) time step: five
stages, each one interface-flux launch and one volume launch with the RK update
fused in.  Metric: DOF-updates per second per RK stage = nodes * 5 * steps / s.

The JSON line reports the FP64 path as the headline and the mixed-precision
path (FP32 pairs, FP64 state) next to it; the roofline object is the FP64
volume kernel's achieved algorithmic FLOP rate (events around every volume
launch of the timed region) against the FP64 vector peak; e2e is the same
metric through the C ABI with pinned host buffers copied in and out every step.
At one GPU the line also carries the other two halves of the metric: "ensemble"
(64 heterogeneous rising-bubble members, 100 steps, batched in mixed precision:
DOF-updates/s, p50/p99 solve latency, speed-up over the same members solved one
after another in plain FP64, per-variable error against those FP64 solves) and
"serving" (a Poisson stream of the serving workload's requests at 8x the
sequential-FP64 service rate: p50/p99 latency, throughput and its ratio to
sequential FP64).

Multi-GPU (torchrun): every rank advances its own replica (ensemble members are
independent, no data-path collective); value = all ranks' DOF-updates / max time.

--impl reference times the CPU oracle (single-threaded C, as it stands) on a
bounded sample of the same workload (8 x 8 x 8 elements, same N, mesh and
physics), one LSRK step per timed step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(K=(32, 32, 32), N=4, lo=(0.0, 0.0, 0.0), hi=(1000.0, 1000.0, 1000.0),
                periodic=(1, 1, 0), warp=0.05, theta0=300.0, amp=0.5,
                centre=(500.0, 500.0, 350.0), radius=250.0, cfl=0.5)
WORKLOAD_NAME = "rising_bubble_32x32x32_N4_warped"
SAMPLE_K = (8, 8, 8)
METRIC = "DOF-updates/s per RK stage"
UNIT = "DOF-updates/s"

# Algorithmic work of the volume kernel, counted from the oracle's own arithmetic by
# its counting instantiation (oracle/count_flops.cpp; tests/test_flop_count.py holds
# these constants to the counts, the same for every order): per unordered node pair of
# the half sweep 114 flops (both orderings of the oracle's pair term, the symmetric
# two-point flux, log means and metric average once, the gravity term and the
# accumulation for each node); per node and stage 56 (primitives 16, and for each of
# the five values its volume value and stage update).  The kernel itself executes
# fewer: 100 per pair and 45 per node in its regrouped arithmetic (FMA = 2 flops).
FLOPS_PER_PAIR = 114
FLOPS_PER_NODE = 56
KERNEL_FLOPS_PER_PAIR = 100
KERNEL_FLOPS_PER_NODE = 45
# Algorithmic bytes of the interface kernel per face node (FP64): two traces
# (2 x 40 B), face geometry (40 B) and the flux write (40 B); RK state traffic
# is fused into the volume kernel.
FACE_BYTES_PER_NODE = {"fp64": 160, "mixed": 140}
# Algorithmic bytes of the mixed volume kernel per node: FP64 state in and out
# (2 x 40 B), FP32 increment in and out (2 x 20 B), FP32 geometry (11 x 4 B), the
# background (3 FP64 + 4 FP32 values) and its FP32 momentum rhs (3 x 4 B), and
# the FP32 face fluxes of the element's six faces (6 x 5 x 4 B per face node,
# i.e. 6 N_q^2 / N_q^3 of them per node).
def mixed_volume_bytes_per_node(N):
    nq = N + 1
    return 2 * 40 + 2 * 20 + 11 * 4 + (3 * 8 + 4 * 4) + 3 * 4 + 6 * 5 * 4 * nq * nq / nq ** 3

# DRAM traffic of one FP64 volume launch (k_volume_pipe64<4, 1, 0>): ncu capture of the same
# kernel on the 24^3 case (dram__bytes_read.sum + dram__bytes_write.sum = 332.80 MB +
# 99.38 MB for 13 824 elements), scaled to the 32^3 launch by the element count.
VOLUME_FP64_TRAFFIC_BYTES = (332.80e6 + 99.38e6) * 32768 / 13824

# Vector issue rates of the part (per SM and clock): 2 FP64 FMA, 128 FP32 FMA.
DFMA_PER_CLK_SM, FFMA_PER_CLK_SM = 2, 128


def device_peaks(device=0):
    """FP64 / FP32 vector peaks (FLOP/s) from the device's SM count and maximum SM
    clock: the SM count from the CUDA device properties, the clock from nvidia-smi's
    clocks.max.sm (a read-only query), else MEASURED_PEAKS.json's sm_max_mhz."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz, src = None, "nvidia-smi clocks.max.sm"
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(device), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip().splitlines()
        mhz = float(out[0])
    except Exception:
        peaks, _ = measured_peaks()
        mhz, src = float(peaks.get("sm_max_mhz", 2070.0)), "MEASURED_PEAKS.json sm_max_mhz"
    hz = mhz * 1e6
    return {"sms": sms, "sm_max_mhz": mhz, "clock_source": src,
            "fp64": sms * hz * DFMA_PER_CLK_SM * 2, "fp32": sms * hz * FFMA_PER_CLK_SM * 2}


def hbm_block(r64, r32, N, hbm_gbs):
    """Achieved HBM bandwidth of the memory-side kernels from their algorithmic bytes
    (the interface kernels per face node, the mixed volume kernel per node) over their
    CUDA-event durations, against the measured copy bandwidth."""
    def entry(nbytes, ms):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"gbs": gbs, "frac": gbs / hbm_gbs, "bytes": nbytes, "ms": ms}
    return {"peak_gbs": hbm_gbs, "unit": "GB/s (algorithmic bytes / event time)",
            "interface_fp64": entry(r64["face_nodes"] * FACE_BYTES_PER_NODE["fp64"], r64["t_face"]),
            "interface_mixed": entry(r32["face_nodes"] * FACE_BYTES_PER_NODE["mixed"], r32["t_face"]),
            "volume_mixed": entry(r32["ndof"] * mixed_volume_bytes_per_node(N), r32["t_vol"])}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def max_over_ranks(x, dist, device="cuda"):
    """The job time of a replica run: the slowest rank's (all-reduce MAX).  dist is
    torch.distributed (NCCL on the GPU box, gloo with device="cpu" in tests) or None."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, ndof, steps, seconds):
    """DOF-updates/s per RK stage of `world` independent replicas timed together: each
    advances ndof nodes through 5 stages per step; the job time is the slowest rank's."""
    return world * ndof * 5 * steps / seconds


def pairs_per_element(N):
    Nq = N + 1
    return 3 * Nq * Nq * Nq * (Nq - 1) // 2


def volume_flops(E, N, per_pair=FLOPS_PER_PAIR, per_node=FLOPS_PER_NODE):
    return E * (pairs_per_element(N) * per_pair + (N + 1) ** 3 * per_node)


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ our GPU arm --

def run_gpu_arm(args, rank, world, dist):
    import numpy as np
    import torch

    from paper_2605_16684_gb300 import _build, _lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    _build.build()
    w = WORKLOAD
    stream = torch.cuda.current_stream()
    results = {}
    sampler = None
    precs = ("fp64", "mixed") if args.precision == "both" else (args.precision,)
    for prec in precs:
        s = _lib.Solver(*w["K"], w["N"], lo=w["lo"], hi=w["hi"], periodic=w["periodic"],
                        warp=w["warp"], precision=prec, stream=stream)
        info = s.info()
        s.init_bubble(w["theta0"], w["amp"], w["centre"], w["radius"])
        dt = s.cfl_dt(w["cfl"])
        # warm-up steps through the same stage launches as the timed region
        for _ in range(args.warmup):
            for st in range(5):
                s.launch(0)
                s.launch(2, st, dt)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)]
              for _ in range(5 * args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if prec == precs[0]:
            sampler = ClockSampler(local)
            time.sleep(0.3)
        t0.record(stream)
        k = 0
        for _ in range(args.steps):
            for st in range(5):
                ev[k][0].record(stream)
                s.launch(0)
                ev[k][1].record(stream)
                s.launch(2, st, dt)
                ev[k][2].record(stream)
                k += 1
        t1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if prec == precs[0] else None
        ms = t0.elapsed_time(t1)
        t_face = sum(e[0].elapsed_time(e[1]) for e in ev) / len(ev)
        t_vol = sum(e[1].elapsed_time(e[2]) for e in ev) / len(ev)
        ms = max_over_ranks(ms, dist)
        # e2e: the C-ABI call with host buffers, copies inside the timed region
        qh = torch.empty(s.shape(), dtype=torch.float64, pin_memory=True)
        s.get_state(qh)
        e2e_steps = max(1, min(args.steps, 5))
        s.set_state(qh)
        s.step(dt, 1)
        s.get_state(qh)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        te = time.perf_counter()
        for _ in range(e2e_steps):
            s.set_state(qh)
            s.step(dt, 1)
            s.get_state(qh)
        torch.cuda.synchronize()
        te = time.perf_counter() - te
        te = max_over_ranks(te, dist)
        q = qh.numpy()
        finite = bool(np.isfinite(q).all())
        ndof = info.ndof
        results[prec] = dict(ms=ms, t_face=t_face, t_vol=t_vol, ndof=ndof, dt=dt,
                             e2e_s=te, e2e_steps=e2e_steps, clocks=clocks, finite=finite,
                             state_bytes=ndof * 5 * 8, E=info.nelem,
                             face_nodes=info.nfaces * info.Nq * info.Nq)
        s.close()
        del qh
    return results


def cpu_sample(seconds_target=10.0):
    """The oracle, as it stands, single-threaded, on a bounded sample."""
    import oracle as O
    w = WORKLOAD
    o = O.Oracle(*SAMPLE_K, w["N"], lo=w["lo"], hi=w["hi"], periodic=w["periodic"], warp=w["warp"])
    q = o.bubble(w["theta0"], w["amp"], w["centre"], w["radius"])
    dt = o.cfl_dt(q, w["cfl"])
    ndof = o.E * o.np
    t = time.perf_counter()
    stages = 0
    while True:
        q = o.steps(q, dt, 1)
        stages += 5
        el = time.perf_counter() - t
        if el >= seconds_target:
            break
    return dict(value=ndof * stages / el, unit=UNIT, cores=1, kind="oracle",
                sample=f"{SAMPLE_K[0]}x{SAMPLE_K[1]}x{SAMPLE_K[2]} elements of the same warped "
                       f"bubble at N={w['N']} ({ndof} nodes), {stages // 5} LSRK steps, "
                       f"single-threaded C oracle in FP64, {el:.1f} s")


def config_block(extra=None):
    w = WORKLOAD
    c = {"workload": WORKLOAD_NAME, "elements": w["K"][0] * w["K"][1] * w["K"][2], "N": w["N"],
         "dof": w["K"][0] * w["K"][1] * w["K"][2] * (w["N"] + 1) ** 3,
         "mesh": "1000 m cube, warp 0.05 L, periodic x/y, walls z",
         "initial_state": "0.5 K cosine bubble r=250 m at (500,500,350) m over theta0=300 K",
         "dt": "CFL 0.5", "step": "one LSRK(5,4) step = 5 stages x (interface + volume/RK)",
         "l2": "working set ~1 GB per stage > 129 MB L2 (no flush needed)",
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


def main_ours(args):
    dist = None
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    if args.K:
        WORKLOAD["K"] = (args.K, args.K, args.K)
    res = run_gpu_arm(args, rank, world, dist)
    if args.precision != "both":
        # single-precision small cases (profiling runs): short report only
        if rank == 0:
            r = res[args.precision]
            print(json.dumps({"precision": args.precision, "K": WORKLOAD["K"],
                              "ms_per_step": r["ms"] / args.steps, "ms_interface": r["t_face"],
                              "ms_volume": r["t_vol"], "finite": r["finite"]}))
        if dist is not None:
            dist.destroy_process_group()
        return
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks, peak_src = measured_peaks()
    dev = device_peaks(int(os.environ.get("LOCAL_RANK", "0")))
    FP64_PEAK, FP32_PEAK = dev["fp64"], dev["fp32"]
    r64, r32 = res["fp64"], res["mixed"]
    w = WORKLOAD
    value = replica_throughput(world, r64["ndof"], args.steps, r64["ms"] * 1e-3)
    value32 = replica_throughput(world, r32["ndof"], args.steps, r32["ms"] * 1e-3)
    vflops = volume_flops(r64["E"], w["N"])
    achieved = vflops / (r64["t_vol"] * 1e-3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block({"precision": "fp64"}),
        "roofline": {"bound": "alu", "kernel": "volume (flux differencing + lift + RK), FP64",
                     "achieved": achieved / 1e12, "peak": FP64_PEAK / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK,
                     "traffic": VOLUME_FP64_TRAFFIC_BYTES if w["K"] == (32, 32, 32) else None,
                     "peak_source": f"{dev['sms']} SMs x {DFMA_PER_CLK_SM} DFMA/clk x "
                                    f"{dev['sm_max_mhz']:.0f} MHz ({dev['clock_source']}); the "
                                    "recipe's nominal FP64 rate is 1.25 TFLOP/s",
                     "flops_per_launch": vflops, "ms_per_launch": r64["t_vol"],
                     "flop_count": "algorithmic, counted from the oracle: 114 per unordered "
                                   "node pair, 56 per node and stage",
                     "kernel_executed_frac": volume_flops(r64["E"], w["N"], KERNEL_FLOPS_PER_PAIR,
                                                          KERNEL_FLOPS_PER_NODE)
                     / (r64["t_vol"] * 1e-3) / FP64_PEAK},
        "kernels_ms_per_stage": {"fp64": {"interface": r64["t_face"], "volume_rk": r64["t_vol"]},
                                 "mixed": {"interface": r32["t_face"], "volume_rk": r32["t_vol"]}},
        "hbm": hbm_block(r64, r32, w["N"], float(peaks.get("hbm_gbs", 6800.0))),
        "mixed": {"value": value32, "unit": UNIT, "dtype": "f32 pairs, f64 state",
                  "ms_per_step": r32["ms"] / args.steps,
                  "volume_fp32_tflops": vflops / (r32["t_vol"] * 1e-3) / 1e12,
                  "volume_fp32_frac": vflops / (r32["t_vol"] * 1e-3) / FP32_PEAK,
                  "speedup_vs_fp64": value32 / value,
                  "e2e": {"value": replica_throughput(world, r32["ndof"], r32["e2e_steps"],
                                                      r32["e2e_s"]),
                          "unit": UNIT}},
        "e2e": {"value": replica_throughput(world, r64["ndof"], r64["e2e_steps"], r64["e2e_s"]),
                "unit": UNIT,
                "h2d_bytes_per_step": r64["state_bytes"], "d2h_bytes_per_step": r64["state_bytes"],
                "steps": r64["e2e_steps"]},
        "gpu_launches": 10 * args.steps,
        "clocks": r64["clocks"],
        "finite": r64["finite"] and r32["finite"],
        "peaks_source": peak_src,
    }
    if not args.no_cpu_baseline and world >= 1:
        out["cpu_baseline"] = cpu_sample(args.cpu_seconds)
    if world == 1 and not args.no_ensemble:
        # the batched-ensemble and serving halves of the metric (single-GPU measurements)
        out["ensemble"] = ensemble_measure(args.members, ENSEMBLE_STEPS)
        out["serving"] = serving_measure(SERVING_DEFAULT["requests"], SERVING_DEFAULT["steps"],
                                         SERVING_DEFAULT["rates"], SERVING_DEFAULT["calib"],
                                         args.slots, args.budget_gb,
                                         check=SERVING_DEFAULT["check"])
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle as O
    w = WORKLOAD
    o = O.Oracle(*SAMPLE_K, w["N"], lo=w["lo"], hi=w["hi"], periodic=w["periodic"], warp=w["warp"])
    q = o.bubble(w["theta0"], w["amp"], w["centre"], w["radius"])
    dt = o.cfl_dt(q, w["cfl"])
    for _ in range(args.warmup):
        q = o.steps(q, dt, 1)
    t = time.perf_counter()
    for _ in range(args.steps):
        q = o.steps(q, dt, 1)
    el = time.perf_counter() - t
    ndof = o.E * o.np
    value = ndof * 5 * args.steps / el
    sample = (f"{SAMPLE_K[0]}x{SAMPLE_K[1]}x{SAMPLE_K[2]} elements of the 32^3 workload's warped "
              f"bubble at N={w['N']} ({ndof} nodes), one LSRK step per timed step, "
              f"single-threaded C oracle in FP64")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_block({"precision": "fp64", "sample": sample}),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ----------------------------------------------------- ensemble and serving --

def _sequential(req, precision):
    """One request solved alone through the single-handle C ABI; returns
    (stepping seconds, ndof, final state)."""
    import torch
    from paper_2605_16684_gb300 import _lib
    if req["kind"] == "bubble":
        s = _lib.Solver(*req["K"], req["N"], precision=precision, warp=req.get("warp", 0.0))
        s.init_bubble(300.0, req.get("amp", 0.5), req.get("centre", (500.0, 500.0, 350.0)), 250.0)
    else:
        s = _lib.Solver(*req["K"], req["N"], lo=(0, 0, 0), hi=(40000e3, 6000e3, 30e3),
                        periodic=(1, 0, 0), precision=precision, f0=1e-4)
        s.init_channel()
    dt = s.cfl_dt(req.get("cfl", SERVER_CFL))
    torch.cuda.synchronize()
    t = time.perf_counter()
    s.step(dt, req["nsteps"])
    s.sync()
    el = time.perf_counter() - t
    q = s.get_state()
    nd = s.E * s.np
    s.close()
    return el, nd, q


def _pct(x, p):
    import numpy as np
    return float(np.percentile(np.asarray(x), p)) if len(x) else None


ENSEMBLE_STEPS = 100  # the batched-ensemble workload's step count
# Courant number of the batched workloads (their definition gives none): the server's
# default, 0.4 -- C = 0.5 is on the stability boundary for unwarped meshes at N >= 4
SERVER_CFL = 0.4


def _state_errors(q, q_ref):
    """Relative L2 error per variable (rho, rho u, rho v, rho w, E) of a final state,
    the momentum components against the norm of the momentum vector (a rising
    bubble starts at rest, so a single component's norm is that of the flow's
    smallest part)."""
    import numpy as np
    q, q_ref = q.reshape(q_ref.shape), q_ref
    mom = np.sqrt(sum(np.linalg.norm(q_ref[:, v]) ** 2 for v in (1, 2, 3)))
    return [float(np.linalg.norm(q[:, v] - q_ref[:, v]) /
                  (mom if v in (1, 2, 3) else np.linalg.norm(q_ref[:, v]))) for v in range(5)]


def ensemble_measure(n_members, steps):
    """Config 3: n_members rising-bubble members (K^3, K ~ U{8..24}, N ~ U{3,4,7},
    amplitude ~ U(0.25, 1) K, centre jitter +-100 m, one seed) solved together by the
    server in mixed precision (one persistent interface + volume launch per order group
    and stage, one CUDA-graph replay per step), the autotuner warmed first.  Then every
    member solved alone in plain FP64 through the single-handle path: the speed-up is
    measured on the same solves, and each member's final mixed state is compared with
    its FP64 state, per variable."""
    import numpy as np
    import torch
    from paper_2605_16684_gb300 import _build, _lib, inputs
    _build.build()
    torch.cuda.init()
    members = inputs.ensemble_members(n_members)
    reqs = [dict(kind="bubble", K=(m["K"],) * 3, N=m["N"], amp=m["amp"], centre=m["centre"],
                 nsteps=steps) for m in members]
    srv = _lib.Server(hbm_budget_bytes=200 << 30, max_slots=len(reqs))
    tw = time.perf_counter()
    srv.warmup((3, 4, 7), "mixed")
    warm_s = time.perf_counter() - tw
    t0 = time.perf_counter()
    tickets = [srv.submit(precision="mixed", **r) for r in reqs]
    res = [srv.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res), stats["error"]
    dof_updates = sum(r["ndof"] * 5 * r["nsteps"] for r in res)
    run = max(r["t_finish"] for r in res) - max(r["t_admit"] for r in res)
    lat = [r["t_finish"] - r["t_submit"] for r in res]
    seq_t, errs = 0.0, []
    for i, r in enumerate(reqs):
        el, nd, q64 = _sequential(r, "fp64")
        seq_t += el
        errs.append(_state_errors(res[i]["q"], q64))
    errs = np.array(errs)
    value = dof_updates / run
    return {"metric": "ensemble DOF-updates/s per RK stage; p50/p99 solve latency",
            "value": value, "unit": UNIT, "steps": steps,
            "config": {"workload": f"batched_ensemble_{len(reqs)}_bubbles", "members": len(reqs),
                       "grids": "K^3, K ~ U{8..24}", "orders": "N ~ U{3,4,7}",
                       "precision": "mixed (FP32 pairs, FP64 state)",
                       "launches": "one persistent interface + volume launch per order group and "
                                   "stage, one LSRK step per CUDA graph replay"},
            "latency_p50_s": _pct(lat, 50), "latency_p99_s": _pct(lat, 99),
            "batched_run_seconds": run, "wall_seconds_incl_admission": wall,
            "autotuner_warmup_seconds": warm_s,
            "sequential_fp64_value": dof_updates / seq_t,
            "speedup_vs_sequential_fp64": value / (dof_updates / seq_t),
            "mixed_vs_fp64_state_rel_err_max_over_members": {
                k: float(errs[:, v].max()) for v, k in enumerate(("rho", "rho_u", "rho_v",
                                                                   "rho_w", "E"))},
            "members_within_1e-4": int((errs.max(axis=1) <= 1e-4).sum()),
            "server_steps": stats["steps"]}


def run_ensemble(args):
    steps = args.steps if args.steps_given else ENSEMBLE_STEPS
    print(json.dumps(ensemble_measure(args.members, steps)))


CHANNEL = dict(K=(120, 24, 12), N=4, lo=(0.0, 0.0, 0.0), hi=(40000e3, 6000e3, 30e3),
               periodic=(1, 0, 0), f0=1e-4, cfl=0.5)


def run_channel(args):
    """The channel configuration: mixed precision against plain FP64 on the GPU over
    `steps` LSRK steps (the FP64 path is the oracle-matched one: parity tests hold its
    right-hand sides to the CPU oracle; the oracle itself would need ~2 h for 500 steps of
    this mesh).  Reports per-variable relative errors of the state and of the flow (state
    minus initial state, momentum as one vector), relative drift of mass and total energy
    for both precisions, and DOF-updates/s per RK stage; the mixed path twice, with the
    channel state at rest as background and with the balanced jet as a moving background."""
    import numpy as np
    import torch
    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    c = CHANNEL
    res = {}
    dt = None
    for case in ("fp64", "mixed", "jet"):
        prec = "fp64" if case == "fp64" else "mixed"
        s = _lib.Solver(*c["K"], c["N"], lo=c["lo"], hi=c["hi"], periodic=c["periodic"],
                        precision=prec, f0=c["f0"])
        s.init_channel(background="jet" if case == "jet" else "rest")
        q0 = s.get_state()
        if dt is None:
            dt = s.cfl_dt(c["cfl"])
        i0 = s.integrals()
        s.step(dt, 2)  # warm-up (state re-set below)
        s.set_state(q0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        s.step(dt, args.steps)
        s.sync()
        el = time.perf_counter() - t
        i1 = s.integrals()
        q = s.get_state()
        res[case] = dict(q=q, q0=q0, s=el, ndof=s.E * s.np,
                         drift=[float((i1[k] - i0[k]) / abs(i0[k])) for k in (0, 1)])
        s.close()
    q64, q0 = res["fp64"]["q"], res["fp64"]["q0"]
    f64 = q64 - q0
    mom = np.sqrt(sum(np.linalg.norm(f64[:, v]) ** 2 for v in (1, 2, 3)))

    def errors(q32):
        state = [float(np.linalg.norm(q32[:, v] - q64[:, v]) / np.linalg.norm(q64[:, v]))
                 for v in range(5)]
        f32 = q32 - q0
        flow = [float(np.linalg.norm(f32[:, v] - f64[:, v]) /
                      (mom if v in (1, 2, 3) else np.linalg.norm(f64[:, v]))) for v in range(5)]
        return state, flow

    state_err, flow_err = errors(res["mixed"]["q"])
    state_jet, flow_jet = errors(res["jet"]["q"])
    out = {"metric": "channel: mixed vs FP64 per-variable error, conservation drift, "
                     "DOF-updates/s per RK stage",
           "unit": "relative / DOF-updates/s", "n_gpus": 1, "steps": args.steps, "dt_s": dt,
           "config": {"workload": "baroclinic_channel_120x24x12_N4", "box_km": [40000, 6000, 30],
                      "boundaries": "periodic x, walls y and z", "f0": c["f0"],
                      "initial_state": "balanced zonal jet (synthetic stand-in) + 1 m/s "
                                       "Gaussian wind perturbation",
                      "reference": "FP64 GPU path (RHS parity with the CPU oracle <= 1e-12)"},
           "state_rel_err_rho_rhou_rhov_rhow_E": state_err,
           "flow_rel_err_rho_rhou_rhov_rhow_E": flow_err,
           "jet_background": {"state_rel_err_rho_rhou_rhov_rhow_E": state_jet,
                              "flow_rel_err_rho_rhou_rhov_rhow_E": flow_jet,
                              "mass_energy_drift": res["jet"]["drift"],
                              "value": res["jet"]["ndof"] * 5 * args.steps / res["jet"]["s"]},
           "mass_energy_drift_fp64": res["fp64"]["drift"],
           "mass_energy_drift_mixed": res["mixed"]["drift"],
           "fp64_value": res["fp64"]["ndof"] * 5 * args.steps / res["fp64"]["s"],
           "mixed_value": res["mixed"]["ndof"] * 5 * args.steps / res["mixed"]["s"]}
    print(json.dumps(out))


SHARP = dict(K=(64, 64, 64), N=4, lo=(-1000.0, -1000.0, 0.0), hi=(1000.0, 1000.0, 2000.0),
             periodic=(1, 1, 0), centre=(0.0, 0.0, 260.0), radius=250.0, amp=0.5, cfl=0.5)
# Section 5.1, Table rb-timing: 8 A100s, N = 4, 64^3 elements, sharp bubble:
# 6622.03 s (64-bit) and 3070.25 s (32-bit) for the whole run
PAPER_SHARP_SPEEDUP_32_OVER_64 = 6622.03 / 3070.25


def _mirror_x(q, K, N):
    """State under x -> -x on a uniform box mesh (x-momentum negated)."""
    Nq = N + 1
    a = q.reshape(K[2], K[1], K[0], 5, Nq, Nq, Nq).flip(2).flip(6).clone()
    a[:, :, :, 1] *= -1
    return a.reshape(q.shape)


def lgl_weights(N):
    """Legendre-Gauss-Lobatto weights 2 / (N (N + 1) P_N(x_i)^2), nodes +-1 and the roots
    of P_N' (for the entropy integral of the measurement only)."""
    import numpy as np
    from numpy.polynomial import legendre as Lg
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    x = np.concatenate([[-1.0], np.sort(np.real(Lg.legroots(Lg.legder(cN)))), [1.0]])
    return 2.0 / (N * (N + 1) * Lg.legval(x, cN) ** 2)


def _entropy_change(q, q0, x, wJ, gamma=1.4, g=9.81):
    """sum_i w_i J_i (eta(q_i) - eta(q0_i)), eta = -rho (ln p - gamma ln rho)/(gamma - 1),
    node by node (unchanged nodes add exactly zero; the integral's own rounding would
    hide changes below 1e-16 of the total)."""
    import torch

    def eta(q):
        rho = q[:, 0]
        p = (gamma - 1) * (q[:, 4] - 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2 + q[:, 3] ** 2) / rho
                           - rho * g * x[:, 2])
        return -rho * (torch.log(p) - gamma * torch.log(rho)) / (gamma - 1)
    return float((wJ * (eta(q) - eta(q0))).sum())


def run_sharp(args):
    """The paper's rising-bubble run with the sharp initial perturbation (Section 5.1,
    Eq. (sharp-rb-ic)): 2000 m box, periodic x and y, walls z, 64^3 elements at N = 4
    (32,768,000 nodes, the paper's L = 6 mesh), on one GPU in FP64 and in mixed precision.
    Reports DOF-updates/s per RK stage of both and their ratio (the paper's 32-bit run was
    2.16x its 64-bit run on 8 A100s), the entropy change and the mass / total-energy drift
    over the run, and the mirror asymmetry of the flow under x -> -x, which the exact
    solution does not have (the paper's figures show FP32 losing the symmetry)."""
    import torch
    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    c = SHARP
    K = (args.K,) * 3 if args.K else c["K"]
    res = {}
    for prec in ("fp64", "mixed"):
        s = _lib.Solver(*K, c["N"], lo=c["lo"], hi=c["hi"], periodic=c["periodic"],
                        precision=prec)
        s.init_bubble(amp=c["amp"], centre=c["centre"], radius=c["radius"], profile="sharp")
        q0 = torch.empty(s.shape(), dtype=torch.float64, device="cuda")
        s.get_state(q0)
        dt = s.cfl_dt(c["cfl"])
        s.step(dt, 2)  # warm-up, then back to the initial state
        s.set_state(q0)
        i0 = s.integrals()
        s.sync()
        torch.cuda.synchronize()
        t = time.perf_counter()
        s.step(dt, args.steps)
        s.sync()
        el = time.perf_counter() - t
        i1 = s.integrals()
        q = torch.empty_like(q0)
        s.get_state(q)
        s.sync()
        torch.cuda.synchronize()
        f = q - q0
        asym = float(torch.linalg.vector_norm(q - _mirror_x(q, K, c["N"])) /
                     torch.linalg.vector_norm(f))
        x, J, _ = s.geometry(device=True)
        w = torch.tensor(lgl_weights(c["N"]), dtype=torch.float64, device="cuda")
        w3 = torch.einsum("k,j,i->kji", w, w, w).reshape(-1)
        dS = _entropy_change(q, q0, x, w3[None, :] * J)
        S0 = float(i0[2])
        del x, J
        res[prec] = dict(value=s.E * s.np * 5 * args.steps / el, seconds=el, dt=dt,
                         drift=[float((i1[k] - i0[k]) / abs(i0[k])) for k in (0, 1)],
                         entropy_change_rel=dS / abs(S0),
                         mirror_asymmetry=asym, q=q, q0=q0)
        s.close()
    d = res["mixed"]["q"] - res["fp64"]["q"]
    f = res["fp64"]["q"] - res["fp64"]["q0"]
    mom = torch.linalg.vector_norm(f[:, 1:4])
    flow_err = [float(torch.linalg.vector_norm(d[:, v]) /
                      (mom if v in (1, 2, 3) else torch.linalg.vector_norm(f[:, v])))
                for v in range(5)]
    out = {"metric": "sharp rising bubble: DOF-updates/s per RK stage (FP64, mixed), "
                     "entropy and conservation monitors, mirror asymmetry",
           "unit": "DOF-updates/s", "n_gpus": 1, "steps": args.steps,
           "config": {"workload": "sharp_rising_bubble_%dx%dx%d_N4" % K,
                      "box_m": [2000, 2000, 2000], "boundaries": "periodic x/y, walls z",
                      "perturbation": "theta + 0.5 K for r <= 250 m about (0, 0, 260) m",
                      "cfl": c["cfl"], "data": "synthetic"},
           "dt_s": res["fp64"]["dt"],
           "fp64": {k: v for k, v in res["fp64"].items() if k not in ("q", "q0")},
           "mixed": {k: v for k, v in res["mixed"].items() if k not in ("q", "q0")},
           "mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"],
           "paper_fp32_over_fp64_8xA100": PAPER_SHARP_SPEEDUP_32_OVER_64,
           "flow_rel_err_mixed_vs_fp64_rho_rhou_rhov_rhow_E": flow_err}
    print(json.dumps(out))


def run_slabs(args):
    """The 32^3 N = 4 bubble cut into P slabs of x layers on one GPU (domain
    decomposition: trace pack, device copies and the two launches per slab and stage)
    against the whole mesh: DOF-updates/s per RK stage per P and precision, and a check
    that the slabs' final state equals the whole mesh's bit for bit."""
    import numpy as np
    import torch
    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    w = WORKLOAD
    K = (args.K,) * 3 if args.K else w["K"]
    res = {}
    for prec in ("fp64", "mixed"):
        ref = None
        for P in (1, 2, 4, 8):
            s = _lib.PartitionedSolver(*K, w["N"], P=P, precision=prec, lo=w["lo"], hi=w["hi"],
                                       periodic=w["periodic"], warp=w["warp"])
            s.init_bubble(theta0=w["theta0"], amp=w["amp"], centre=w["centre"],
                          radius=w["radius"])
            dt = s.cfl_dt(w["cfl"])
            s.step(dt, args.warmup)
            s.sync()
            torch.cuda.synchronize()
            t = time.perf_counter()
            s.step(dt, args.steps)
            s.sync()
            el = time.perf_counter() - t
            q = s.get_state()
            if ref is None:
                ref = q
            res.setdefault(prec, []).append(
                {"slabs": P, "value": s.E * s.np * 5 * args.steps / el,
                 "ms_per_step": 1e3 * el / args.steps, "equal_to_whole": bool(np.array_equal(q, ref))})
            s.close()
    out = {"metric": "domain decomposition on one GPU: DOF-updates/s per RK stage by slab count",
           "unit": "DOF-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "config": {"workload": WORKLOAD_NAME + "_x_slabs", "slabs": "x element layers",
                      "exchange": "pack kernel + one device copy per cut plane and stage; "
                                  "one stream per slab ordered by events, one LSRK step "
                                  "captured as a CUDA graph and replayed"},
           "fp64": res["fp64"], "mixed": res["mixed"]}
    print(json.dumps(out))


# The serving line of the default run: a reduced stream of the serving workload
# (its request mix and 200 steps per request; 24 requests instead of 2000) at one
# offered rate, 8x what sequential plain FP64 solves can serve, so the server runs
# saturated and its throughput is its capacity.  --workload serving runs the rate sweep.
SERVING_DEFAULT = dict(requests=24, steps=200, rates=(8.0,), calib=6, check=2)


def serving_measure(n_requests, steps, rates, calib, slots, budget_gb, check=0):
    """Serving workload: Poisson streams of n_requests solve requests (70 % rising
    bubbles K^3, K ~ U{8..32}; 30 % channels (40s, 8s, 4s), s ~ U[1,3]; N ~ U{3,4,7};
    `steps` LSRK steps each) submitted by a client thread at each offered rate (a
    multiple of the sequential plain-FP64 service rate) to a server in mixed
    precision (FIFO admission by HBM footprint, continuous batching), autotuner warmed.
    The sequential FP64 rate is measured on the first `calib` requests of the stream
    (single-handle solves, 20 steps each: DOF-updates/s does not depend on the step
    count); the service rate follows from the stream's mean work per request.  The
    `check` smallest requests are also solved alone in FP64 for their full step count
    and compared with their served results, per variable."""
    import threading
    import numpy as np
    import torch
    from paper_2605_16684_gb300 import _build, _lib, inputs
    _build.build()
    torch.cuda.init()
    base = inputs.request_stream(n_requests, 1.0, seed=inputs.DEFAULT_SEED + 1, steps=steps)
    cal_t = cal_dof = 0.0
    for r in base[:calib]:
        el, nd, _ = _sequential(dict(r, nsteps=20), "fp64")
        cal_t += el
        cal_dof += nd * 5 * 20
    seq_value = cal_dof / cal_t

    def work(r):
        Nq = r["N"] + 1
        return r["K"][0] * r["K"][1] * r["K"][2] * Nq ** 3 * 5 * r["steps"]

    mean_work = float(np.mean([work(r) for r in base]))
    seq_rate = seq_value / mean_work  # requests/s that sequential FP64 solves can serve
    points = []
    for mult in rates:
        rate = mult * seq_rate
        stream = inputs.request_stream(n_requests, rate, seed=inputs.DEFAULT_SEED + 1, steps=steps)
        srv = _lib.Server(hbm_budget_bytes=budget_gb << 30, max_slots=slots)
        srv.warmup((3, 4, 7), "mixed")
        tickets = [None] * len(stream)

        def submitter():
            start = time.perf_counter()
            for i, r in enumerate(stream):
                d = r["arrival"] - (time.perf_counter() - start)
                if d > 0:
                    time.sleep(d)
                kw = dict(kind=r["kind"], K=r["K"], N=r["N"], nsteps=r["steps"], precision="mixed")
                if r["kind"] == "bubble":
                    kw["amp"] = r["amp"]
                tickets[i] = srv.submit(**kw)

        th = threading.Thread(target=submitter)
        t0 = time.perf_counter()
        th.start()
        th.join()
        res = [srv.wait(t, timeout=3600.0) for t in tickets]
        makespan = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        ok = [r for r in res if r["status"] == 0]
        lat = [r["t_finish"] - r["t_submit"] for r in ok]
        dof = sum(r["ndof"] * 5 * r["nsteps"] for r in ok)
        pt = {"rate_x_seq_fp64": mult, "rate_hz": rate, "completed": len(ok),
              "latency_p50_s": _pct(lat, 50), "latency_p99_s": _pct(lat, 99),
              "throughput": dof / makespan, "makespan_s": makespan,
              "sequential_fp64_value": seq_value,
              "throughput_over_sequential_fp64": dof / makespan / seq_value, "error": st["error"]}
        if check and mult == rates[-1]:
            small = sorted(range(len(stream)), key=lambda i: work(stream[i]))[:check]
            errs = []
            for i in small:
                r = stream[i]
                _, _, q64 = _sequential(dict(r, nsteps=r["steps"]), "fp64")
                errs.append({"request": i, "kind": r["kind"], "K": list(r["K"]), "N": r["N"],
                             "rel_err_rho_rhou_rhov_rhow_E": _state_errors(res[i]["q"], q64)})
            pt["mixed_vs_fp64_state_rel_err"] = errs
        points.append(pt)
    return {"metric": "serving p50/p99 solve latency and DOF-updates/s per RK stage",
            "unit": "s / DOF-updates/s", "higher_is_better": False, "n_gpus": 1,
            "config": {"workload": "poisson_serving", "requests": n_requests,
                       "steps_per_request": steps,
                       "mix": "70% bubbles K^3 (K 8..32), 30% channels (40s,8s,4s), N in {3,4,7}",
                       "precision": "mixed", "admission": "FIFO by HBM footprint",
                       "autotuner": "warmed for N in {3,4,7} before the stream"},
            "sequential_fp64_value": seq_value, "sequential_fp64_service_rate_hz": seq_rate,
            "points": points}


def run_serving(args):
    rates = tuple(float(x) for x in args.rates.split(","))
    steps = args.steps if args.steps_given else SERVING_DEFAULT["steps"]
    print(json.dumps(serving_measure(args.requests, steps, rates, args.calib, args.slots,
                                     args.budget_gb, check=args.check)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--K", type=int, default=0, help="elements per direction (small profiling cases)")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"])
    ap.add_argument("--workload", default="bubble32",
                    choices=["bubble32", "ensemble", "serving", "channel", "sharp", "slabs"])
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--check", type=int, default=2,
                    help="served requests also solved alone in FP64 and compared")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="leave the ensemble and serving objects out of the default line")
    ap.add_argument("--requests", type=int, default=60)
    ap.add_argument("--rates", default="0.25,0.5,1,2,4")
    ap.add_argument("--calib", type=int, default=6)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--budget-gb", type=int, default=200)
    args = ap.parse_args()
    args.steps_given = any(a == "--steps" or a.startswith("--steps=") for a in sys.argv[1:])
    if args.workload == "ensemble":
        run_ensemble(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "channel":
        run_channel(args)
        return
    if args.workload == "sharp":
        run_sharp(args)
        return
    if args.workload == "slabs":
        run_slabs(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
